// Instance, topology, memory slots, processing units, execution states,
// fence and counters of the HiCR C ABI (HiCR paper Sec. 3.1.1-3.1.5).
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <map>

#include <algorithm>
#include <atomic>
#include <thread>

#include "hicr_internal.h"

namespace hicr {

const void* builtin_fill_kernel();
const void* builtin_digest_kernel();

// HICR_LOG set (to anything but "0") in the environment: every recorded
// error is also printed to stderr as it happens.
void log_error(Instance* in, const std::string& msg) {
  if (in) in->last_err = msg;
  static const bool on = [] {
    const char* v = getenv("HICR_LOG");
    return v && *v && strcmp(v, "0") != 0;
  }();
  if (on) {
    fprintf(stderr, "hicr: %s\n", msg.c_str());
    fflush(stderr);
  }
}

hicr_status cuda_fail(Instance* in, cudaError_t e, const char* what) {
  log_error(in, std::string(what) + ": " + cudaGetErrorString(e));
  (void)cudaGetLastError();  // clear a non-sticky error
  return HICR_ERR_DEVICE;
}

// Writes one slot-table entry in stream order (kernel parameters are copied
// at launch, so no host buffer has to outlive the call).
__global__ void k_set_slot(DevTables dt, uint32_t id, uint64_t base, uint64_t size, uint32_t meta) {
  dt.slot_base[id] = base;
  dt.slot_size[id] = size;
  dt.slot_meta[id] = meta;
}

static hicr_status push_slot(Instance* in, uint32_t id) {
  const HostSlot& s = in->slots[id];
  k_set_slot<<<1, 1, 0, in->comm()>>>(in->dt, id, s.base, s.size, meta_pack(s.live ? 1 : 0, s.space, s.tag));
  HICR_CUDA(in, cudaGetLastError());
  return HICR_OK;
}

hicr_status record_done(Instance* in) {
  if (in->capturing) return HICR_OK;
  in->opaque = true;
  HICR_CUDA(in, cudaEventRecord(in->done_ev, in->comm()));
  return HICR_OK;
}

hicr_status record_signalled(Instance* in) {
  if (in->capturing) return HICR_OK;
  HICR_CUDA(in, cudaEventRecord(in->done_ev, in->comm()));
  return HICR_OK;
}

void note_signal(Instance* in, const uint64_t* mask) {
  if (in->capturing) {
    ++in->cap_sigs;
    return;
  }
  const uint64_t v = ++in->sig_issued;
  if (!mask) {
    in->any_sig = v;
    return;
  }
  for (int w = 0; w < TAG_WORDS; ++w)
    for (uint64_t m = mask[w]; m; m &= m - 1) in->tag_sig[w * 64 + __builtin_ctzll(m)] = v;
}

void tag_mask(const Instance* in, const hicr_op_t* ops, uint64_t count, uint64_t* mask) {
  for (uint64_t i = 0; i < count; ++i) {
    const uint32_t a = in->slots[ops[i].dst].tag, b = in->slots[ops[i].src].tag;
    mask[a >> 6] |= 1ull << (a & 63);
    mask[b >> 6] |= 1ull << (b & 63);
  }
}

// Wait until the device has emitted completion signal `target` (mapped host
// memory, written by the launch's last thread), or timeout. Spins first,
// then yields, then sleeps in short steps.
static hicr_status wait_signal(Instance* in, uint64_t target, uint64_t timeout_ns) {
  volatile unsigned long long* m = in->sig_mirror;
  if (*m >= target) return HICR_OK;
  const uint64_t t0 = now_ns();
  for (uint32_t spins = 0;; ++spins) {
    if (*m >= target) return HICR_OK;
    if ((spins & 63) == 0) {
      const uint64_t dt = now_ns() - t0;
      if (dt >= timeout_ns) return *m >= target ? HICR_OK : HICR_ERR_TIMEOUT;
      if (dt > WAIT_YIELD_NS) std::this_thread::sleep_for(std::chrono::microseconds(20));
      else if (dt > WAIT_SPIN_NS) std::this_thread::yield();
    }
  }
}

hicr_status wait_event(Instance* in, cudaEvent_t ev, uint64_t timeout_ns) {
  const uint64_t t0 = now_ns();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return HICR_OK;
    if (e != cudaErrorNotReady) return cuda_fail(in, e, "cudaEventQuery");
    const uint64_t dt = now_ns() - t0;
    if (dt >= timeout_ns) return HICR_ERR_TIMEOUT;
    if (dt > WAIT_YIELD_NS) std::this_thread::sleep_for(std::chrono::microseconds(20));
    else std::this_thread::yield();
  }
}

static bool valid_slot(const Instance* in, uint32_t id) {
  return id < in->slots.size() && in->slots[id].live;
}

hicr_status validate_op(const Instance* in, const hicr_op_t& op) {
  if (!valid_slot(in, op.dst) || !valid_slot(in, op.src)) return HICR_ERR_INVALID;
  const HostSlot& d = in->slots[op.dst];
  const HostSlot& s = in->slots[op.src];
  if (!pair_supported(in->support, d.space, s.space)) return HICR_ERR_UNSUPPORTED;
  if (op.src_off > s.size || op.n > s.size - op.src_off) return HICR_ERR_BOUNDS;
  if (op.dst_off > d.size || op.n > d.size - op.dst_off) return HICR_ERR_BOUNDS;
  if (op.dst == op.src && op.n > 0 && op.dst_off < op.src_off + op.n && op.src_off < op.dst_off + op.n)
    return HICR_ERR_OVERLAP;
  return HICR_OK;
}

// Cross-op hazard check of one epoch: the first op (in issue order) whose
// destination range intersects an earlier op's destination or source range
// on the same slot, or whose source range intersects an earlier destination.
// Earlier destinations are disjoint (else the check already stopped), so they
// are kept as a start->end map; earlier sources are kept as their union.
hicr_status first_hazard(const Instance* in, const hicr_op_t* ops, uint64_t count, uint64_t* bad) {
  (void)in;
  typedef std::map<uint64_t, uint64_t> Set;  // start -> end, disjoint
  std::unordered_map<uint32_t, Set> writes, reads;
  auto hits = [](const Set& m, uint64_t a, uint64_t b) {
    auto it = m.lower_bound(b);  // first interval starting at or after b
    if (it == m.begin()) return false;
    --it;                        // last interval starting before b
    return it->second > a;
  };
  auto add_union = [](Set& m, uint64_t a, uint64_t b) {
    auto it = m.upper_bound(a);
    if (it != m.begin()) {
      auto p = std::prev(it);
      if (p->second >= a) { a = p->first; b = std::max(b, p->second); it = m.erase(p); }
    }
    while (it != m.end() && it->first <= b) { b = std::max(b, it->second); it = m.erase(it); }
    m[a] = b;
  };
  for (uint64_t j = 0; j < count; ++j) {
    const hicr_op_t& o = ops[j];
    if (o.n == 0) continue;
    const uint64_t da = o.dst_off, db = o.dst_off + o.n, sa = o.src_off, sb = o.src_off + o.n;
    bool h = false;
    auto w = writes.find(o.dst);
    if (w != writes.end() && hits(w->second, da, db)) h = true;
    auto r = reads.find(o.dst);
    if (!h && r != reads.end() && hits(r->second, da, db)) h = true;
    auto ws = writes.find(o.src);
    if (!h && ws != writes.end() && hits(ws->second, sa, sb)) h = true;
    if (h) {
      *bad = j;
      return HICR_ERR_HAZARD;
    }
    writes[o.dst][da] = db;
    add_union(reads[o.src], sa, sb);
  }
  return HICR_OK;
}

}  // namespace hicr

using namespace hicr;

static Instance* I(hicr_instance_t h) { return h ? &h->impl : nullptr; }

extern "C" {

const char* hicr_status_str(hicr_status s) {
  switch (s) {
    case HICR_OK: return "HICR_OK";
    case HICR_ERR_INVALID: return "HICR_ERR_INVALID";
    case HICR_ERR_UNSUPPORTED: return "HICR_ERR_UNSUPPORTED";
    case HICR_ERR_BOUNDS: return "HICR_ERR_BOUNDS";
    case HICR_ERR_OVERLAP: return "HICR_ERR_OVERLAP";
    case HICR_ERR_HAZARD: return "HICR_ERR_HAZARD";
    case HICR_ERR_NOMEM: return "HICR_ERR_NOMEM";
    case HICR_ERR_FULL: return "HICR_ERR_FULL";
    case HICR_ERR_EMPTY: return "HICR_ERR_EMPTY";
    case HICR_ERR_TOO_LARGE: return "HICR_ERR_TOO_LARGE";
    case HICR_ERR_TIMEOUT: return "HICR_ERR_TIMEOUT";
    case HICR_ERR_BUSY: return "HICR_ERR_BUSY";
    case HICR_ERR_DEVICE: return "HICR_ERR_DEVICE";
    default: return "HICR_ERR_UNKNOWN";
  }
}

hicr_status hicr_init(int cuda_device, hicr_instance_t* out) {
  if (!out) return HICR_ERR_INVALID;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
    (void)cudaGetLastError();
    return HICR_ERR_INVALID;
  }
  hicr_instance_t h = new hicr_instance_s();
  Instance* in = &h->impl;
  in->device = cuda_device;
  auto fail = [&](hicr_status st) {
    delete h;
    return st;
  };
  if (cudaSetDevice(cuda_device) != cudaSuccess) return fail(HICR_ERR_DEVICE);
  if (cudaGetDeviceProperties(&in->prop, cuda_device) != cudaSuccess) return fail(HICR_ERR_DEVICE);
  in->sm_count = in->prop.multiProcessorCount;
  in->support = 1u << (HICR_SPACE_HBM * 8 + HICR_SPACE_HBM);

  // one allocation for all device tables
  const size_t S = HICR_MAX_SLOTS;
  size_t bytes = S * 8 * 2 + S * 4 + S * 8 * 2 + HICR_MAX_TAGS * 8 + 2 * 8 + 2 * 8;
  char* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return fail(HICR_ERR_NOMEM);
  if (cudaMemset(p, 0, bytes) != cudaSuccess) { cudaFree(p); return fail(HICR_ERR_DEVICE); }
  in->dt.slot_base = (uint64_t*)p; p += S * 8;
  in->dt.slot_size = (uint64_t*)p; p += S * 8;
  in->dt.sent = (unsigned long long*)p; p += S * 8;
  in->dt.recv = (unsigned long long*)p; p += S * 8;
  in->dt.tag_ops = (unsigned long long*)p; p += HICR_MAX_TAGS * 8;
  in->dt.sticky = (unsigned long long*)p; p += 2 * 8;
  in->dt.sig = (unsigned long long*)p; p += 2 * 8;
  in->dt.slot_meta = (uint32_t*)p;
  in->tag_sig.assign(HICR_MAX_TAGS, 0);
  in->tag_lat.assign(HICR_MAX_TAGS, 0);

  Pu pu0;
  if (cudaStreamCreateWithFlags(&pu0.stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(in->dt.slot_base);
    return fail(HICR_ERR_DEVICE);
  }
  pu0.owned = true;
  pu0.live = true;
  in->pus.push_back(pu0);
  cudaEventCreateWithFlags(&in->done_ev, cudaEventDisableTiming);
  if (cudaHostAlloc((void**)&in->sig_mirror, 64, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&in->dt.sig_host, in->sig_mirror, 0) != cudaSuccess)
    return fail(HICR_ERR_DEVICE);
  memset(in->sig_mirror, 0, 64);
  cudaEventCreateWithFlags(&in->pinned_ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&in->pinned_ev[1], cudaEventDisableTiming);
  cudaEventRecord(in->done_ev, pu0.stream);
  cudaEventRecord(in->pinned_ev[0], pu0.stream);
  cudaEventRecord(in->pinned_ev[1], pu0.stream);
  default_config(in, &in->cfg);
  if (noalloc_setup(in) != HICR_OK) {
    cudaFreeHost(in->sig_mirror);
    cudaStreamDestroy(pu0.stream);
    cudaFree(in->dt.slot_base);
    return fail(HICR_ERR_DEVICE);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(HICR_ERR_DEVICE);
  *out = h;
  return HICR_OK;
}

hicr_status hicr_finalize(hicr_instance_t h) {
  Instance* in = I(h);
  if (!in) return HICR_ERR_INVALID;
  cudaSetDevice(in->device);
  if (in->capturing) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(in->comm(), &g);
    if (g) cudaGraphDestroy(g);
  }
  // Outstanding work on the instance's streams gets a bounded wait: if it
  // does not finish, nothing is freed (it may still be in use) and the call
  // reports BUSY instead of blocking forever.
  {
    const uint64_t until = now_ns() + 30ull * 1000000000ull;
    bool busy = false;
    for (auto& p : in->pus) {
      if (!p.live) continue;
      while (cudaStreamQuery(p.stream) == cudaErrorNotReady) {
        if (now_ns() > until) {
          busy = true;
          break;
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
      }
      if (busy) break;
    }
    (void)cudaGetLastError();
    if (busy) {
      fprintf(stderr, "hicr_finalize: work still running after 30 s; instance left allocated\n");
      fflush(stderr);
      return HICR_ERR_BUSY;
    }
  }
  lat_destroy(in);
  cudaDeviceSynchronize();
  destroy_channels(in);
  destroy_servers(in);
  forget_data_objects(in);
  for (auto& g : in->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  for (auto& s : in->slots) {
    if (s.live && s.owned) {
      if (s.space == HICR_SPACE_HOST) cudaFreeHost(s.host_ptr);
      else cudaFree((void*)s.base);
    }
  }
  for (auto& kv : in->execs) cudaEventDestroy(kv.second);
  for (cudaEvent_t ev : in->exec_events) cudaEventDestroy(ev);
  for (auto e : in->prof_ev) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k) {
    if (in->pinned[k]) cudaFreeHost(in->pinned[k]);
    if (in->pinned_ev[k]) cudaEventDestroy(in->pinned_ev[k]);
  }
  if (in->d_ops) cudaFree(in->d_ops);
  if (in->scratch.cost) cudaFree(in->scratch.cost);
  if (in->dt.slot_base) cudaFree(in->dt.slot_base);
  if (in->done_ev) cudaEventDestroy(in->done_ev);
  if (in->sig_mirror) cudaFreeHost(in->sig_mirror);
  for (auto& p : in->pus)
    if (p.live && p.owned) cudaStreamDestroy(p.stream);
  delete h;
  return HICR_OK;
}

hicr_status hicr_is_root(hicr_instance_t h, int32_t* out) {
  if (!I(h) || !out) return HICR_ERR_INVALID;
  *out = 1;
  return HICR_OK;
}

hicr_status hicr_topology_query(hicr_instance_t h, hicr_topology_t* out) {
  Instance* in = I(h);
  if (!in || !out) return HICR_ERR_INVALID;
  hicr_topology_t t;
  memset(&t, 0, sizeof(t));
  t.device = in->device;
  strncpy(t.name, in->prop.name, sizeof(t.name) - 1);
  size_t fr = 0, tot = 0;
  HICR_CUDA(in, cudaMemGetInfo(&fr, &tot));
  t.n_spaces = 2;
  t.spaces[0].id = 0;
  t.spaces[0].kind = HICR_SPACE_HBM;
  t.spaces[0].device = in->device;
  t.spaces[0].phys_size = in->prop.totalGlobalMem;
  t.spaces[0].free_size = fr;
  {
    int clk_khz = 0, bus_bits = 0;
    if (cudaDeviceGetAttribute(&clk_khz, cudaDevAttrMemoryClockRate, in->device) == cudaSuccess &&
        cudaDeviceGetAttribute(&bus_bits, cudaDevAttrGlobalMemoryBusWidth, in->device) == cudaSuccess) {
      const unsigned long long mbps = 2ull * (unsigned long long)clk_khz * (unsigned long long)bus_bits / 8ull / 1000ull;
      t.spaces[0].peak_mbps = mbps > 0xffffffffull ? 0u : (uint32_t)mbps;
    } else {
      (void)cudaGetLastError();
    }
  }
  t.spaces[1].id = 1;
  t.spaces[1].kind = HICR_SPACE_HOST;
  t.spaces[1].device = -1;
  {
    // physical host memory (pages x page size)
    long pages = 0, psize = 0;
#ifdef _SC_PHYS_PAGES
    pages = sysconf(_SC_PHYS_PAGES);
    psize = sysconf(_SC_PAGE_SIZE);
#endif
    t.spaces[1].phys_size = (pages > 0 && psize > 0) ? (uint64_t)pages * (uint64_t)psize : 0;
  }
  t.n_resources = 1;
  hicr_compute_resource_t& r = t.resources[0];
  r.id = 0;
  r.kind = HICR_RESOURCE_GPU;
  r.device = in->device;
  r.sm_count = in->prop.multiProcessorCount;
  r.max_threads_per_sm = in->prop.maxThreadsPerMultiProcessor;
  r.cc_major = in->prop.major;
  r.cc_minor = in->prop.minor;
  r.l2_bytes = in->prop.l2CacheSize;
  r.smem_per_block_optin = in->prop.sharedMemPerBlockOptin;
  *out = t;
  return HICR_OK;
}

static hicr_status new_slot(Instance* in, const HostSlot& s, hicr_slot_t* out) {
  uint32_t id;
  if (!in->free_ids.empty()) {
    id = in->free_ids.back();
    in->free_ids.pop_back();
    in->slots[id] = s;
  } else {
    if (in->slots.size() >= HICR_MAX_SLOTS) return HICR_ERR_INVALID;
    id = (uint32_t)in->slots.size();
    in->slots.push_back(s);
  }
  hicr_status st = push_slot(in, id);
  if (st != HICR_OK) {
    in->slots[id].live = false;
    in->free_ids.push_back(id);
    return st;
  }
  *out = id;
  return HICR_OK;
}

hicr_status hicr_mem_alloc(hicr_instance_t h, uint32_t space, uint64_t size, uint32_t tag, hicr_slot_t* out) {
  Instance* in = I(h);
  if (!in || !out || size == 0 || tag >= HICR_MAX_TAGS || in->capturing) return HICR_ERR_INVALID;
  if (space != HICR_SPACE_HBM && space != HICR_SPACE_HOST) return HICR_ERR_INVALID;
  if (in->slots.size() >= HICR_MAX_SLOTS && in->free_ids.empty()) return HICR_ERR_INVALID;
  HostSlot s;
  s.size = size;
  s.space = space;
  s.tag = tag;
  s.live = true;
  s.owned = true;
  if (space == HICR_SPACE_HBM) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, size);
    if (e == cudaErrorMemoryAllocation) { (void)cudaGetLastError(); return HICR_ERR_NOMEM; }
    HICR_CUDA(in, e);
    s.base = (uint64_t)p;
    s.host_ptr = nullptr;
  } else {
    void* p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, size, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaErrorMemoryAllocation) { (void)cudaGetLastError(); return HICR_ERR_NOMEM; }
    HICR_CUDA(in, e);
    void* dp = nullptr;
    HICR_CUDA(in, cudaHostGetDevicePointer(&dp, p, 0));
    s.base = (uint64_t)dp;
    s.host_ptr = p;
  }
  hicr_status st = new_slot(in, s, out);
  if (st != HICR_OK) {
    if (space == HICR_SPACE_HOST) cudaFreeHost(s.host_ptr);
    else cudaFree((void*)s.base);
  }
  return st;
}

hicr_status hicr_mem_free(hicr_instance_t h, hicr_slot_t slot) {
  Instance* in = I(h);
  if (!in || in->capturing || !valid_slot(in, slot) || !in->slots[slot].owned) return HICR_ERR_INVALID;
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  if (in->lat_ring) {
    // ops the latency-mode server still holds may touch the slot; a stopped
    // server does not keep the device synchronisation below waiting
    hicr_status ls = lat_wait(in, in->lat_head, 60ull * 1000000000ull);
    if (ls == HICR_OK) ls = lat_stop(in);
    if (ls != HICR_OK) return ls;
  }
  HICR_CUDA(in, cudaDeviceSynchronize());
  HostSlot& s = in->slots[slot];
  if (s.space == HICR_SPACE_HOST) cudaFreeHost(s.host_ptr);
  else cudaFree((void*)s.base);
  s = HostSlot();
  hicr_status st = push_slot(in, slot);
  in->free_ids.push_back(slot);
  return st;
}

hicr_status hicr_slot_register(hicr_instance_t h, uint32_t space, void* ptr, uint64_t size, uint32_t tag,
                               hicr_slot_t* out) {
  Instance* in = I(h);
  if (!in || !out || (ptr == nullptr && size > 0) || tag >= HICR_MAX_TAGS || in->capturing)
    return HICR_ERR_INVALID;
  if (space != HICR_SPACE_HBM && space != HICR_SPACE_HOST) return HICR_ERR_INVALID;
  HostSlot s;
  s.size = size;
  s.space = space;
  s.tag = tag;
  s.live = true;
  s.owned = false;
  s.base = (uint64_t)ptr;
  s.host_ptr = space == HICR_SPACE_HOST ? ptr : nullptr;
  if (space == HICR_SPACE_HOST && ptr) {
    // page-locked host memory must be reachable from the device
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess || a.devicePointer == nullptr) {
      (void)cudaGetLastError();
      return HICR_ERR_INVALID;
    }
    s.base = (uint64_t)a.devicePointer;
  }
  return new_slot(in, s, out);
}

hicr_status hicr_slot_deregister(hicr_instance_t h, hicr_slot_t slot) {
  Instance* in = I(h);
  if (!in || in->capturing || !valid_slot(in, slot) || in->slots[slot].owned) return HICR_ERR_INVALID;
  if (!in->queue.empty()) return HICR_ERR_BUSY;
  if (in->lat_ring && *(volatile unsigned long long*)&in->lat_ring->done < in->lat_head) return HICR_ERR_BUSY;
  cudaError_t e = cudaEventQuery(in->done_ev);
  // A fence returns at the completion signal, which the last thread of a
  // launch writes just before the kernel ends: when every signal issued is
  // in and nothing else is pending, the done event follows within moments.
  if (e == cudaErrorNotReady && !in->opaque && *(volatile unsigned long long*)in->sig_mirror >= in->sig_issued)
    e = cudaEventSynchronize(in->done_ev);
  if (e == cudaErrorNotReady) return HICR_ERR_BUSY;
  HICR_CUDA(in, e);
  in->slots[slot] = HostSlot();
  hicr_status st = push_slot(in, slot);
  in->free_ids.push_back(slot);
  return st;
}

hicr_status hicr_slot_info(hicr_instance_t h, hicr_slot_t slot, void** ptr, uint64_t* size, uint32_t* space,
                           uint32_t* tag) {
  Instance* in = I(h);
  if (!in || !valid_slot(in, slot)) return HICR_ERR_INVALID;
  const HostSlot& s = in->slots[slot];
  if (ptr) *ptr = s.space == HICR_SPACE_HOST ? s.host_ptr : (void*)s.base;
  if (size) *size = s.size;
  if (space) *space = s.space;
  if (tag) *tag = s.tag;
  return HICR_OK;
}

// Wait for the work fences must cover: when work without completion signals
// was issued on the communication stream since the last full wait, the done
// event covers everything once; then completion signal `target`. Returns the
// sticky batch error the device mirrored with the last signal, if any.
static hicr_status fence_wait(hicr_instance_t h, Instance* in, uint64_t target, uint64_t timeout_ns) {
  const uint64_t t0 = now_ns();
  if (in->opaque) {
    HICR_CUDA(in, cudaEventRecord(in->done_ev, in->comm()));
    hicr_status st = wait_event(in, in->done_ev, timeout_ns);
    if (st != HICR_OK) return st;
    in->opaque = false;
  }
  const uint64_t used = now_ns() - t0;
  hicr_status st = wait_signal(in, target, timeout_ns > used ? timeout_ns - used : 0);
  if (st != HICR_OK) return st;
  std::atomic_thread_fence(std::memory_order_acquire);
  if (*(volatile unsigned long long*)(in->sig_mirror + 1) == 0) return HICR_OK;
  hicr_status bst = HICR_OK;
  uint64_t bad = 0;
  st = hicr_batch_error(h, &bst, &bad);  // reads and clears it
  if (st != HICR_OK) return st;
  return bst;
}

hicr_status hicr_fence(hicr_instance_t h, uint32_t tag, uint64_t timeout_ns) {
  hicr::NvtxRange nvtx_range("hicr_fence");
  Instance* in = I(h);
  if (!in || tag >= HICR_MAX_TAGS || in->capturing) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  // Every memcpy launch ends with a completion signal; the host knows the
  // signal of the last launch with an op of this tag (or of unknown tags).
  // Later launches of other tags are not waited for.
  const uint64_t t0 = now_ns();
  st = lat_wait(in, in->tag_lat[tag], timeout_ns);  // small batches the latency-mode server took
  if (st != HICR_OK) return st;
  const uint64_t used = now_ns() - t0;
  return fence_wait(h, in, std::max(in->tag_sig[tag], in->any_sig), timeout_ns > used ? timeout_ns - used : 0);
}

static hicr_status read_u64_pair(Instance* in, const unsigned long long* a, const unsigned long long* b,
                                 uint64_t* x, uint64_t* y) {
  unsigned long long v[2] = {0, 0};
  // Synchronous device reads on the legacy stream would wait for other
  // blocking streams; a plain cudaMemcpy of 8 bytes is enough here because
  // the communication stream is non-blocking.
  HICR_CUDA(in, cudaMemcpy(&v[0], a, 8, cudaMemcpyDeviceToHost));
  if (b) HICR_CUDA(in, cudaMemcpy(&v[1], b, 8, cudaMemcpyDeviceToHost));
  if (x) *x = v[0];
  if (y) *y = v[1];
  return HICR_OK;
}

hicr_status hicr_slot_counters(hicr_instance_t h, hicr_slot_t slot, uint64_t* sent, uint64_t* recv) {
  Instance* in = I(h);
  if (!in || slot >= HICR_MAX_SLOTS || slot >= in->slots.size()) return HICR_ERR_INVALID;
  return read_u64_pair(in, in->dt.sent + slot, in->dt.recv + slot, sent, recv);
}

hicr_status hicr_slot_counters_range(hicr_instance_t h, hicr_slot_t first, uint32_t count, uint64_t* sent,
                                     uint64_t* recv) {
  Instance* in = I(h);
  if (!in || (uint64_t)first + count > HICR_MAX_SLOTS) return HICR_ERR_INVALID;
  if (count == 0) return HICR_OK;
  if (sent) HICR_CUDA(in, cudaMemcpy(sent, in->dt.sent + first, 8ull * count, cudaMemcpyDeviceToHost));
  if (recv) HICR_CUDA(in, cudaMemcpy(recv, in->dt.recv + first, 8ull * count, cudaMemcpyDeviceToHost));
  return HICR_OK;
}

hicr_status hicr_tag_counter(hicr_instance_t h, uint32_t tag, uint64_t* ops) {
  Instance* in = I(h);
  if (!in || tag >= HICR_MAX_TAGS || !ops) return HICR_ERR_INVALID;
  return read_u64_pair(in, in->dt.tag_ops + tag, nullptr, ops, nullptr);
}

hicr_status hicr_fence_slot(hicr_instance_t h, hicr_slot_t slot, uint64_t expect_sent, uint64_t expect_recv,
                            uint64_t timeout_ns) {
  hicr::NvtxRange nvtx_range("hicr_fence_slot");
  Instance* in = I(h);
  if (!in || slot >= in->slots.size() || in->capturing) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  // Only launches with an op of the slot's tag can move its counters: wait
  // for the last of them (polling mapped host memory), then read the
  // counters once. If they fall short, no issued op can still raise them.
  const uint32_t tag = in->slots[slot].tag;
  if ((st = lat_wait(in, in->tag_lat[tag], timeout_ns)) != HICR_OK) return st;
  st = fence_wait(h, in, std::max(in->tag_sig[tag], in->any_sig), timeout_ns);
  if (st != HICR_OK) return st;
  uint64_t s = 0, r = 0;
  st = hicr_slot_counters(h, slot, &s, &r);
  if (st != HICR_OK) return st;
  return (s >= expect_sent && r >= expect_recv) ? HICR_OK : HICR_ERR_TIMEOUT;
}

hicr_status hicr_batch_error(hicr_instance_t h, hicr_status* status, uint64_t* first_bad) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  unsigned long long v = 0;
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  HICR_CUDA(in, cudaMemcpy(&v, in->dt.sticky, 8, cudaMemcpyDeviceToHost));
  if (v != 0) {
    unsigned long long z = 0;
    HICR_CUDA(in, cudaMemcpy(in->dt.sticky, &z, 8, cudaMemcpyHostToDevice));
  }
  // the stream is idle: no signal can be writing the mirror now
  *(volatile unsigned long long*)(in->sig_mirror + 1) = 0;
  if (status) *status = v ? -(hicr_status)(v & 0xFF) : HICR_OK;
  if (first_bad) *first_bad = v ? (v >> 8) : 0;
  return HICR_OK;
}

hicr_status hicr_set_host_copies(hicr_instance_t h, int32_t on) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  const uint32_t hbm = 1u << (HICR_SPACE_HBM * 8 + HICR_SPACE_HBM);
  const uint32_t host = (1u << (HICR_SPACE_HBM * 8 + HICR_SPACE_HOST)) | (1u << (HICR_SPACE_HOST * 8 + HICR_SPACE_HBM)) |
                        (1u << (HICR_SPACE_HOST * 8 + HICR_SPACE_HOST));
  in->support = on ? (hbm | host) : hbm;
  return HICR_OK;
}

hicr_status hicr_set_checked(hicr_instance_t h, int32_t on) {
  Instance* in = I(h);
  if (!in) return HICR_ERR_INVALID;
  in->checked = on ? 1 : 0;
  return HICR_OK;
}

// --- processing units ------------------------------------------------------

hicr_status hicr_pu_create(hicr_instance_t h, void* stream, hicr_pu_t* out) {
  Instance* in = I(h);
  if (!in || !out) return HICR_ERR_INVALID;
  Pu p;
  if (stream) {
    p.stream = (cudaStream_t)stream;
    p.owned = false;
  } else {
    HICR_CUDA(in, cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking));
    p.owned = true;
  }
  p.live = true;
  for (uint32_t i = 1; i < in->pus.size(); ++i) {
    if (!in->pus[i].live) {
      in->pus[i] = p;
      *out = i;
      return HICR_OK;
    }
  }
  if (in->pus.size() >= HICR_MAX_PUS) {
    if (p.owned) cudaStreamDestroy(p.stream);
    return HICR_ERR_INVALID;
  }
  in->pus.push_back(p);
  *out = (hicr_pu_t)(in->pus.size() - 1);
  return HICR_OK;
}

hicr_status hicr_pu_destroy(hicr_instance_t h, hicr_pu_t pu) {
  Instance* in = I(h);
  if (!in || pu == 0 || pu >= in->pus.size() || !in->pus[pu].live || pu == in->comm_pu) return HICR_ERR_INVALID;
  HICR_CUDA(in, cudaStreamSynchronize(in->pus[pu].stream));
  if (in->pus[pu].owned) cudaStreamDestroy(in->pus[pu].stream);
  in->pus[pu] = Pu();
  return HICR_OK;
}

hicr_status hicr_pu_stream(hicr_instance_t h, hicr_pu_t pu, void** stream) {
  Instance* in = I(h);
  if (!in || !stream || pu >= in->pus.size() || !in->pus[pu].live) return HICR_ERR_INVALID;
  *stream = (void*)in->pus[pu].stream;
  return HICR_OK;
}

hicr_status hicr_comm_set_pu(hicr_instance_t h, hicr_pu_t pu) {
  Instance* in = I(h);
  if (!in || in->capturing || pu >= in->pus.size() || !in->pus[pu].live) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  // Batches share scratch memory: let the old stream drain before the new
  // one can start a batch.
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  in->comm_pu = pu;
  return record_done(in);
}

// --- execution units / states ---------------------------------------------

hicr_status hicr_exec_unit_builtin(const char* name, hicr_exec_unit_t* out) {
  if (!name || !out) return HICR_ERR_INVALID;
  hicr_exec_unit_t u;
  memset(&u, 0, sizeof(u));
  u.grid[0] = 1184;
  u.grid[1] = u.grid[2] = 1;
  u.block[0] = 256;
  u.block[1] = u.block[2] = 1;
  if (strcmp(name, "fill_seeded") == 0) {
    u.func = builtin_fill_kernel();
    u.n_args = 4;
  } else if (strcmp(name, "digest_words") == 0) {
    u.func = builtin_digest_kernel();
    u.n_args = 3;
  } else {
    return HICR_ERR_INVALID;
  }
  *out = u;
  return HICR_OK;
}

hicr_status hicr_exec_launch(hicr_instance_t h, hicr_pu_t pu, const hicr_exec_unit_t* u, void** args,
                             hicr_exec_t* out) {
  Instance* in = I(h);
  if (!in || !u || !u->func || !out || pu >= in->pus.size() || !in->pus[pu].live) return HICR_ERR_INVALID;
  if (u->grid[0] == 0 || u->grid[1] == 0 || u->grid[2] == 0 || u->block[0] == 0 || u->block[1] == 0 ||
      u->block[2] == 0)
    return HICR_ERR_INVALID;
  if (u->n_args > 0 && !args) return HICR_ERR_INVALID;
  cudaStream_t st = in->pus[pu].stream;
  if (pu == in->comm_pu) in->opaque = true;  // fences on this stream wait for it once
  HICR_CUDA(in, cudaLaunchKernel(u->func, dim3(u->grid[0], u->grid[1], u->grid[2]),
                                 dim3(u->block[0], u->block[1], u->block[2]), args, u->smem_bytes, st));
  // completion event: one returned by an earlier await, else a new one
  cudaEvent_t ev;
  if (!in->exec_events.empty()) {
    ev = in->exec_events.back();
    in->exec_events.pop_back();
  } else {
    HICR_CUDA(in, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  cudaError_t e = cudaEventRecord(ev, st);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_fail(in, e, "cudaEventRecord");
  }
  uint64_t id = in->next_exec++;
  in->execs[id] = ev;
  *out = id;
  return HICR_OK;
}

hicr_status hicr_exec_query(hicr_instance_t h, hicr_exec_t e, int32_t* done) {
  Instance* in = I(h);
  if (!in || !done) return HICR_ERR_INVALID;
  auto it = in->execs.find(e);
  if (it == in->execs.end()) return HICR_ERR_INVALID;
  cudaError_t r = cudaEventQuery(it->second);
  if (r == cudaErrorNotReady) {
    *done = 0;
    return HICR_OK;
  }
  HICR_CUDA(in, r);
  *done = 1;
  return HICR_OK;
}

hicr_status hicr_exec_await(hicr_instance_t h, hicr_exec_t e, uint64_t timeout_ns) {
  Instance* in = I(h);
  if (!in) return HICR_ERR_INVALID;
  auto it = in->execs.find(e);
  if (it == in->execs.end()) return HICR_ERR_INVALID;
  hicr_status st = wait_event(in, it->second, timeout_ns);
  if (st != HICR_OK) return st;
  in->exec_events.push_back(it->second);
  in->execs.erase(it);
  return HICR_OK;
}

hicr_status hicr_last_error_string(hicr_instance_t h, char* buf, uint64_t len) {
  Instance* in = I(h);
  if (!in || !buf || len == 0) return HICR_ERR_INVALID;
  size_t n = std::min<size_t>(len - 1, in->last_err.size());
  memcpy(buf, in->last_err.data(), n);
  buf[n] = 0;
  return HICR_OK;
}

}  // extern "C"
