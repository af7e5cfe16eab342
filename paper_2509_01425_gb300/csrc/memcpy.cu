// Batched local-to-local memcpy between memory slots (HiCR paper Sec. 3.1.4,
// "memcpy" and "fence"; Fig. 5). One batch = these steps on the
// communication stream (k_plan_scan fuses the first two on the main path;
// the allocation-free entry runs them as two kernels):
//
//   k_plan  (grid over ops)  validate each op against the device slot table
//                            with the same rules as the host, charge it
//                            cost = n + op_cost, zero its piece counter;
//   k_scan  (one CTA)        exclusive prefix sum of the costs, chunk count,
//                            first bad op -> the batch copies nothing and the
//                            error is left for the next fence;
//   k_copy  (persistent)     (or k_copy_tma, the bulk-copy engine)
//                            every warp repeatedly claims a chunk of
//                            `chunk` cost units, finds the op holding its
//                            first unit by a 32-ary search of the prefix sums,
//                            and copies the byte pieces of every op the chunk
//                            overlaps. The warp that finishes an op's last
//                            piece bumps sent[src], recv[dst] and the tag
//                            counters (the message counters fence reads).
//
// The cost model (bytes + a fixed per-op charge) is the size binning: large
// ops are cut into many chunks that different warps copy in parallel, runs of
// small ops are packed into one chunk, and the per-op charge keeps a warp
// from being handed too many tiny ops at once.
//
// Host-validated batches of a few small ops skip all of this: k_copy_small
// takes them as kernel parameters (see SMALL_OPS).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "copy.cuh"
#include "hicr_internal.h"

namespace hicr {

static constexpr unsigned FULL = 0xffffffffu;
static constexpr unsigned long long NO_BAD = ~0ull;

// ---------------------------------------------------------------------------
// Validation on the device: the rules of validate_op() in runtime.cu.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dev_validate(const DevTables& dt, unsigned support, const hicr_op_t& op) {
  if (op.dst >= HICR_MAX_SLOTS || op.src >= HICR_MAX_SLOTS) return HICR_ERR_INVALID;
  const uint32_t md = dt.slot_meta[op.dst], ms = dt.slot_meta[op.src];
  if (!meta_live(md) || !meta_live(ms)) return HICR_ERR_INVALID;
  if (!pair_supported(support, meta_space(md), meta_space(ms))) return HICR_ERR_UNSUPPORTED;
  const uint64_t ds = dt.slot_size[op.dst], ss = dt.slot_size[op.src];
  if (op.src_off > ss || op.n > ss - op.src_off) return HICR_ERR_BOUNDS;
  if (op.dst_off > ds || op.n > ds - op.dst_off) return HICR_ERR_BOUNDS;
  if (op.dst == op.src && op.n > 0 && op.dst_off < op.src_off + op.n && op.src_off < op.dst_off + op.n)
    return HICR_ERR_OVERLAP;
  return HICR_OK;
}

__global__ void k_plan(BatchArgs a) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const hicr_op_t op = a.ops[i];
  const int st = dev_validate(a.dt, a.support, op);
  if (st != HICR_OK) atomicMin(&a.ctrl->bad, (i << 8) | (unsigned long long)(-st));
  a.cost[i] = op.n + a.op_cost;
  a.done[i] = 0;
}

// Single-CTA exclusive scan (1024 threads): thread t sums a contiguous run
// of ceil(count / 1024) costs, the 1024 run totals are scanned with warp
// shuffles, then every run is written out.
__global__ void __launch_bounds__(1024) k_scan(BatchArgs a) {
  __shared__ unsigned long long warp_tot[32];
  const unsigned t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned long long n = a.count;
  const unsigned long long per = (n + 1023) / 1024;
  const unsigned long long b = per * t, e = min(n, b + per);
  unsigned long long s = 0;
  for (unsigned long long i = b; i < e; ++i) s += a.cost[i];
  // inclusive scan within the warp
  unsigned long long x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(FULL, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long v = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(FULL, v, o);
      if (lane >= (unsigned)o) v += y;
    }
    warp_tot[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  unsigned long long run = x - s + (w ? warp_tot[w - 1] : 0ull);  // exclusive start of this run
  for (unsigned long long i = b; i < e; ++i) {
    a.cstart[i] = run;
    run += a.cost[i];
  }
  if (t == 1023) {
    const unsigned long long total = warp_tot[31];
    a.cstart[n] = total;
    const unsigned long long bad = a.ctrl->bad;
    a.ctrl->total = total;
    a.ctrl->claim = 0;
    a.ctrl->exited = 0;
    if (bad != NO_BAD) {
      a.ctrl->nchunks = 0;
      // keep the first failure until a fence reads it
      atomicCAS(a.dt.sticky, 0ull, bad);
    } else {
      a.ctrl->nchunks = (total + a.chunk - 1) / a.chunk;
    }
    a.ctrl->bad = NO_BAD;  // ready for the next batch
  }
}

// Fused plan + scan for the main path: one CTA per tile of PS_TILE ops
// (tiles numbered in the order CTAs start, by an atomic counter). Each CTA
// validates and costs its ops, scans them in the block and chains the tile
// prefixes by decoupled look-back: a tile publishes its aggregate, sums
// predecessors' aggregates until it reaches a published inclusive prefix,
// then publishes its own inclusive prefix. Predecessors started earlier, so
// the look-back always progresses; it is still bounded by a deadline. The
// look-back words and the tile counter are zeroed before each batch (memset).
// The last tile finishes the batch as k_scan does.
static constexpr unsigned PS_THREADS = 256, PS_ITEMS = 8, PS_TILE = PS_THREADS * PS_ITEMS;
static constexpr unsigned long long PS_AGG = 1ull << 62, PS_INC = 2ull << 62, PS_VAL = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ps_ld_acq(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void ps_st_rel(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ps_time() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(PS_THREADS) k_plan_scan(BatchArgs a, unsigned long long* tiles,
                                                           unsigned long long n_tiles) {
  __shared__ unsigned long long s_tile, s_prefix, s_warp[PS_THREADS / 32];
  const unsigned t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned int* tile_ctr = reinterpret_cast<unsigned int*>(tiles + n_tiles);
  if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const unsigned long long tile = s_tile;
  const unsigned long long n = a.count;
  const unsigned long long i0 = tile * PS_TILE + (unsigned long long)t * PS_ITEMS;
  unsigned long long c[PS_ITEMS];
  unsigned long long sum = 0;
#pragma unroll
  for (int j = 0; j < (int)PS_ITEMS; ++j) {
    const unsigned long long i = i0 + j;
    c[j] = 0;
    if (i < n) {
      const hicr_op_t op = a.ops[i];
      const int st = dev_validate(a.dt, a.support, op);
      if (st != HICR_OK) atomicMin(&a.ctrl->bad, (i << 8) | (unsigned long long)(-st));
      c[j] = op.n + a.op_cost;
      a.done[i] = 0;
    }
    sum += c[j];
  }
  // block exclusive scan of the per-thread sums
  unsigned long long x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __threadfence();  // this thread's validation results before the tile is published
  __syncthreads();
  if (t == 0) {
    unsigned long long acc = 0;
    for (unsigned k = 0; k < PS_THREADS / 32; ++k) {
      const unsigned long long v = s_warp[k];
      s_warp[k] = acc;
      acc += v;
    }
    const unsigned long long agg = acc;
    unsigned long long prefix = 0;
    if (tile == 0) {
      ps_st_rel(&tiles[0], PS_INC | agg);
    } else {
      ps_st_rel(&tiles[tile], PS_AGG | agg);
      const unsigned long long deadline = ps_time() + 10000000000ull;
      for (unsigned long long p = tile; p-- > 0;) {
        unsigned long long v;
        for (;;) {
          v = ps_ld_acq(&tiles[p]);
          if (v >> 62) break;
          if (ps_time() > deadline) break;
          __nanosleep(32);
        }
        if (!(v >> 62)) {  // predecessor never published: fail the batch, do not hang
          atomicMin(&a.ctrl->bad, (0ull << 8) | (unsigned long long)(-HICR_ERR_TIMEOUT));
          break;
        }
        prefix += v & PS_VAL;
        if ((v >> 62) == 2) break;
      }
      ps_st_rel(&tiles[tile], PS_INC | (prefix + agg));
    }
    s_prefix = prefix;
    s_tile = agg;  // reuse: the tile aggregate
  }
  __syncthreads();
  unsigned long long run = s_prefix + s_warp[w] + (x - sum);
#pragma unroll
  for (int j = 0; j < (int)PS_ITEMS; ++j) {
    const unsigned long long i = i0 + j;
    if (i < n) a.cstart[i] = run;
    run += c[j];
  }
  const unsigned long long last = (n + PS_TILE - 1) / PS_TILE - 1;
  if (tile == last && t == 0) {
    const unsigned long long total = s_prefix + s_tile;
    a.cstart[n] = total;
    const unsigned long long bad = atomicAdd(&a.ctrl->bad, 0ull);
    a.ctrl->total = total;
    a.ctrl->claim = 0;
    a.ctrl->exited = 0;
    if (bad != NO_BAD) {
      a.ctrl->nchunks = 0;
      atomicCAS(a.dt.sticky, 0ull, bad);
    } else {
      a.ctrl->nchunks = (total + a.chunk - 1) / a.chunk;
    }
    a.ctrl->bad = NO_BAD;
  }
}

__device__ __forceinline__ void op_complete(const BatchArgs& a, const hicr_op_t& op) {
  __threadfence();
  atomicAdd(&a.dt.sent[op.src], 1ull);
  atomicAdd(&a.dt.recv[op.dst], 1ull);
  const uint32_t ts = meta_tag(a.dt.slot_meta[op.src]);
  const uint32_t td = meta_tag(a.dt.slot_meta[op.dst]);
  atomicAdd(&a.dt.tag_ops[ts], 1ull);
  if (td != ts) atomicAdd(&a.dt.tag_ops[td], 1ull);
}

__global__ void __launch_bounds__(1024) k_copy(BatchArgs a) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long nchunks = *(volatile unsigned long long*)&a.ctrl->nchunks;
  const unsigned long long total = *(volatile unsigned long long*)&a.ctrl->total;
  const unsigned long long chunk = a.chunk;
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(&a.ctrl->claim, 1ull);
    c = __shfl_sync(FULL, c, 0);
    if (c >= nchunks) break;
    const unsigned long long lo = c * chunk;
    const unsigned long long hi = min(lo + chunk, total);
    for (unsigned long long i = find_op(a.cstart, a.count, lo, lane); i < a.count; ++i) {
      const unsigned long long cs = a.cstart[i];
      if (cs >= hi) break;
      const hicr_op_t op = a.ops[i];
      const unsigned long long bs = cs + a.op_cost;  // cost coordinate of byte 0
      const unsigned long long be = bs + op.n;       // == cstart[i + 1]
      const unsigned long long b0 = lo > bs ? lo - bs : 0ull;
      const unsigned long long b1 = (hi < be ? hi : be) > bs ? (hi < be ? hi : be) - bs : 0ull;
      if (b1 > b0) {
        uint8_t* d = reinterpret_cast<uint8_t*>(a.dt.slot_base[op.dst]) + op.dst_off + b0;
        const uint8_t* s = reinterpret_cast<const uint8_t*>(a.dt.slot_base[op.src]) + op.src_off + b0;
        warp_copy(d, s, b1 - b0, lane);
      }
      // this chunk's piece of op i is done
      const unsigned pieces = (unsigned)((be - 1) / chunk - cs / chunk + 1);
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        const unsigned prev = atomicAdd(&a.done[i], 1u);
        if (prev + 1 == pieces) op_complete(a, op);
      }
    }
  }
  copy_exit(a, lane);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

void default_config(Instance* in, hicr_batch_config_t* c) {
  memset(c, 0, sizeof(*c));
  c->chunk_bytes = 64 * 1024;
  c->op_cost_bytes = 2048;
  c->blocks_per_sm = 2;
  c->threads = 512;
  c->engine = 0;
  c->tma_min_bytes = 32 * 1024;
  (void)in;
}

hicr_status check_config(const Instance* in, const hicr_batch_config_t* c) {
  (void)in;
  if (c->chunk_bytes < 1024 || c->chunk_bytes % 1024 || c->chunk_bytes > (64u << 20)) return HICR_ERR_INVALID;
  if (c->op_cost_bytes < 1 || c->op_cost_bytes > (1u << 20)) return HICR_ERR_INVALID;
  if (c->blocks_per_sm < 1 || c->blocks_per_sm > 32) return HICR_ERR_INVALID;
  if (c->threads < 32 || c->threads > 1024 || c->threads % 32) return HICR_ERR_INVALID;
  if (c->engine > 1) return HICR_ERR_INVALID;
  if (c->tma_min_bytes < 1024) return HICR_ERR_INVALID;
  if (!copy_tma_shape_valid(*c)) return HICR_ERR_INVALID;
  if (c->engine == 1) {
    // the TMA engine's stages must fit: blocks_per_sm CTAs resident per SM
    int per_sm = 0;
    if (copy_tma_prepare(const_cast<Instance*>(in), *c, &per_sm) != HICR_OK) return HICR_ERR_DEVICE;
    if (per_sm < (int)c->blocks_per_sm) return HICR_ERR_INVALID;
  }
  return HICR_OK;
}

hicr_status ensure_scratch(Instance* in, uint64_t count) {
  if (count <= in->scratch.cap && in->scratch.cost) return HICR_OK;
  if (in->capturing) return HICR_ERR_INVALID;
  uint64_t cap = std::max<uint64_t>(count, 1024);
  cap = std::max<uint64_t>(cap, in->scratch.cap * 2 > cap ? std::min<uint64_t>(in->scratch.cap * 2, cap * 2) : cap);
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  if (in->scratch.cost) cudaFree(in->scratch.cost);
  in->scratch = Scratch();
  const uint64_t n_tiles = (cap + PS_TILE - 1) / PS_TILE + 1;
  const size_t ctrl_off = ((cap * 8 + (cap + 1) * 8 + cap * 4 + 63) / 64) * 64;
  const size_t tiles_off = ((ctrl_off + sizeof(BatchCtrl) + 255) / 256) * 256;
  const size_t bytes = tiles_off + (n_tiles + 1) * 8;
  char* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    return HICR_ERR_NOMEM;
  }
  HICR_CUDA(in, e);
  in->scratch.cap = cap;
  in->scratch.cost = (unsigned long long*)p;
  in->scratch.cstart = (unsigned long long*)(p + cap * 8);
  in->scratch.done = (unsigned int*)(p + cap * 8 + (cap + 1) * 8);
  in->scratch.ctrl = (BatchCtrl*)(p + ctrl_off);
  in->scratch.tiles = (unsigned long long*)(p + tiles_off);
  in->scratch.n_tiles = n_tiles;
  BatchCtrl init;
  init.claim = 0;
  init.nchunks = 0;
  init.total = 0;
  init.bad = NO_BAD;
  init.exited = 0;
  HICR_CUDA(in, cudaMemcpy(in->scratch.ctrl, &init, sizeof(init), cudaMemcpyHostToDevice));
  return HICR_OK;
}

static BatchArgs make_args(Instance* in, const hicr_op_t* d_ops, uint64_t count) {
  BatchArgs a;
  a.ops = d_ops;
  a.count = count;
  a.dt = in->dt;
  a.cost = in->scratch.cost;
  a.cstart = in->scratch.cstart;
  a.done = in->scratch.done;
  a.ctrl = in->scratch.ctrl;
  a.chunk = in->cfg.chunk_bytes;
  a.op_cost = in->cfg.op_cost_bytes;
  a.support = in->support;
  a.engine = in->cfg.engine;
  a.tma_min = in->cfg.tma_min_bytes;
  a.tma_stage = 0;
  return a;
}

static hicr_status prof_event(Instance* in, cudaEvent_t* ev) {
  if (in->prof_used >= in->prof_ev.size()) {
    cudaEvent_t e;
    HICR_CUDA(in, cudaEventCreate(&e));
    in->prof_ev.push_back(e);
  }
  *ev = in->prof_ev[in->prof_used++];
  return HICR_OK;
}

static hicr_status record_prof(Instance* in, cudaEvent_t ev, cudaStream_t st) {
  if (in->capturing) HICR_CUDA(in, cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  else HICR_CUDA(in, cudaEventRecord(ev, st));
  return HICR_OK;
}

hicr_status launch_batch(Instance* in, const hicr_op_t* d_ops, uint64_t count, cudaStream_t st,
                         const uint64_t* tags) {
  hicr::NvtxRange nvtx_range("launch_batch");
  if (count == 0) return HICR_OK;
  hicr_status s = ensure_scratch(in, count);
  if (s != HICR_OK) return s;
  BatchArgs a = make_args(in, d_ops, count);
  const unsigned long long nt = (count + PS_TILE - 1) / PS_TILE;
  HICR_CUDA(in, cudaMemsetAsync(in->scratch.tiles, 0, (in->scratch.n_tiles + 1) * 8, st));
  k_plan_scan<<<(unsigned)nt, PS_THREADS, 0, st>>>(a, in->scratch.tiles, in->scratch.n_tiles);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (in->prof) {
    if ((s = prof_event(in, &e0)) != HICR_OK) return s;
    if ((s = prof_event(in, &e1)) != HICR_OK) return s;
    if ((s = record_prof(in, e0, st)) != HICR_OK) return s;
  }
  const unsigned grid = (unsigned)in->sm_count * in->cfg.blocks_per_sm;
  if (in->cfg.engine == 1) {
    if ((s = launch_copy_tma(in, a, in->cfg, grid, st)) != HICR_OK) return s;
  } else {
    k_copy<<<grid, in->cfg.threads, 0, st>>>(a);
  }
  HICR_CUDA(in, cudaGetLastError());
  note_signal(in, tags);  // the copy kernel is launched: its last warp will signal
  if (in->prof && (s = record_prof(in, e1, st)) != HICR_OK) return s;
  return HICR_OK;
}

// Host-validated batches of at most SMALL_OPS ops of at most SMALL_BYTES bytes
// each (single memcpys before a fence, small tables) skip the op-table upload
// and the plan/scan: the ops travel as kernel parameters, one CTA per op
// copies it with all its warps and then bumps the op's counters.
static constexpr uint32_t SMALL_OPS = 8;
static constexpr uint64_t SMALL_BYTES = 256u << 10;
struct SmallBatch {
  unsigned long long dst[SMALL_OPS], src[SMALL_OPS], n[SMALL_OPS];  // device-usable addresses, bytes
  uint32_t dslot[SMALL_OPS], sslot[SMALL_OPS], dtag[SMALL_OPS], stag[SMALL_OPS];
  unsigned long long* sent;
  unsigned long long* recv;
  unsigned long long* tag_ops;
  DevTables dt;                    // completion signal
  unsigned long long ticket_end;   // small-batch CTA ticket of this launch's last CTA, plus one
};

__global__ void __launch_bounds__(512) k_copy_small(SmallBatch b) {
  const unsigned i = blockIdx.x;
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long n = b.n[i];
  const unsigned long long lo = n * w / nw, hi = n * (w + 1) / nw;
  if (hi > lo)
    warp_copy(reinterpret_cast<uint8_t*>(b.dst[i]) + lo, reinterpret_cast<const uint8_t*>(b.src[i]) + lo, hi - lo,
              lane);
  // the barrier, then one cumulative fence by thread 0 before the counters
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&b.sent[b.sslot[i]], 1ull);
    atomicAdd(&b.recv[b.dslot[i]], 1ull);
    atomicAdd(&b.tag_ops[b.stag[i]], 1ull);
    if (b.dtag[i] != b.stag[i]) atomicAdd(&b.tag_ops[b.dtag[i]], 1ull);
    // CTAs draw tickets from a counter that runs across launches; the one
    // drawing this launch's last ticket finishes it
    __threadfence();
    if (atomicAdd(&b.dt.sig[1], 1ull) + 1 == b.ticket_end) emit_signal(b.dt);
  }
}

static bool small_batch(const Instance* in, const hicr_op_t* ops, uint64_t count) {
  if (count == 0 || count > SMALL_OPS || in->prof) return false;
  for (uint64_t i = 0; i < count; ++i)
    if (ops[i].n > SMALL_BYTES) return false;
  return true;
}

static hicr_status launch_small(Instance* in, const hicr_op_t* ops, uint64_t count) {
  SmallBatch b;
  memset(&b, 0, sizeof(b));
  for (uint64_t i = 0; i < count; ++i) {
    const HostSlot& d = in->slots[ops[i].dst];
    const HostSlot& sl = in->slots[ops[i].src];
    b.dst[i] = d.base + ops[i].dst_off;
    b.src[i] = sl.base + ops[i].src_off;
    b.n[i] = ops[i].n;
    b.dslot[i] = ops[i].dst;
    b.sslot[i] = ops[i].src;
    b.dtag[i] = d.tag;
    b.stag[i] = sl.tag;
  }
  b.sent = in->dt.sent;
  b.recv = in->dt.recv;
  b.tag_ops = in->dt.tag_ops;
  b.dt = in->dt;
  b.ticket_end = in->small_tickets + count;
  k_copy_small<<<(unsigned)count, 512, 0, in->comm()>>>(b);
  HICR_CUDA(in, cudaGetLastError());
  in->small_tickets += count;
  uint64_t mask[TAG_WORDS] = {};
  tag_mask(in, ops, count, mask);
  note_signal(in, mask);
  return record_signalled(in);
}

// Host tables of at least this many ops are validated and staged by the
// instance's host worker pool (HostPool, up to 8 threads with the caller);
// smaller ones on the calling thread.
static constexpr uint64_t PAR_OPS = 8192;

static HostPool& host_pool(Instance* in) {
  if (!in->pool) {
    const unsigned hw = std::thread::hardware_concurrency();
    in->pool.reset(new HostPool((int)std::min(8u, hw ? hw : 1u)));
  }
  return *in->pool;
}

// Staging buffer k (pinned host memory) and the device op table, grown to
// hold `count` ops; buffer k may still feed an earlier upload, so its last
// upload is waited for first.
static hicr_status stage_prepare(Instance* in, uint64_t count, int k) {
  HICR_CUDA(in, cudaEventSynchronize(in->pinned_ev[k]));
  if (in->pinned_cap[k] < count) {
    if (in->pinned[k]) cudaFreeHost(in->pinned[k]);
    in->pinned[k] = nullptr;
    in->pinned_cap[k] = 0;
    uint64_t cap = std::max<uint64_t>(count, 4096);
    HICR_CUDA(in, cudaHostAlloc((void**)&in->pinned[k], cap * sizeof(hicr_op_t), cudaHostAllocDefault));
    in->pinned_cap[k] = cap;
  }
  if (in->d_ops_cap < count) {
    HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
    if (in->d_ops) cudaFree(in->d_ops);
    in->d_ops = nullptr;
    in->d_ops_cap = 0;
    uint64_t cap = std::max<uint64_t>(count, 4096);
    cudaError_t e = cudaMalloc(&in->d_ops, cap * sizeof(hicr_op_t));
    if (e == cudaErrorMemoryAllocation) {
      (void)cudaGetLastError();
      return HICR_ERR_NOMEM;
    }
    HICR_CUDA(in, e);
    in->d_ops_cap = cap;
  }
  return HICR_OK;
}

// Upload the ops staged in buffer k and launch the batch on them.
static hicr_status launch_staged(Instance* in, uint64_t count, int k, const uint64_t* tags) {
  in->pinned_idx = k ^ 1;
  cudaStream_t st = in->comm();
  HICR_CUDA(in, cudaMemcpyAsync(in->d_ops, in->pinned[k], count * sizeof(hicr_op_t), cudaMemcpyHostToDevice, st));
  HICR_CUDA(in, cudaEventRecord(in->pinned_ev[k], st));
  hicr_status s = launch_batch(in, in->d_ops, count, st, tags);
  if (s != HICR_OK) return s;
  return record_signalled(in);
}

// Copy a host op table to the device through a double-buffered pinned
// staging area and launch it.
static hicr_status upload_and_launch(Instance* in, const hicr_op_t* ops, uint64_t count) {
  if (small_batch(in, ops, count)) return in->lat_idle_ns ? lat_submit(in, ops, count) : launch_small(in, ops, count);
  const int k = in->pinned_idx;
  hicr_status s = stage_prepare(in, count, k);
  if (s != HICR_OK) return s;
  hicr_op_t* dst = in->pinned[k];
  uint64_t mask[TAG_WORDS] = {};
  if (count >= PAR_OPS) {
    HostPool& pool = host_pool(in);
    std::vector<uint64_t> masks((size_t)pool.size() * TAG_WORDS, 0);
    pool.run([&](int t, int nt) {
      const uint64_t a = count * t / nt, b = count * (t + 1) / nt;
      memcpy(dst + a, ops + a, (b - a) * sizeof(hicr_op_t));
      tag_mask(in, ops + a, b - a, masks.data() + (size_t)t * TAG_WORDS);
    });
    for (size_t t = 0; t < (size_t)pool.size(); ++t)
      for (int w = 0; w < TAG_WORDS; ++w) mask[w] |= masks[t * TAG_WORDS + w];
  } else {
    memcpy(dst, ops, count * sizeof(hicr_op_t));
    tag_mask(in, ops, count, mask);
  }
  return launch_staged(in, count, k, mask);
}

// Index of the first invalid op of ops[a, b) (b when all are valid); with
// `stage` the range is also copied there, and with `mask` the tags of its
// ops are added to it.
static uint64_t validate_range(const Instance* in, const hicr_op_t* ops, uint64_t a, uint64_t b, hicr_op_t* stage,
                               uint64_t* mask = nullptr) {
  for (uint64_t i = a; i < b; ++i)
    if (validate_op(in, ops[i]) != HICR_OK) return i;
  if (stage) memcpy(stage + a, ops + a, (b - a) * sizeof(hicr_op_t));
  if (mask) tag_mask(in, ops + a, b - a, mask);
  return b;
}

// Validate every op (and, with `stage`, copy the table there and collect the
// ops' tags in `mask`) on the pool; returns the index of the first invalid op
// in issue order, or count.
static uint64_t validate_par(Instance* in, const hicr_op_t* ops, uint64_t count, hicr_op_t* stage,
                             uint64_t* mask = nullptr) {
  HostPool& pool = host_pool(in);
  std::vector<uint64_t> first((size_t)pool.size(), count);
  std::vector<uint64_t> masks(mask ? (size_t)pool.size() * TAG_WORDS : 0, 0);
  pool.run([&](int t, int nt) {
    const uint64_t a = count * t / nt, b = count * (t + 1) / nt;
    const uint64_t f = validate_range(in, ops, a, b, stage, mask ? masks.data() + (size_t)t * TAG_WORDS : nullptr);
    first[t] = f < b ? f : count;
  });
  uint64_t f = count;
  for (uint64_t x : first) f = std::min(f, x);
  if (mask)
    for (size_t t = 0; t < (size_t)pool.size(); ++t)
      for (int w = 0; w < TAG_WORDS; ++w) mask[w] |= masks[t * TAG_WORDS + w];
  return f;
}

static hicr_status validate_all(Instance* in, const hicr_op_t* ops, uint64_t count, uint64_t* first_bad) {
  // every op is checked; the reported one is the first invalid in issue order
  const uint64_t first = count >= PAR_OPS ? validate_par(in, ops, count, nullptr)
                                          : validate_range(in, ops, 0, count, nullptr);
  if (first < count) {
    if (first_bad) *first_bad = first;
    return validate_op(in, ops[first]);
  }
  if (in->checked) {
    uint64_t bad = 0;
    hicr_status s = first_hazard(in, ops, count, &bad);
    if (s != HICR_OK) {
      if (first_bad) *first_bad = bad;
      return s;
    }
  }
  return HICR_OK;
}

}  // namespace hicr

using namespace hicr;

static Instance* I(hicr_instance_t h) { return h ? &h->impl : nullptr; }

static const uint64_t QUEUE_MAX = 1u << 16;

extern "C" {

hicr_status hicr_memcpy(hicr_instance_t h, hicr_slot_t dst, uint64_t dst_off, hicr_slot_t src, uint64_t src_off,
                        uint64_t n) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  hicr_op_t op;
  op.dst = dst;
  op.src = src;
  op.dst_off = dst_off;
  op.src_off = src_off;
  op.n = n;
  hicr_status s = validate_op(in, op);
  if (s != HICR_OK) return s;
  if (in->checked) {
    in->queue.push_back(op);
    uint64_t bad = 0;
    s = first_hazard(in, in->queue.data(), in->queue.size(), &bad);
    if (s != HICR_OK) {
      in->queue.pop_back();
      return s;
    }
  } else {
    in->queue.push_back(op);
  }
  if (in->queue.size() >= QUEUE_MAX) return hicr_flush(h);
  return HICR_OK;
}

hicr_status hicr_flush(hicr_instance_t h) {
  hicr::NvtxRange nvtx_range("hicr_flush");
  Instance* in = I(h);
  if (!in) return HICR_ERR_INVALID;
  if (in->queue.empty()) return HICR_OK;
  if (in->capturing) return HICR_ERR_INVALID;
  hicr_status s = upload_and_launch(in, in->queue.data(), in->queue.size());
  in->queue.clear();
  return s;
}

hicr_status hicr_memcpy_batch(hicr_instance_t h, const hicr_op_t* ops, uint64_t count, uint64_t* first_bad) {
  Instance* in = I(h);
  if (!in || (count && !ops) || in->capturing) return HICR_ERR_INVALID;
  if (count >= PAR_OPS && !in->checked && in->queue.empty()) {
    // one pass of the host workers validates the table and stages it for
    // upload; nothing is launched unless every op is valid
    const int k = in->pinned_idx;
    hicr_status s = stage_prepare(in, count, k);
    if (s != HICR_OK) return s;
    uint64_t mask[TAG_WORDS] = {};
    const uint64_t first = validate_par(in, ops, count, in->pinned[k], mask);
    if (first < count) {
      if (first_bad) *first_bad = first;
      return validate_op(in, ops[first]);
    }
    return launch_staged(in, count, k, mask);
  }
  hicr_status s = validate_all(in, ops, count, first_bad);
  if (s != HICR_OK) return s;
  if (count == 0) return HICR_OK;
  // queued single ops belong to the same epoch and go first
  if ((s = hicr_flush(h)) != HICR_OK) return s;
  return upload_and_launch(in, ops, count);
}

hicr_status hicr_memcpy_batch_device(hicr_instance_t h, const hicr_op_t* d_ops, uint64_t count) {
  Instance* in = I(h);
  if (!in || (count && !d_ops) || ((uintptr_t)d_ops & 7u)) return HICR_ERR_INVALID;
  if (count == 0) return HICR_OK;
  if (in->capturing && count > in->scratch.cap) return HICR_ERR_INVALID;
  hicr_status s = hicr_flush(h);
  if (s != HICR_OK) return s;
  s = launch_batch(in, d_ops, count, in->comm(), nullptr);  // the host does not read the table: tags unknown
  if (s != HICR_OK) return s;
  return record_signalled(in);
}

hicr_status hicr_batch_reserve(hicr_instance_t h, uint64_t max_ops) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  return ensure_scratch(in, max_ops);
}

hicr_status hicr_memcpy_batch_plain(hicr_instance_t h, const hicr_op_t* ops, uint64_t count, uint64_t* first_bad) {
  Instance* in = I(h);
  if (!in || (count && !ops) || in->capturing) return HICR_ERR_INVALID;
  hicr_status s = validate_all(in, ops, count, first_bad);
  if (s != HICR_OK) return s;
  if ((s = hicr_flush(h)) != HICR_OK) return s;
  cudaStream_t st = in->comm();
  for (uint64_t i = 0; i < count; ++i) {
    const hicr_op_t& o = ops[i];
    if (o.n == 0) continue;
    void* d = (void*)(in->slots[o.dst].base + o.dst_off);
    const void* sp = (const void*)(in->slots[o.src].base + o.src_off);
    HICR_CUDA(in, cudaMemcpyAsync(d, sp, o.n, cudaMemcpyDefault, st));
  }
  return record_done(in);
}

hicr_status hicr_batch_get_config(hicr_instance_t h, hicr_batch_config_t* out) {
  Instance* in = I(h);
  if (!in || !out) return HICR_ERR_INVALID;
  *out = in->cfg;
  return HICR_OK;
}

hicr_status hicr_batch_set_config(hicr_instance_t h, const hicr_batch_config_t* cfg) {
  Instance* in = I(h);
  if (!in || !cfg || in->capturing) return HICR_ERR_INVALID;
  hicr_status s = check_config(in, cfg);
  if (s != HICR_OK) return s;
  in->cfg = *cfg;
  return HICR_OK;
}

hicr_status hicr_graph_begin(hicr_instance_t h) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  hicr_status s = hicr_flush(h);
  if (s != HICR_OK) return s;
  HICR_CUDA(in, cudaStreamBeginCapture(in->comm(), cudaStreamCaptureModeThreadLocal));
  in->capturing = true;
  in->cap_sigs = 0;
  return HICR_OK;
}

hicr_status hicr_graph_end(hicr_instance_t h, hicr_graph_t* out) {
  Instance* in = I(h);
  if (!in || !in->capturing || !out) return HICR_ERR_INVALID;
  in->capturing = false;
  GraphRec g;
  HICR_CUDA(in, cudaStreamEndCapture(in->comm(), &g.graph));
  cudaError_t e = cudaGraphInstantiate(&g.exec, g.graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g.graph);
    return cuda_fail(in, e, "cudaGraphInstantiate");
  }
  g.live = true;
  g.sigs = in->cap_sigs;
  for (size_t i = 0; i < in->graphs.size(); ++i) {
    if (!in->graphs[i].live) {
      in->graphs[i] = g;
      *out = (hicr_graph_t)(i + 1);
      return HICR_OK;
    }
  }
  in->graphs.push_back(g);
  *out = (hicr_graph_t)in->graphs.size();
  return HICR_OK;
}

hicr_status hicr_graph_launch(hicr_instance_t h, hicr_graph_t g) {
  hicr::NvtxRange nvtx_range("hicr_graph_launch");
  Instance* in = I(h);
  if (!in || in->capturing || g == 0 || g > in->graphs.size() || !in->graphs[g - 1].live) return HICR_ERR_INVALID;
  hicr_status s = hicr_flush(h);
  if (s != HICR_OK) return s;
  HICR_CUDA(in, cudaGraphLaunch(in->graphs[g - 1].exec, in->comm()));
  for (uint64_t k = 0; k < in->graphs[g - 1].sigs; ++k) note_signal(in, nullptr);
  return record_signalled(in);
}

hicr_status hicr_graph_destroy(hicr_instance_t h, hicr_graph_t g) {
  Instance* in = I(h);
  if (!in || g == 0 || g > in->graphs.size() || !in->graphs[g - 1].live) return HICR_ERR_INVALID;
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  cudaGraphExecDestroy(in->graphs[g - 1].exec);
  cudaGraphDestroy(in->graphs[g - 1].graph);
  in->graphs[g - 1] = GraphRec();
  return HICR_OK;
}

hicr_status hicr_profile_enable(hicr_instance_t h, int32_t on) {
  Instance* in = I(h);
  if (!in) return HICR_ERR_INVALID;
  in->prof = on != 0;
  return HICR_OK;
}

hicr_status hicr_profile_reset(hicr_instance_t h) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  in->prof_used = 0;
  return HICR_OK;
}

hicr_status hicr_profile_read(hicr_instance_t h, float* copy_ms, uint32_t* launches) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  float tot = 0.f;
  for (size_t k = 0; k + 1 < in->prof_used; k += 2) {
    float ms = 0.f;
    HICR_CUDA(in, cudaEventElapsedTime(&ms, in->prof_ev[k], in->prof_ev[k + 1]));
    tot += ms;
  }
  if (copy_ms) *copy_ms = tot;
  if (launches) *launches = (uint32_t)(in->prof_used / 2);
  return HICR_OK;
}

namespace {
// One line of the tuning cache: a JSON object with a fixed field order
// (TUNE_FMT reads it, TUNE_WFMT writes it: the same text, %s for the name).
const char* TUNE_WFMT =
    "{\"device\":\"%s\",\"sms\":%d,\"ops_log2\":%d,\"bytes_log2\":%d,\"chunk_bytes\":%u,"
    "\"op_cost_bytes\":%u,\"blocks_per_sm\":%u,\"threads\":%u,\"engine\":%u,\"tma_min_bytes\":%u,\"ms\":%f}";
const char* TUNE_FMT =
    "{\"device\":\"%127[^\"]\",\"sms\":%d,\"ops_log2\":%d,\"bytes_log2\":%d,\"chunk_bytes\":%u,"
    "\"op_cost_bytes\":%u,\"blocks_per_sm\":%u,\"threads\":%u,\"engine\":%u,\"tma_min_bytes\":%u,\"ms\":%f}";

int ilog2(unsigned long long x) {
  int k = -1;
  while (x) {
    x >>= 1;
    ++k;
  }
  return k;
}

bool tune_lookup(const char* path, const char* dev, int sms, int ol, int bl, hicr_batch_config_t* c, float* ms) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool hit = false;
  while (fgets(line, sizeof line, f)) {
    char d[128];
    int s2, o2, b2;
    hicr_batch_config_t x = *c;
    float t = 0;
    if (sscanf(line, TUNE_FMT, d, &s2, &o2, &b2, &x.chunk_bytes, &x.op_cost_bytes, &x.blocks_per_sm, &x.threads,
               &x.engine, &x.tma_min_bytes, &t) == 11 &&
        strcmp(d, dev) == 0 && s2 == sms && o2 == ol && b2 == bl) {
      *c = x;  // the last matching line wins
      *ms = t;
      hit = true;
    }
  }
  fclose(f);
  return hit;
}

void tune_store(const char* path, const char* dev, int sms, int ol, int bl, const hicr_batch_config_t& c, float ms) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, TUNE_WFMT, dev, sms, ol, bl, c.chunk_bytes, c.op_cost_bytes, c.blocks_per_sm, c.threads, c.engine,
          c.tma_min_bytes, (double)ms);
  fputc('\n', f);
  fclose(f);
}
}  // namespace

hicr_status hicr_batch_autotune(hicr_instance_t h, const hicr_op_t* d_ops, uint64_t count, uint32_t reps,
                                hicr_batch_config_t* best, float* best_ms) {
  Instance* in = I(h);
  if (!in || !d_ops || count == 0 || reps == 0 || in->capturing) return HICR_ERR_INVALID;
  hicr_status s = hicr_flush(h);
  if (s != HICR_OK) return s;
  if ((s = ensure_scratch(in, count)) != HICR_OK) return s;
  const hicr_batch_config_t base = in->cfg;
  // tuning cache: the key needs the table's payload bytes, which one run with
  // the current configuration leaves in the batch control block
  const char* cache = getenv("HICR_TUNE_CACHE");
  int key_ops = 0, key_bytes = 0;
  if (cache && *cache) {
    if ((s = launch_batch(in, d_ops, count, in->comm(), nullptr)) != HICR_OK) return s;
    BatchCtrl ctl;
    HICR_CUDA(in, cudaMemcpyAsync(&ctl, in->scratch.ctrl, sizeof(ctl), cudaMemcpyDeviceToHost, in->comm()));
    HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
    const unsigned long long charged = (unsigned long long)in->cfg.op_cost_bytes * count;
    key_ops = ilog2(count);
    key_bytes = ilog2(ctl.total > charged ? ctl.total - charged : 0ull);
    hicr_batch_config_t c = base;
    float ms = 0;
    if (tune_lookup(cache, in->prop.name, in->sm_count, key_ops, key_bytes, &c, &ms) && check_config(in, &c) == HICR_OK) {
      in->cfg = c;
      hicr_status bst = HICR_OK;
      uint64_t bad = 0;
      hicr_batch_error(h, &bst, &bad);
      if (bst != HICR_OK) return bst;
      if (best) *best = c;
      if (best_ms) *best_ms = ms;
      return record_signalled(in);
    }
  }
  std::vector<hicr_batch_config_t> cands;
  const uint32_t chunks[] = {32u << 10, 64u << 10, 128u << 10, 256u << 10};
  const uint32_t shapes[][2] = {{1, 1024}, {2, 512}, {4, 256}, {2, 1024}, {4, 512}};
  const uint32_t costs[] = {1024, 4096};
  for (uint32_t ch : chunks)
    for (auto& sh : shapes)
      for (uint32_t oc : costs) {
        hicr_batch_config_t c = base;
        c.chunk_bytes = ch;
        c.blocks_per_sm = sh[0];
        c.threads = sh[1];
        c.op_cost_bytes = oc;
        c.engine = 0;
        cands.push_back(c);
      }
  // the TMA engine: CTA shapes x stage shapes (stages x stage bytes per
  // warp); candidates whose shared memory does not fit are skipped below
  const uint32_t tma_shapes[][2] = {{1, 192}, {1, 256}, {1, 384}, {2, 192}, {1, 512}, {2, 256}, {1, 768}};
  const uint32_t stage_shapes[][2] = {{2, 4096}, {4, 4096}, {2, 8192}, {4, 8192}, {8, 4096}, {2, 16384}};
  for (uint32_t ch : {128u << 10, 256u << 10})
    for (auto& sh : tma_shapes)
      for (auto& ss : stage_shapes) {
        hicr_batch_config_t c = base;
        c.chunk_bytes = ch;
        c.blocks_per_sm = sh[0];
        c.threads = sh[1];
        c.op_cost_bytes = 4096;
        c.engine = 1;
        c.tma_min_bytes = 32u << 10;
        c.tma_stages = ss[0];
        c.tma_stage_bytes = ss[1];
        cands.push_back(c);
      }
  cudaEvent_t e0, e1;
  HICR_CUDA(in, cudaEventCreate(&e0));
  HICR_CUDA(in, cudaEventCreate(&e1));
  cudaStream_t st = in->comm();
  float best_t = 1e30f;
  hicr_batch_config_t best_c = base;
  for (auto& c : cands) {
    // skip shapes the device cannot hold
    int per_sm = 0;
    if (c.engine == 1) {
      if (copy_tma_prepare(in, c, &per_sm) != HICR_OK) per_sm = 0;
    } else {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_copy, c.threads, 0);
    }
    if (per_sm < (int)c.blocks_per_sm) continue;
    in->cfg = c;
    std::vector<float> ts;
    for (uint32_t r = 0; r <= reps; ++r) {
      cudaEventRecord(e0, st);
      s = launch_batch(in, d_ops, count, st, nullptr);
      if (s != HICR_OK) break;
      cudaEventRecord(e1, st);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        s = cuda_fail(in, e, "autotune");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r) ts.push_back(ms);
    }
    if (s != HICR_OK) break;
    std::sort(ts.begin(), ts.end());
    const float med = ts[ts.size() / 2];
    if (med < best_t) {
      best_t = med;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  in->cfg = best_c;
  if (s != HICR_OK) return s;
  hicr_status bst = HICR_OK;
  uint64_t bad = 0;
  hicr_batch_error(h, &bst, &bad);
  if (bst != HICR_OK) return bst;
  if (cache && *cache) tune_store(cache, in->prop.name, in->sm_count, key_ops, key_bytes, best_c, best_t);
  if (best) *best = best_c;
  if (best_ms) *best_ms = best_t;
  return record_signalled(in);
}

}  // extern "C"
