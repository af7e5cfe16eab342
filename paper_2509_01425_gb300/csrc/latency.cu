// Latency mode (hicr_set_latency_mode): small host-validated batches (the
// ones k_copy_small would take) and the channel host calls (push, peek, pop,
// depth) go to a short-lived persistent server kernel instead of a kernel
// launch each.
//
// The host writes the ops' descriptors into a ring in mapped page-locked
// memory and publishes them by advancing `head` (release). One CTA of the
// server, on a stream of its own, polls `head` (acquire, system scope), copies
// each op with all its warps, bumps the op's slot and tag counters, and
// publishes `done` (release, system scope) in mapped memory, which the fences
// poll. A server that has seen no work for the idle window announces its exit
// (`exit_epoch`), takes whatever was published meanwhile, and ends; the next
// batch launches a new one on the same stream, which therefore starts only
// after the old one has ended, so every op is taken exactly once. Every wait
// is bounded: the idle window, and a stop flag the host raises before
// finalize.
//
// Ordering against the communication stream: the server runs beside it, and
// that is what the model allows -- ops between two fences are unordered, and
// a fence waits for the ops of its tag on both (the server's `done` and the
// stream's completion signals). A channel call is synchronous and, like its
// launched form, must come after everything issued before it: it goes to the
// server only while the communication stream has nothing pending (the server
// takes its ring in order, so copies published before it are done first).
#include <string.h>

#include <atomic>
#include <thread>

#include "channel_calls.cuh"
#include "copy.cuh"
#include "hicr_internal.h"

namespace hicr {

static_assert(sizeof(ChanCall) <= sizeof(((LatOp*)nullptr)->call), "a channel call fits its ring entry");

static constexpr unsigned LAT_THREADS = 512;
static constexpr unsigned LAT_OP_WORDS = sizeof(LatOp) / 8;
static_assert(sizeof(LatOp) % 8 == 0 && LAT_OP_WORDS <= LAT_THREADS, "a ring entry is read one word per thread");

__device__ __forceinline__ unsigned long long lat_ld_acq_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long lat_ld_rlx_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lat_st_rel_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long lat_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct LatArgs {
  LatRing* ring;  // device address of the mapped ring
  DevTables dt;
  unsigned long long epoch;
  unsigned long long idle_ns;
};

// Copy op (d, s, n) with every warp of the CTA: warp w takes its share.
__device__ __forceinline__ void lat_copy(const LatOp& op) {
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long lo = op.n * w / nw, hi = op.n * (w + 1) / nw;
  if (hi > lo)
    warp_copy(reinterpret_cast<uint8_t*>(op.dst) + lo, reinterpret_cast<const uint8_t*>(op.src) + lo, hi - lo, lane);
}

__global__ void __launch_bounds__(LAT_THREADS) k_lat_server(LatArgs a) {
  __shared__ unsigned long long s_head, s_tail;
  __shared__ int s_exit;
  __shared__ LatOp s_op;
  LatRing* r = a.ring;
  unsigned long long tail = 0;  // thread 0: ops taken (starts at the previous server's `done`)
  if (threadIdx.x == 0) tail = lat_ld_acq_sys(&r->done);
  bool announced = false;  // thread 0's decision, shared through s_exit
  for (;;) {
    if (threadIdx.x == 0) {
      unsigned long long h = lat_ld_acq_sys(&r->head);
      int ex = 0;
      if (h == tail && !announced) {
        const unsigned long long t0 = lat_now();
        // each poll is a round trip to host memory (about a microsecond), so
        // the pause between polls stays short: it only adds to the latency
        while (h == tail) {
          if (lat_ld_acq_sys(&r->stop) || lat_now() - t0 > a.idle_ns) break;
          __nanosleep(32);
          h = lat_ld_acq_sys(&r->head);
        }
        if (h == tail) {
          // nothing came: announce the exit, then take what was published
          // before the announcement became visible (the host launches a new
          // server for anything published after it saw it). Store, full
          // fence, load, as the host does in the other order: one of the
          // two sees the other's store.
          lat_st_rel_sys(&r->exit_epoch, a.epoch);
          __threadfence_system();
          announced = true;
          h = lat_ld_acq_sys(&r->head);
        }
      }
      // after the announcement this server takes one last batch and ends
      ex = (h == tail) ? 1 : (announced ? 2 : 0);
      s_head = h;
      s_tail = tail;
      s_exit = ex;
    }
    __syncthreads();
    const int ex = s_exit;
    if (ex == 1) break;
    const unsigned long long h = s_head;
    for (unsigned long long t = s_tail; t < h; ++t) {
      // the entry, one word per thread: a single round trip to host memory
      // (ordered after thread 0's acquire of `head` by the barrier above)
      if (threadIdx.x < LAT_OP_WORDS)
        reinterpret_cast<unsigned long long*>(&s_op)[threadIdx.x] =
            lat_ld_rlx_sys(reinterpret_cast<const unsigned long long*>(&r->ops[t % LAT_RING_OPS]) + threadIdx.x);
      __syncthreads();
      if (s_op.kind == LAT_CHANNEL) {
        ChanCall c;
        memcpy(&c, s_op.call, sizeof c);
        chan_call(c);  // posts its own status to the caller's mailbox
        __syncthreads();
        continue;
      }
      const LatOp& op = s_op;  // thread 0 rewrites it only after the barrier below
      lat_copy(op);
      // the barrier, then one cumulative fence before the counters
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&a.dt.sent[op.sslot], 1ull);
        atomicAdd(&a.dt.recv[op.dslot], 1ull);
        atomicAdd(&a.dt.tag_ops[op.stag], 1ull);
        if (op.dtag != op.stag) atomicAdd(&a.dt.tag_ops[op.dtag], 1ull);
      }
    }
    if (threadIdx.x == 0) {
      tail = h;
      __threadfence_system();
      lat_st_rel_sys(&r->done, h);
    }
    __syncthreads();
    if (ex == 2) break;
  }
}

hicr_status lat_setup(Instance* in) {
  if (in->lat_ring) return HICR_OK;
  LatRing* hr = nullptr;
  HICR_CUDA(in, cudaHostAlloc((void**)&hr, sizeof(LatRing), cudaHostAllocMapped));
  memset(hr, 0, sizeof(LatRing));
  LatRing* dr = nullptr;
  cudaError_t e = cudaHostGetDevicePointer((void**)&dr, hr, 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&in->lat_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFreeHost(hr);
    return cuda_fail(in, e, "latency-mode set-up");
  }
  in->lat_ring = hr;
  in->lat_ring_dev = dr;
  in->lat_head = 0;
  in->lat_epoch = 0;
  return HICR_OK;
}

// Ask a running server to end and wait for it (bounded).
hicr_status lat_stop(Instance* in) {
  if (!in->lat_ring) return HICR_OK;
  __atomic_store_n(&in->lat_ring->stop, 1ull, __ATOMIC_RELEASE);
  const uint64_t until = now_ns() + 10ull * 1000000000ull;
  cudaError_t e;
  while ((e = cudaStreamQuery(in->lat_stream)) == cudaErrorNotReady && now_ns() < until) std::this_thread::yield();
  __atomic_store_n(&in->lat_ring->stop, 0ull, __ATOMIC_RELEASE);
  if (e == cudaErrorNotReady) return HICR_ERR_TIMEOUT;
  if (e != cudaSuccess) return cuda_fail(in, e, "latency-mode server");
  return HICR_OK;
}

void lat_destroy(Instance* in) {
  if (!in->lat_ring) return;
  lat_stop(in);
  cudaStreamSynchronize(in->lat_stream);
  cudaStreamDestroy(in->lat_stream);
  cudaFreeHost(in->lat_ring);
  in->lat_ring = nullptr;
  in->lat_ring_dev = nullptr;
}

// Wait (bounded: a live server drains the ring) until `count` more entries fit.
static hicr_status lat_room(Instance* in, uint64_t count) {
  volatile unsigned long long* done = &in->lat_ring->done;
  const uint64_t t0 = now_ns();
  while (in->lat_head + count - *done > LAT_RING_OPS) {
    if (now_ns() - t0 > 10ull * 1000000000ull) return HICR_ERR_TIMEOUT;
    std::this_thread::yield();
  }
  return HICR_OK;
}

// Publish the entries written up to lat_head, then launch a server if the
// last one launched has announced its exit. Publish, full fence, then read
// the announcement (the server stores its announcement, fences, then reads
// head): one of the two sees the other's store.
static hicr_status lat_publish(Instance* in) {
  LatRing* r = in->lat_ring;
  __atomic_store_n(&r->head, (unsigned long long)in->lat_head, __ATOMIC_SEQ_CST);
  __atomic_thread_fence(__ATOMIC_SEQ_CST);
  if (__atomic_load_n(&r->exit_epoch, __ATOMIC_SEQ_CST) == in->lat_epoch) {
    LatArgs a;
    a.ring = in->lat_ring_dev;
    a.dt = in->dt;
    a.epoch = ++in->lat_epoch;
    a.idle_ns = in->lat_idle_ns;
    k_lat_server<<<1, LAT_THREADS, 0, in->lat_stream>>>(a);
    HICR_CUDA(in, cudaGetLastError());
  }
  return HICR_OK;
}

// Publish validated ops (at most LAT_RING_OPS in flight) to the server,
// launching one when the last has announced its exit.
hicr_status lat_submit(Instance* in, const hicr_op_t* ops, uint64_t count) {
  LatRing* r = in->lat_ring;
  hicr_status st = lat_room(in, count);
  if (st != HICR_OK) return st;
  uint64_t mask[TAG_WORDS] = {};
  for (uint64_t i = 0; i < count; ++i) {
    const HostSlot& d = in->slots[ops[i].dst];
    const HostSlot& s = in->slots[ops[i].src];
    LatOp& o = r->ops[(in->lat_head + i) % LAT_RING_OPS];
    o.dst = d.base + ops[i].dst_off;
    o.src = s.base + ops[i].src_off;
    o.n = ops[i].n;
    o.dslot = ops[i].dst;
    o.sslot = ops[i].src;
    o.dtag = d.tag;
    o.stag = s.tag;
    o.kind = LAT_COPY;
    mask[d.tag >> 6] |= 1ull << (d.tag & 63);
    mask[s.tag >> 6] |= 1ull << (s.tag & 63);
  }
  in->lat_head += count;
  for (int w = 0; w < TAG_WORDS; ++w)
    for (uint64_t m = mask[w]; m; m &= m - 1) in->tag_lat[w * 64 + __builtin_ctzll(m)] = in->lat_head;
  return lat_publish(in);
}

bool lat_takes_calls(Instance* in) {
  if (!in->lat_idle_ns || !in->lat_ring || in->capturing) return false;
  if (in->opaque) {
    // other work was issued on the communication stream: quiet once the done
    // event (recorded after every launch there) has completed
    const cudaError_t e = cudaEventQuery(in->done_ev);
    if (e != cudaSuccess) {
      if (e != cudaErrorNotReady) (void)cudaGetLastError();
      return false;
    }
    in->opaque = false;
  }
  return *(volatile unsigned long long*)in->sig_mirror >= in->sig_issued;
}

hicr_status lat_channel_call(Instance* in, const ChanCall& c, volatile int* status) {
  hicr_status st = lat_room(in, 1);
  if (st != HICR_OK) return st;
  LatOp& o = in->lat_ring->ops[in->lat_head % LAT_RING_OPS];
  o.kind = LAT_CHANNEL;
  memcpy(o.call, &c, sizeof c);
  in->lat_head += 1;
  if ((st = lat_publish(in)) != HICR_OK) return st;
  // The server posts the status last, behind a system-scope fence. Bounded
  // wait; a server that ended without posting it (a failed kernel) ends it.
  const uint64_t t0 = now_ns();
  for (uint32_t spins = 0;; ++spins) {
    const int v = *status;
    if (v != 1) {
      __atomic_thread_fence(__ATOMIC_ACQUIRE);
      return (hicr_status)v;
    }
    if ((spins & 255) == 255) {
      const cudaError_t e = cudaStreamQuery(in->lat_stream);
      if (e != cudaErrorNotReady) {
        if (*status != 1) continue;
        if (e != cudaSuccess) return cuda_fail(in, e, "latency-mode server");
        return HICR_ERR_DEVICE;
      }
      const uint64_t dt = now_ns() - t0;
      if (dt > 60ull * 1000000000ull) return HICR_ERR_TIMEOUT;
      if (dt > WAIT_YIELD_NS) std::this_thread::sleep_for(std::chrono::microseconds(20));
      else if (dt > WAIT_SPIN_NS) std::this_thread::yield();
    }
  }
}

// Wait until the server has completed op count `target` (mapped memory).
hicr_status lat_wait(Instance* in, uint64_t target, uint64_t timeout_ns) {
  if (!in->lat_ring || target == 0) return HICR_OK;
  volatile unsigned long long* done = &in->lat_ring->done;
  if (*done >= target) {
    __atomic_thread_fence(__ATOMIC_ACQUIRE);
    return HICR_OK;
  }
  const uint64_t t0 = now_ns();
  for (uint32_t spins = 0;; ++spins) {
    if (*done >= target) {
      __atomic_thread_fence(__ATOMIC_ACQUIRE);
      return HICR_OK;
    }
    if ((spins & 63) == 0) {
      const uint64_t dt = now_ns() - t0;
      if (dt >= timeout_ns) return HICR_ERR_TIMEOUT;
      if (dt > WAIT_YIELD_NS) std::this_thread::sleep_for(std::chrono::microseconds(20));
      else if (dt > WAIT_SPIN_NS) std::this_thread::yield();
    }
  }
}

hicr_status lat_drain(Instance* in) {
  if (!in->lat_ring) return HICR_OK;
  return lat_wait(in, in->lat_head, 60ull * 1000000000ull);
}

}  // namespace hicr

using namespace hicr;

extern "C" hicr_status hicr_set_latency_mode(hicr_instance_t h, uint32_t idle_us) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || in->capturing || idle_us > 1000000u) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  if (idle_us == 0) {
    st = lat_wait(in, in->lat_head, 60ull * 1000000000ull);
    if (st != HICR_OK) return st;
    in->lat_idle_ns = 0;
    return lat_stop(in);
  }
  if ((st = lat_setup(in)) != HICR_OK) return st;
  in->lat_idle_ns = (uint64_t)idle_us * 1000ull;
  return HICR_OK;
}
