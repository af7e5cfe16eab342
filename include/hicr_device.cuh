/*
 * hicr_device.cuh -- device-side channel calls for CUDA kernels (header-only).
 *
 * HiCR paper Sec. 4.3 (Channels): producers push while the consumer's ring is
 * not full and otherwise wait for the consumer to report consumption; the
 * consumer takes messages in order. The host calls of hicr_channels.h act on
 * a channel from the CPU; the functions below let a kernel be the producer or
 * the consumer of the same channel. The host fills a hicr_channel_view_t with
 * hicr_channel_device_view() (hicr_channels.h) and passes it to the kernel by
 * value.
 *
 * Every function is warp-collective: all 32 lanes of one warp call it with the
 * same arguments (the warp is the producer or consumer agent). Waits (for room,
 * for a message) are bounded by timeout_ns of %globaltimer time; a wait that
 * gives up returns HICR_ERR_TIMEOUT and leaves the channel unchanged. The
 * state is shared with the host calls: counters, placement rule and metadata
 * are those of hicr_channels.h, so a channel can be filled on the device and
 * drained from the host (or the reverse), as long as each side is the only
 * producer or consumer it claims to be (SPSC: one producer agent and one
 * consumer agent at a time; MPSC locking mode: any number of producer warps,
 * one consumer agent; non-locking mode: one producer agent per ring, one
 * consumer agent).
 *
 * Memory: src/dst buffers are device-accessible addresses; any alignment.
 */
#ifndef HICR_DEVICE_CUH
#define HICR_DEVICE_CUH

#include <stdint.h>

#include "hicr_channels.h"

#ifdef __CUDACC__

namespace hicr_dev {

static constexpr unsigned long long M40 = (1ull << 40) - 1;
static constexpr unsigned long long M24 = (1ull << 24) - 1;

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long r16(unsigned long long n) { return (n + 15) & ~15ull; }

// Warp copy of n bytes: 16-byte vectors when both ends are 16-byte aligned,
// bytes otherwise. Reads at L2 (the bytes may come from another SM).
__device__ __forceinline__ void copy(uint8_t* d, const uint8_t* s, unsigned long long n, unsigned lane) {
  if ((((uintptr_t)d | (uintptr_t)s) & 15) == 0) {
    const unsigned long long nv = n / 16;
    for (unsigned long long i = lane; i < nv; i += 32)
      reinterpret_cast<uint4*>(d)[i] = __ldcg(reinterpret_cast<const uint4*>(s) + i);
    for (unsigned long long i = nv * 16 + lane; i < n; i += 32) d[i] = __ldcg(s + i);
  } else {
    for (unsigned long long i = lane; i < n; i += 32) d[i] = __ldcg(s + i);
  }
}

}  // namespace hicr_dev

/* SPSC: push k tokens (k * token_size bytes from src). Waits for room.
 * Returns HICR_OK, HICR_ERR_FULL (k > capacity), HICR_ERR_INVALID (not SPSC)
 * or HICR_ERR_TIMEOUT. */
__device__ inline int hicr_dev_spsc_push(const hicr_channel_view_t& v, const void* src, uint32_t k,
                                         unsigned long long timeout_ns) {
  using namespace hicr_dev;
  const unsigned lane = threadIdx.x & 31u;
  if (v.kind != 0) return HICR_ERR_INVALID;
  if (k > v.capacity) return HICR_ERR_FULL;
  unsigned long long h = 0;
  int st = HICR_OK;
  if (lane == 0) {
    h = *(volatile unsigned long long*)v.head;  // this warp is the only producer
    const unsigned long long t0 = now();
    while (h + k - ld_acquire(v.tail) > v.capacity) {
      if (now() - t0 > timeout_ns) {
        st = HICR_ERR_TIMEOUT;
        break;
      }
      __nanosleep(64);
    }
  }
  st = __shfl_sync(0xffffffffu, st, 0);
  if (st != HICR_OK) return st;
  h = __shfl_sync(0xffffffffu, h, 0);
  const unsigned long long first = h % v.capacity;
  const unsigned long long run1 = k < v.capacity - first ? k : v.capacity - first;
  const uint8_t* s = static_cast<const uint8_t*>(src);
  copy(v.ring + first * v.token_size, s, run1 * v.token_size, lane);
  if (k > run1) copy(v.ring, s + run1 * v.token_size, (k - run1) * v.token_size, lane);
  __threadfence();
  __syncwarp();
  if (lane == 0) st_release(v.head, h + k);
  return HICR_OK;
}

/* SPSC: pop k tokens into dst (k * token_size bytes). Waits for them.
 * Returns HICR_OK, HICR_ERR_EMPTY (k > capacity), HICR_ERR_INVALID or
 * HICR_ERR_TIMEOUT. */
__device__ inline int hicr_dev_spsc_pop(const hicr_channel_view_t& v, void* dst, uint32_t k,
                                        unsigned long long timeout_ns) {
  using namespace hicr_dev;
  const unsigned lane = threadIdx.x & 31u;
  if (v.kind != 0) return HICR_ERR_INVALID;
  if (k > v.capacity) return HICR_ERR_EMPTY;
  unsigned long long t = 0;
  int st = HICR_OK;
  if (lane == 0) {
    t = *(volatile unsigned long long*)v.tail;  // this warp is the only consumer
    const unsigned long long t0 = now();
    while (ld_acquire(v.head) - t < k) {
      if (now() - t0 > timeout_ns) {
        st = HICR_ERR_TIMEOUT;
        break;
      }
      __nanosleep(64);
    }
  }
  st = __shfl_sync(0xffffffffu, st, 0);
  if (st != HICR_OK) return st;
  __syncwarp();
  t = __shfl_sync(0xffffffffu, t, 0);
  const unsigned long long first = t % v.capacity;
  const unsigned long long run1 = k < v.capacity - first ? k : v.capacity - first;
  uint8_t* d = static_cast<uint8_t*>(dst);
  copy(d, v.ring + first * v.token_size, run1 * v.token_size, lane);
  if (k > run1) copy(d + run1 * v.token_size, v.ring, (k - run1) * v.token_size, lane);
  __syncwarp();
  if (lane == 0) st_release(v.tail, t + k);
  return HICR_OK;
}

/* MPSC (locking mode): push one message of n bytes from src as producer
 * `producer` with sequence number `seq` (recorded in the metadata). The
 * reservation is one compare-and-swap under the placement rule of
 * hicr_mpsc_create (16-byte rounding, skip to the ring start, capacity in
 * bytes and messages); waits while there is no room. Returns HICR_OK,
 * HICR_ERR_TOO_LARGE (rounded size above the ring), HICR_ERR_INVALID or
 * HICR_ERR_TIMEOUT. */
__device__ inline int hicr_dev_mpsc_push(const hicr_channel_view_t& v, uint32_t producer, uint32_t seq,
                                         const void* src, uint32_t n, unsigned long long timeout_ns) {
  using namespace hicr_dev;
  const unsigned lane = threadIdx.x & 31u;
  if (v.kind != 1) return HICR_ERR_INVALID;
  const unsigned long long R = v.ring_bytes, r = r16(n);
  if (r > R) return HICR_ERR_TOO_LARGE;
  unsigned long long W = 0, start = 0;
  int st = HICR_OK;
  if (lane == 0) {
    const unsigned long long t0 = now();
    for (;;) {
      W = ld_acquire(v.head);
      const unsigned long long b = W & M40, pos = b & (R - 1);
      start = pos + r > R ? (b + (R - pos)) & M40 : b;
      const unsigned long long end = (start + r) & M40, tk = W >> 40;
      const bool room = ((end - ld_acquire(v.freed)) & M40) <= R && (((tk + 1) - ld_acquire(v.tail)) & M24) <= v.max_msgs;
      if (room && atomicCAS(v.head, W, (((tk + 1) & M24) << 40) | end) == W) break;
      if (now() - t0 > timeout_ns) {
        st = HICR_ERR_TIMEOUT;
        break;
      }
      if (!room) __nanosleep(64);
    }
  }
  st = __shfl_sync(0xffffffffu, st, 0);
  if (st != HICR_OK) return st;
  W = __shfl_sync(0xffffffffu, W, 0);
  start = __shfl_sync(0xffffffffu, start, 0);
  copy(v.ring + (start & (R - 1)), static_cast<const uint8_t*>(src), n, lane);
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    const unsigned long long tk = W >> 40;
    hicr_mpsc_meta_t* e = static_cast<hicr_mpsc_meta_t*>(v.meta) + (tk & (v.max_msgs - 1));
    e->start = start;
    e->size = n;
    e->producer = producer;
    e->seq = seq;
    e->flags = 0;
    st_release(&e->ready, (tk & M24) + 1);
  }
  return HICR_OK;
}

/* MPSC (locking mode): pop the oldest message into dst (at most dst_cap
 * bytes), waiting for one to be published; *info (if not NULL; written by
 * lane 0) receives its ring offset, size, producer and sequence number.
 * Returns HICR_OK, HICR_ERR_TOO_LARGE (the message exceeds dst_cap; nothing
 * is popped), HICR_ERR_INVALID or HICR_ERR_TIMEOUT. */
__device__ inline int hicr_dev_mpsc_pop(const hicr_channel_view_t& v, void* dst, uint64_t dst_cap,
                                        hicr_msg_info_t* info, unsigned long long timeout_ns) {
  using namespace hicr_dev;
  const unsigned lane = threadIdx.x & 31u;
  if (v.kind != 1) return HICR_ERR_INVALID;
  unsigned long long t = 0, start = 0;
  unsigned n = 0, prod = 0, seq = 0;
  int st = HICR_OK;
  if (lane == 0) {
    t = *(volatile unsigned long long*)v.tail;  // this warp is the only consumer
    const hicr_mpsc_meta_t* e = static_cast<const hicr_mpsc_meta_t*>(v.meta) + (t & (v.max_msgs - 1));
    const unsigned long long t0 = now();
    while (ld_acquire(&e->ready) != (t & M24) + 1) {
      if (now() - t0 > timeout_ns) {
        st = HICR_ERR_TIMEOUT;
        break;
      }
      __nanosleep(64);
    }
    if (st == HICR_OK) {
      start = __ldcg(&e->start);
      n = __ldcg(&e->size);
      prod = __ldcg(&e->producer);
      seq = __ldcg(&e->seq);
      if (n > dst_cap) st = HICR_ERR_TOO_LARGE;
    }
  }
  st = __shfl_sync(0xffffffffu, st, 0);
  if (st != HICR_OK) return st;
  __syncwarp();
  t = __shfl_sync(0xffffffffu, t, 0);
  start = __shfl_sync(0xffffffffu, start, 0);
  n = __shfl_sync(0xffffffffu, n, 0);
  copy(static_cast<uint8_t*>(dst), v.ring + (start & (v.ring_bytes - 1)), n, lane);
  __syncwarp();
  if (lane == 0) {
    if (info) {
      info->offset = start & (v.ring_bytes - 1);
      info->size = n;
      info->producer = prod;
      info->reserved = 0;
      info->seq = seq;
    }
    st_release(v.freed, (start + r16(n)) & M40);
    st_release(v.tail, t + 1);
  }
  return HICR_OK;
}

/* Non-locking MPSC: producer `producer` pushes one message of n bytes into
 * its own ring (the calling warp must be that ring's only producer). Same
 * placement rule per ring; waits while the ring has no room. Returns
 * HICR_OK, HICR_ERR_TOO_LARGE, HICR_ERR_INVALID or HICR_ERR_TIMEOUT. */
__device__ inline int hicr_dev_mpsc_nl_push(const hicr_channel_view_t& v, uint32_t producer, uint32_t seq,
                                            const void* src, uint32_t n, unsigned long long timeout_ns) {
  using namespace hicr_dev;
  const unsigned lane = threadIdx.x & 31u;
  if (v.kind != 2 || producer >= v.capacity) return HICR_ERR_INVALID;
  const unsigned long long R = v.ring_bytes, r = r16(n);
  if (r > R) return HICR_ERR_TOO_LARGE;
  unsigned long long* cnt = v.head + (unsigned long long)producer * HICR_NL_STATE_WORDS;
  unsigned long long start = 0, pub = 0;
  int st = HICR_OK;
  if (lane == 0) {
    const unsigned long long b = *(volatile unsigned long long*)(cnt + HICR_NL_RESERVE);
    pub = *(volatile unsigned long long*)(cnt + HICR_NL_PUB);
    const unsigned long long pos = b & (R - 1);
    start = pos + r > R ? b + (R - pos) : b;
    const unsigned long long t0 = now();
    while (start + r - ld_acquire(cnt + HICR_NL_FREED) > R || pub + 1 - ld_acquire(cnt + HICR_NL_CONS) > v.max_msgs) {
      if (now() - t0 > timeout_ns) {
        st = HICR_ERR_TIMEOUT;
        break;
      }
      __nanosleep(64);
    }
  }
  st = __shfl_sync(0xffffffffu, st, 0);
  if (st != HICR_OK) return st;
  start = __shfl_sync(0xffffffffu, start, 0);
  pub = __shfl_sync(0xffffffffu, pub, 0);
  copy(v.ring + (unsigned long long)producer * R + (start & (R - 1)), static_cast<const uint8_t*>(src), n, lane);
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    hicr_nl_meta_t* e = static_cast<hicr_nl_meta_t*>(v.meta) + (unsigned long long)producer * v.max_msgs +
                        (pub & (v.max_msgs - 1));
    e->start = start;
    e->size = n;
    e->seq = seq;
    *(volatile unsigned long long*)(cnt + HICR_NL_RESERVE) = start + r;
    st_release(cnt + HICR_NL_PUB, pub + 1);
  }
  return HICR_OK;
}

/* Non-locking MPSC: pop the oldest message of ring `producer` into dst (at
 * most dst_cap bytes), waiting for one; the calling warp must be that ring's
 * only consumer. *info (if not NULL; written by lane 0) receives its ring
 * offset, size, producer and sequence number. Returns HICR_OK,
 * HICR_ERR_TOO_LARGE (nothing popped), HICR_ERR_INVALID or HICR_ERR_TIMEOUT. */
__device__ inline int hicr_dev_mpsc_nl_pop(const hicr_channel_view_t& v, uint32_t producer, void* dst,
                                           uint64_t dst_cap, hicr_msg_info_t* info, unsigned long long timeout_ns) {
  using namespace hicr_dev;
  const unsigned lane = threadIdx.x & 31u;
  if (v.kind != 2 || producer >= v.capacity) return HICR_ERR_INVALID;
  unsigned long long* cnt = v.head + (unsigned long long)producer * HICR_NL_STATE_WORDS;
  unsigned long long c = 0, start = 0;
  unsigned n = 0, seq = 0;
  int st = HICR_OK;
  if (lane == 0) {
    c = *(volatile unsigned long long*)(cnt + HICR_NL_CONS);
    const unsigned long long t0 = now();
    while (ld_acquire(cnt + HICR_NL_PUB) == c) {
      if (now() - t0 > timeout_ns) {
        st = HICR_ERR_TIMEOUT;
        break;
      }
      __nanosleep(64);
    }
    if (st == HICR_OK) {
      const hicr_nl_meta_t* e = static_cast<const hicr_nl_meta_t*>(v.meta) +
                                (unsigned long long)producer * v.max_msgs + (c & (v.max_msgs - 1));
      start = __ldcg(&e->start);
      n = __ldcg(&e->size);
      seq = __ldcg(&e->seq);
      if (n > dst_cap) st = HICR_ERR_TOO_LARGE;
    }
  }
  st = __shfl_sync(0xffffffffu, st, 0);
  if (st != HICR_OK) return st;
  __syncwarp();
  c = __shfl_sync(0xffffffffu, c, 0);
  start = __shfl_sync(0xffffffffu, start, 0);
  n = __shfl_sync(0xffffffffu, n, 0);
  copy(static_cast<uint8_t*>(dst), v.ring + (unsigned long long)producer * v.ring_bytes + (start & (v.ring_bytes - 1)),
       n, lane);
  __syncwarp();
  if (lane == 0) {
    if (info) {
      info->offset = start & (v.ring_bytes - 1);
      info->size = n;
      info->producer = producer;
      info->reserved = 0;
      info->seq = seq;
    }
    st_release(cnt + HICR_NL_FREED, start + r16(n));
    st_release(cnt + HICR_NL_CONS, c + 1);
  }
  return HICR_OK;
}

/* Non-locking MPSC: pop one message from whichever ring has one, scanning
 * the rings round-robin from *next (32 rings per step, one per lane) until
 * one is non-empty; *next (every lane's copy) becomes the ring after the one
 * popped. The calling warp must be the only consumer of every ring. Returns
 * as hicr_dev_mpsc_nl_pop; HICR_ERR_TIMEOUT when every ring stayed empty. */
__device__ inline int hicr_dev_mpsc_nl_pop_any(const hicr_channel_view_t& v, uint32_t* next, void* dst,
                                               uint64_t dst_cap, hicr_msg_info_t* info,
                                               unsigned long long timeout_ns) {
  using namespace hicr_dev;
  const unsigned lane = threadIdx.x & 31u;
  if (v.kind != 2 || v.capacity == 0) return HICR_ERR_INVALID;
  const unsigned P = v.capacity;
  const unsigned long long t0 = now();
  for (;;) {
    const unsigned first = *next % P;
    for (unsigned base = 0; base < P; base += 32) {
      const unsigned off = base + lane;
      const unsigned p = (first + off) % P;
      bool ready = false;
      if (off < P) {
        const unsigned long long* cnt = v.head + (unsigned long long)p * HICR_NL_STATE_WORDS;
        ready = ld_acquire(cnt + HICR_NL_PUB) != *(volatile const unsigned long long*)(cnt + HICR_NL_CONS);
      }
      const unsigned m = __ballot_sync(0xffffffffu, ready);
      if (m) {
        const unsigned pick = __shfl_sync(0xffffffffu, p, __ffs(m) - 1);
        const int st = hicr_dev_mpsc_nl_pop(v, pick, dst, dst_cap, info, timeout_ns);
        if (st == HICR_OK) *next = (pick + 1) % P;
        return st;
      }
    }
    int give_up = 0;
    if (lane == 0) give_up = now() - t0 > timeout_ns;
    if (__shfl_sync(0xffffffffu, give_up, 0)) return HICR_ERR_TIMEOUT;
    if (lane == 0) __nanosleep(64);
    __syncwarp();
  }
}

#endif /* __CUDACC__ */

#endif /* HICR_DEVICE_CUH */
