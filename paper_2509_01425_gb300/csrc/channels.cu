// SPSC and MPSC channels (HiCR paper Sec. 4.3, Channels frontend).
//
// A channel is a circular buffer (ring) in HBM at the consumer plus 64-bit
// coordination counters, each on its own 128-byte line:
//   SPSC  head = tokens published, tail = tokens consumed;
//         token t lives at ring offset (t mod capacity) * token_size.
//   MPSC  reserve = (ticket mod 2^24) << 40 | (reserved bytes mod 2^40),
//         freed   = bytes freed (mod 2^40), msg_tail = messages freed,
//         plus a metadata ring of max_msgs entries {start, size, producer,
//         seq, ready}. The "locking" mode's exclusive access is one
//         compare-and-swap of `reserve`, taken only when the placement rule
//         (16-byte rounding, skip to the ring start instead of crossing its
//         end, reserved-minus-freed <= ring bytes, in-flight <= max_msgs)
//         finds room; a producer then copies its payload with the warp copy
//         of the memcpy path and publishes the entry with a release store of
//         `ready`. The consumer drains tickets in order and frees with
//         release stores.
//   MPSC non-locking (a dedicated ring per producer): producer i of the
//         channel owns ring i, its metadata ring and the counters reserve
//         (bytes reserved), pub (messages published) -- written only by the
//         producer -- and freed / cons, written only by the consumer. No
//         compare-and-swap: a producer places its messages with the same
//         rule in its own ring and publishes them with one release store of
//         pub; 64-bit absolute counters.
// Ring bytes and max_msgs are powers of two, so positions modulo 2^40 and
// tickets modulo 2^24 map consistently onto the rings.
//
// Host calls run a one-CTA kernel and read its result from a mapped host
// mailbox. The streaming runs launch producers and consumers as one
// cooperative grid (all CTAs resident at once); every wait is bounded by the
// %globaltimer deadline and raises a shared abort flag on expiry.
#include <stddef.h>
#include <string.h>

#include <thread>
#include <vector>

#include "../../include/hicr_channels.h"
#include "channel_common.cuh"
#include "copy.cuh"
#include "hicr_internal.h"
#include "splitmix.cuh"

namespace hicr {

struct Channel {
  int kind = 0;  // 0 SPSC, 1 MPSC (locking), 2 MPSC (non-locking)
  bool live = false;
  uint32_t token_size = 0, capacity = 0;
  uint32_t n_producers = 0, max_msgs = 0;
  uint64_t ring_bytes = 0;
  uint8_t* ring = nullptr;
  void* state = nullptr;
  MpscMeta* meta = nullptr;
  hicr_slot_t ring_slot = 0;
  std::vector<uint32_t> seq;  // host-API producers' next sequence numbers
};

// ---------------------------------------------------------------------------
// Host-call kernels (one CTA, result in the mailbox).
// ---------------------------------------------------------------------------
// Copy n bytes with every warp of the CTA taking an equal share.
__device__ __forceinline__ void cta_copy(uint8_t* d, const uint8_t* s, unsigned long long n) {
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long a = n * w / nw, b = n * (w + 1) / nw;
  if (b > a) warp_copy(d + a, s + a, b - a, lane);
}

__global__ void k_spsc_push_host(SpscView v, const uint8_t* src, unsigned long long k, Mailbox* mb) {
  __shared__ unsigned long long s_head;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned long long h = ld_rlx(&v.st->head.v), t = ld_acq(&v.st->tail.v);
    s_ok = (h - t + k <= v.cap);
    s_head = h;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) mb_post(mb, HICR_ERR_FULL);
    return;
  }
  // at most two contiguous runs: up to the ring end, then from its start
  const unsigned long long first = s_head % v.cap;
  const unsigned long long run1 = min(k, (unsigned long long)v.cap - first);
  cta_copy(v.ring + first * v.ts, src, run1 * v.ts);
  if (k > run1) cta_copy(v.ring, src + run1 * v.ts, (k - run1) * v.ts);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    st_rel(&v.st->head.v, s_head + k);
    mb->v[0] = s_head;
    mb_post(mb, HICR_OK);
  }
}

// op 0 = peek(k), 1 = pop(k), 2 = depth
__global__ void k_spsc_ctl(SpscView v, int op, unsigned long long k, Mailbox* mb) {
  const unsigned long long h = ld_acq(&v.st->head.v), t = ld_acq(&v.st->tail.v);
  const unsigned long long depth = h - t;
  if (op == 2) {
    mb->v[0] = depth;
    mb->v[1] = depth * v.ts;
    mb_post(mb, HICR_OK);
  } else if (op == 0) {
    if (k >= depth) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    mb->v[0] = ((t + k) % v.cap) * v.ts;
    mb->v[1] = v.ts;
    mb->v[2] = 0;
    mb->v[3] = t + k;
    mb_post(mb, HICR_OK);
  } else {
    if (k > depth) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    st_rel(&v.st->tail.v, t + k);
    mb_post(mb, HICR_OK);
  }
}

__global__ void k_mpsc_push_host(MpscView v, unsigned int producer, unsigned int seq, const uint8_t* src,
                                 unsigned long long n, Mailbox* mb) {
  __shared__ unsigned long long s_start, s_ticket;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned long long r = round16(n);
    int ok = 0;
    for (int attempt = 0; attempt < 1000; ++attempt) {
      const unsigned long long W = ld_rlx(&v.st->reserve.v);
      unsigned long long start;
      const unsigned long long end = mpsc_place(W, &r, 1, v.R, &start);
      const unsigned long long freed = ld_acq(&v.st->freed.v);
      const unsigned long long mt = ld_acq(&v.st->msg_tail.v);
      const unsigned long long t0 = W >> 40;
      const unsigned long long inflight = (end - freed) & MASK40;
      const unsigned long long msgs = ((t0 + 1) - mt) & MASK24;
      if (inflight > v.R || msgs > v.M) break;  // FULL under the placement rule
      const unsigned long long nw = (((t0 + 1) & MASK24) << 40) | end;
      if (atomicCAS(&v.st->reserve.v, W, nw) == W) {
        ok = 1;
        s_start = start;
        s_ticket = t0;
        atomicMax(&v.st->max_bytes.v, inflight);
        atomicMax(&v.st->max_msgs.v, msgs);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) mb_post(mb, HICR_ERR_FULL);
    return;
  }
  cta_copy(v.ring + (s_start & (v.R - 1)), src, n);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    MpscMeta* e = v.meta + (s_ticket & (v.M - 1));
    e->start = s_start;
    e->size = (unsigned int)n;
    e->producer = producer;
    e->seq = seq;
    e->flags = 0;
    st_rel(&e->ready, (s_ticket & MASK24) + 1);
    mb->v[0] = s_start & (v.R - 1);
    mb->v[1] = s_ticket;
    mb_post(mb, HICR_OK);
  }
}

// op 0 = peek(k), 1 = pop(k), 2 = depth
__global__ void k_mpsc_ctl(MpscView v, int op, unsigned long long k, Mailbox* mb) {
  const unsigned long long W = ld_acq(&v.st->reserve.v);
  const unsigned long long mt = ld_acq(&v.st->msg_tail.v);
  const unsigned long long freed = ld_acq(&v.st->freed.v);
  const unsigned long long depth = ((W >> 40) - mt) & MASK24;
  if (op == 2) {
    mb->v[0] = depth;
    mb->v[1] = ((W & MASK40) - freed) & MASK40;
    mb_post(mb, HICR_OK);
    return;
  }
  if (op == 0) {
    if (k >= depth) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    const unsigned long long t = mt + k;
    MpscMeta* e = v.meta + (t & (v.M - 1));
    if (ld_acq(&e->ready) != (t & MASK24) + 1) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    mb->v[0] = __ldcg(&e->start) & (v.R - 1);
    mb->v[1] = __ldcg(&e->size);
    mb->v[2] = __ldcg(&e->producer);
    mb->v[3] = __ldcg(&e->seq);
    mb_post(mb, HICR_OK);
    return;
  }
  if (k > depth) {
    mb_post(mb, HICR_ERR_EMPTY);
    return;
  }
  if (k == 0) {
    mb_post(mb, HICR_OK);
    return;
  }
  for (unsigned long long i = 0; i < k; ++i) {
    const unsigned long long t = mt + i;
    if (ld_acq(&v.meta[t & (v.M - 1)].ready) != (t & MASK24) + 1) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
  }
  const MpscMeta* last = v.meta + ((mt + k - 1) & (v.M - 1));
  const unsigned long long end = (__ldcg(&last->start) + round16(__ldcg(&last->size))) & MASK40;
  st_rel(&v.st->freed.v, end);
  st_rel(&v.st->msg_tail.v, mt + k);
  mb_post(mb, HICR_OK);
}

// ---------------------------------------------------------------------------
// Non-locking MPSC layout and host-call kernels.
// ---------------------------------------------------------------------------
struct NlState {
  Line reserve;  // bytes reserved (absolute, including skipped bytes); producer
  Line pub;      // messages published; producer
  Line freed;    // bytes freed; consumer
  Line cons;     // messages consumed; consumer
};
struct NlHead {
  Line max_bytes;  // high-water marks of reserved-minus-freed / in-flight
  Line max_msgs;   // messages over the channel's rings (streaming runs)
};
struct NlMeta {
  unsigned long long start;  // absolute reservation start
  unsigned int size;
  unsigned int seq;
};
static_assert(sizeof(NlMeta) == 16, "non-locking metadata entry is 16 bytes");
// the public description of the non-locking layout (hicr_channels.h)
static_assert(sizeof(hicr_nl_meta_t) == sizeof(NlMeta), "public non-locking metadata layout");
static_assert(sizeof(NlState) == 8 * HICR_NL_STATE_WORDS && offsetof(NlState, reserve) == 8 * HICR_NL_RESERVE &&
                  offsetof(NlState, pub) == 8 * HICR_NL_PUB && offsetof(NlState, freed) == 8 * HICR_NL_FREED &&
                  offsetof(NlState, cons) == 8 * HICR_NL_CONS,
              "public non-locking counter layout");
// the public description of a locking-mode metadata entry (hicr_channels.h)
static_assert(sizeof(hicr_mpsc_meta_t) == sizeof(MpscMeta) && offsetof(hicr_mpsc_meta_t, start) == offsetof(MpscMeta, start) &&
                  offsetof(hicr_mpsc_meta_t, size) == offsetof(MpscMeta, size) &&
                  offsetof(hicr_mpsc_meta_t, producer) == offsetof(MpscMeta, producer) &&
                  offsetof(hicr_mpsc_meta_t, seq) == offsetof(MpscMeta, seq) &&
                  offsetof(hicr_mpsc_meta_t, ready) == offsetof(MpscMeta, ready),
              "public MPSC metadata layout");
struct NlView {
  uint8_t* ring;  // ring i at ring + i * R
  NlHead* head;
  NlState* st;    // st[i]
  NlMeta* meta;   // ring i's entries at meta + i * M
  unsigned long long R;
  unsigned int M;
  unsigned int P;
};

// Placement of k messages with rounded sizes r[] from absolute position b
// (the locking mode's rule on one ring, without the ticket packing).
__device__ __forceinline__ unsigned long long nl_place(unsigned long long b, const unsigned long long* r, int k,
                                                        unsigned long long R, unsigned long long* start) {
  for (int i = 0; i < k; ++i) {
    const unsigned long long pos = b & (R - 1);
    if (pos + r[i] > R) b += R - pos;
    start[i] = b;
    b += r[i];
  }
  return b;
}

__global__ void k_nl_push_host(NlView v, unsigned int producer, unsigned int seq, const uint8_t* src,
                               unsigned long long n, Mailbox* mb) {
  __shared__ unsigned long long s_start, s_pub;
  __shared__ int s_ok;
  NlState* st = v.st + producer;
  if (threadIdx.x == 0) {
    const unsigned long long r = round16(n);
    unsigned long long start;
    const unsigned long long end = nl_place(ld_rlx(&st->reserve.v), &r, 1, v.R, &start);
    const unsigned long long pub = ld_rlx(&st->pub.v);
    const unsigned long long freed = ld_acq(&st->freed.v), cons = ld_acq(&st->cons.v);
    s_ok = end - freed <= v.R && pub + 1 - cons <= v.M;
    s_start = start;
    s_pub = pub;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) mb_post(mb, HICR_ERR_FULL);
    return;
  }
  uint8_t* ring = v.ring + (unsigned long long)producer * v.R;
  cta_copy(ring + (s_start & (v.R - 1)), src, n);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    NlMeta* e = v.meta + (unsigned long long)producer * v.M + (s_pub & (v.M - 1));
    e->start = s_start;
    e->size = (unsigned int)n;
    e->seq = seq;
    st_rel(&st->reserve.v, s_start + round16(n));
    __threadfence();
    st_rel(&st->pub.v, s_pub + 1);
    mb->v[0] = s_start & (v.R - 1);
    mb->v[1] = s_pub;
    mb_post(mb, HICR_OK);
  }
}

// op 0 = peek(k), 1 = pop(k), 2 = depth; the consumer order is "producers in
// index order, each producer's messages oldest first". One thread.
__global__ void k_nl_ctl(NlView v, int op, unsigned long long k, Mailbox* mb) {
  unsigned long long msgs = 0, bytes = 0;
  for (unsigned p = 0; p < v.P; ++p) {
    const NlState* st = v.st + p;
    msgs += ld_acq(&st->pub.v) - ld_acq(&st->cons.v);
    bytes += ld_acq(&st->reserve.v) - ld_acq(&st->freed.v);
  }
  if (op == 2) {
    mb->v[0] = msgs;
    mb->v[1] = bytes;
    mb_post(mb, HICR_OK);
    return;
  }
  if (op == 0 ? k >= msgs : k > msgs) {
    mb_post(mb, HICR_ERR_EMPTY);
    return;
  }
  unsigned long long left = k;
  for (unsigned p = 0; p < v.P; ++p) {
    NlState* st = v.st + p;
    const unsigned long long cons = ld_rlx(&st->cons.v);
    const unsigned long long d = ld_acq(&st->pub.v) - cons;
    const NlMeta* m = v.meta + (unsigned long long)p * v.M;
    if (op == 0) {
      if (left < d) {
        const NlMeta* e = m + ((cons + left) & (v.M - 1));
        mb->v[0] = __ldcg(&e->start) & (v.R - 1);
        mb->v[1] = __ldcg(&e->size);
        mb->v[2] = p;
        mb->v[3] = __ldcg(&e->seq);
        mb_post(mb, HICR_OK);
        return;
      }
      left -= d;
    } else {
      const unsigned long long take = left < d ? left : d;
      if (take) {
        const NlMeta* e = m + ((cons + take - 1) & (v.M - 1));
        st_rel(&st->freed.v, __ldcg(&e->start) + round16(__ldcg(&e->size)));
        st_rel(&st->cons.v, cons + take);
        left -= take;
      }
      if (!left) break;
    }
  }
  mb_post(mb, HICR_OK);
}

// ---------------------------------------------------------------------------
// SPSC streaming: CTA 2i produces into channel i, CTA 2i+1 consumes it.
// ---------------------------------------------------------------------------
struct SpscStreamArgs {
  const SpscView* chans;
  unsigned int n;
  unsigned int batch;
  unsigned long long tokens;
  unsigned long long timeout_ns;
  hicr_spsc_result_t* res;
  unsigned int* abort;
};

static constexpr int SPSC_U = 8;

__global__ void __launch_bounds__(512) k_spsc_stream(SpscStreamArgs a) {
  __shared__ int s_stop;
  __shared__ unsigned long long s_red[2][16];
  const unsigned ci = blockIdx.x >> 1;
  const bool producer = (blockIdx.x & 1u) == 0;
  const SpscView v = a.chans[ci];
  const unsigned vpt = v.ts / 16;  // 16-byte vectors per token
  const unsigned long long wpt = v.ts / 8;
  const unsigned long long key0 = (unsigned long long)ci << 40;
  const unsigned long long deadline = gtime() + a.timeout_ns;
  const unsigned tid = threadIdx.x;
  // The channel starts empty (head == tail); token s of this run has counter
  // value base + s and ring slot (base + s) mod capacity.
  __shared__ unsigned long long s_base;
  if (tid == 0) s_base = ld_acq(producer ? &v.st->head.v : &v.st->tail.v);
  __syncthreads();
  const unsigned long long base = s_base;
  // fast layout when the vectors of a token divide the block
  const bool fast = (blockDim.x % vpt) == 0;
  const unsigned tpi = fast ? blockDim.x / vpt : 1;  // tokens per pass of the block
  const unsigned jv = fast ? tid % vpt : 0, tl0 = fast ? tid / vpt : 0;
  const unsigned long long step = tpi % v.cap;
  unsigned long long cached = base, max_occ = 0, done = 0, mism = 0, dig = 0;
  int stop = 0;
  for (unsigned long long s0 = 0; s0 < a.tokens; s0 += a.batch) {
    const unsigned long long k = min((unsigned long long)a.batch, a.tokens - s0);
    if (tid == 0) {
      stop = 0;
      if (producer) {
        // room for k more tokens: s0 + k - tail <= capacity
        while (base + s0 + k - cached > v.cap) {
          cached = ld_acq(&v.st->tail.v);
          if (base + s0 + k - cached <= v.cap) break;
          if (aborted(a.abort) || gtime() > deadline) { stop = 1; break; }
          __nanosleep(32);
        }
        if (!stop) max_occ = max(max_occ, base + s0 + k - cached);
      } else {
        // k more tokens published: head >= base + s0 + k
        while (cached < base + s0 + k) {
          cached = ld_acq(&v.st->head.v);
          if (cached >= base + s0 + k) break;
          if (aborted(a.abort) || gtime() > deadline) { stop = 1; break; }
          __nanosleep(32);
        }
      }
      if (stop) atomicExch(a.abort, 1u);
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    if (fast) {
      // thread = vector column jv of tokens tl0, tl0 + tpi, ...; ring slots
      // advance by `step` (tpi mod capacity) without a division per vector
      unsigned long long slot = (base + s0 + tl0) % v.cap;
      for (unsigned long long tl = tl0; tl < k; tl += (unsigned long long)SPSC_U * tpi) {
        if (producer) {
#pragma unroll
          for (int u = 0; u < SPSC_U; ++u) {
            const unsigned long long t_ = tl + (unsigned long long)u * tpi;
            if (t_ < k) {
              const unsigned long long word = (s0 + t_) * wpt + 2ull * jv;
              uint4* p = reinterpret_cast<uint4*>(v.ring + slot * v.ts) + jv;
              const unsigned long long w0 = sm64_first_output(key0 + word), w1 = sm64_first_output(key0 + word + 1);
              uint4 x;
              x.x = (unsigned)w0;
              x.y = (unsigned)(w0 >> 32);
              x.z = (unsigned)w1;
              x.w = (unsigned)(w1 >> 32);
              *p = x;
            }
            slot += step;
            if (slot >= v.cap) slot -= v.cap;
          }
        } else {
          uint4 x[SPSC_U];
          unsigned long long sl = slot;
#pragma unroll
          for (int u = 0; u < SPSC_U; ++u) {
            if (tl + (unsigned long long)u * tpi < k)
              x[u] = __ldcg(reinterpret_cast<const uint4*>(v.ring + sl * v.ts) + jv);
            sl += step;
            if (sl >= v.cap) sl -= v.cap;
          }
          slot = sl;
          // Vector u of this pass starts at word W0 + u D (D = tpi wpt), so
          // its digest term w0 (2 word + 1) + w1 (2 word + 3) sums over the
          // pass to (2 W0 + 1) S + 2 D U + 2 W1, with S = sum_u (w0 + w1),
          // U = sum_u u (w0 + w1) (suffix sums, u descending), W1 = sum_u w1
          // (mod 2^64): two products per pass instead of one per vector.
          const unsigned long long W0 = (s0 + tl) * wpt + 2ull * jv;
          unsigned long long S = 0, U = 0, W1 = 0;
#pragma unroll
          for (int u = SPSC_U - 1; u >= 0; --u) {
            const unsigned long long t_ = tl + (unsigned long long)u * tpi;
            if (t_ < k) {
              const unsigned long long word = W0 + (unsigned long long)u * tpi * wpt;
              const unsigned long long w0 = (unsigned long long)x[u].x | ((unsigned long long)x[u].y << 32);
              const unsigned long long w1 = (unsigned long long)x[u].z | ((unsigned long long)x[u].w << 32);
              mism += (w0 != sm64_first_output(key0 + word)) + (w1 != sm64_first_output(key0 + word + 1));
              S += w0 + w1;
              W1 += w1;
            }
            if (u > 0) U += S;
          }
          dig += S * (2ull * W0 + 1ull) + U * (2ull * tpi * wpt) + (W1 << 1);
        }
      }
    } else {
      // general token sizes: one vector per thread per step
      const unsigned long long nv = k * vpt;
      for (unsigned long long q = tid; q < nv; q += blockDim.x) {
        const unsigned long long tok = s0 + q / vpt;
        const unsigned long long word = tok * wpt + (q % vpt) * 2;  // index of the first 8-byte word
        uint4* p = reinterpret_cast<uint4*>(v.ring + ((base + tok) % v.cap) * v.ts) + (q % vpt);
        if (producer) {
          const unsigned long long w0 = sm64_first_output(key0 + word), w1 = sm64_first_output(key0 + word + 1);
          uint4 x;
          x.x = (unsigned)w0;
          x.y = (unsigned)(w0 >> 32);
          x.z = (unsigned)w1;
          x.w = (unsigned)(w1 >> 32);
          *p = x;
        } else {
          const uint4 x = __ldcg(p);
          const unsigned long long w0 = (unsigned long long)x.x | ((unsigned long long)x.y << 32);
          const unsigned long long w1 = (unsigned long long)x.z | ((unsigned long long)x.w << 32);
          mism += (w0 != sm64_first_output(key0 + word)) + (w1 != sm64_first_output(key0 + word + 1));
          dig += (w0 + w1) * (2ull * word + 1ull) + (w1 << 1);
        }
      }
    }
    // the barrier orders every thread's ring accesses before thread 0's
    // release store, which is cumulative: no per-thread fence is needed
    __syncthreads();
    if (tid == 0) st_rel(producer ? &v.st->head.v : &v.st->tail.v, base + s0 + k);
    done = s0 + k;
  }
  // block reduction of the consumer's counts
  for (int o = 16; o > 0; o >>= 1) {
    mism += __shfl_xor_sync(FULLM, mism, o);
    dig += __shfl_xor_sync(FULLM, dig, o);
  }
  if ((tid & 31) == 0) {
    s_red[0][tid >> 5] = mism;
    s_red[1][tid >> 5] = dig;
  }
  __syncthreads();
  if (tid == 0) {
    hicr_spsc_result_t* r = a.res + ci;
    if (producer) {
      r->pushed = done;
      r->max_occupancy = max_occ;
    } else {
      unsigned long long m = 0, d = 0;
      for (unsigned w = 0; w < blockDim.x / 32; ++w) {
        m += s_red[0][w];
        d += s_red[1][w];
      }
      r->popped = done;
      r->mismatches = m;
      r->digest = d;
    }
    if (s_stop) r->status = HICR_ERR_TIMEOUT;
  }
}

// ---------------------------------------------------------------------------
// MPSC streaming: CTAs [0, n_cons) consume, the rest hold one producer per
// warp; producer p feeds consumer p mod n_cons.
// ---------------------------------------------------------------------------
struct MpscStreamArgs {
  const MpscView* chans;
  unsigned int n_cons;
  unsigned int n_prod;
  unsigned int mpp;
  unsigned int group;
  const unsigned long long* sizes;
  const unsigned long long* src_off;
  const uint8_t* staging;
  unsigned long long timeout_ns;
  hicr_mpsc_log_t* log;
  unsigned long long log_stride;
  hicr_mpsc_result_t* res;
  unsigned int* abort;
  unsigned int G;                  // CTAs per consumer
  unsigned long long* claim;       // per consumer (stride 16 words): next unclaimed ticket
  const unsigned long long* base;  // per consumer: first ticket of the run
  unsigned int pw;                 // producer warps per producer CTA
  const int* bad;                  // verdict of the pre-stream check (nonzero: the run does not start)
};

static constexpr int MPSC_MAX_GROUP = 8;
// Producer warps copy their groups through PROD_NST shared-memory stages of
// PROD_STG bytes each (bulk copies); a producer CTA holds at most PROD_WARPS
// producer warps.
static constexpr unsigned PROD_NST = 2, PROD_STG = 6144, PROD_WARPS = 16;
static constexpr size_t PROD_SMEM = (size_t)PROD_WARPS * PROD_NST * (PROD_STG + 8);
static constexpr unsigned long long PROD_WAIT_NS = 2000000000ull;  // bound of one stage wait

// The warp's stages and mbarriers in the dynamic shared memory of a producer
// CTA; lane 0 initialises the mbarriers.
__device__ __forceinline__ void prod_stages(uint8_t* smem, unsigned warp, unsigned lane, uint8_t** stage,
                                            unsigned long long** bars) {
  *stage = smem + (size_t)warp * PROD_NST * PROD_STG;
  *bars = reinterpret_cast<unsigned long long*>(smem + (size_t)PROD_WARPS * PROD_NST * PROD_STG) + warp * PROD_NST;
  if (lane == 0) {
    for (unsigned k = 0; k < PROD_NST; ++k) mbar_init(*bars + k);
    mbar_init_fence();
  }
  __syncwarp();
}

__device__ void mpsc_producer(const MpscStreamArgs& a, unsigned p, unsigned lane, unsigned long long deadline,
                              uint8_t* stage, unsigned long long* bars) {
  unsigned phase = 0;
  const unsigned c = p % a.n_cons;
  const MpscView v = a.chans[c];
  const unsigned long long half = v.R / 2;
  unsigned long long freed = 0, mt = 0, cas_fail = 0, room_wait = 0;
  if (lane == 0) {
    freed = ld_acq(&v.st->freed.v);
    mt = ld_acq(&v.st->msg_tail.v);
  }
  for (unsigned s = 0; s < a.mpp;) {
    // the group: up to `group` (and at most max_msgs) messages whose rounded
    // sizes sum to <= R/2, so that it always fits an emptied ring
    unsigned long long r[MPSC_MAX_GROUP], st[MPSC_MAX_GROUP] = {};
    int k = 0;
    unsigned long long sum = 0;
    for (; k < (int)a.group && (unsigned)k < v.M && s + k < a.mpp; ++k) {
      const unsigned long long rk = round16(a.sizes[(unsigned long long)p * a.mpp + s + k]);
      if (k > 0 && sum + rk > half) break;
      r[k] = rk;
      sum += rk;
    }
    unsigned long long W = 0, end = 0;
    int stop = 0;
    if (lane == 0) {
      // freed / msg_tail only grow, so a stale copy can only under-report
      // room; they are re-read only when the cached copies say "full", with
      // an exponentially growing pause so that waiting producers do not
      // crowd the lines the consumer releases.
      unsigned sleep_ns = 32;
      for (;;) {
        W = ld_rlx(&v.st->reserve.v);
        end = mpsc_place(W, r, k, v.R, st);
        const unsigned long long t0 = W >> 40;
        bool room = ((end - freed) & MASK40) <= v.R && (((t0 + k) - mt) & MASK24) <= v.M;
        if (!room) {
          freed = ld_acq(&v.st->freed.v);
          mt = ld_acq(&v.st->msg_tail.v);
          room = ((end - freed) & MASK40) <= v.R && (((t0 + k) - mt) & MASK24) <= v.M;
        }
        if (room) {
          const unsigned long long nw = (((t0 + k) & MASK24) << 40) | end;
          if (atomicCAS(&v.st->reserve.v, W, nw) == W) break;
          ++cas_fail;
        } else {
          ++room_wait;
        }
        if (aborted(a.abort) || gtime() > deadline) {
          stop = 1;
          atomicExch(a.abort, 1u);
          break;
        }
        if (!room) {
          __nanosleep(sleep_ns);
          sleep_ns = min(sleep_ns * 2, 4096u);
        }
      }
    }
    stop = __shfl_sync(FULLM, stop, 0);
    if (stop) {
      if (lane == 0) a.res[c].status = HICR_ERR_TIMEOUT;
      return;
    }
    W = __shfl_sync(FULLM, W, 0);
    const unsigned long long t0 = W >> 40;
    // lane i < k takes message i of the group
    unsigned long long my_st = 0;
#pragma unroll
    for (int i = 0; i < MPSC_MAX_GROUP; ++i) {
      const unsigned long long si = __shfl_sync(FULLM, st[i], 0);
      if (lane == (unsigned)i) my_st = si;
    }
    const unsigned long long idx = (unsigned long long)p * a.mpp + s + lane;
    const bool mine = lane < (unsigned)k;
    const unsigned long long my_n = mine ? a.sizes[idx] : 0;
    if (!group_copy_bulk<PROD_NST, PROD_STG>(mine ? v.ring + (my_st & (v.R - 1)) : nullptr,
                                             mine ? a.staging + a.src_off[idx] : nullptr, my_n, k, lane, stage, bars,
                                             phase, PROD_WAIT_NS)) {
      if (lane == 0) {
        atomicExch(a.abort, 1u);
        a.res[c].status = HICR_ERR_TIMEOUT;
      }
      return;
    }
    __threadfence();
    __syncwarp();
    if (mine) {
      const unsigned long long t = t0 + lane;
      MpscMeta* e = v.meta + (t & (v.M - 1));
      e->start = my_st;
      e->size = (unsigned int)my_n;
      e->producer = p;
      e->seq = s + lane;
      e->flags = 0;
      st_rel(&e->ready, (t & MASK24) + 1);
    }
    if (lane == 0) {
      atomicMax(&v.st->max_bytes.v, (end - freed) & MASK40);
      atomicMax(&v.st->max_msgs.v, ((t0 + k) - mt) & MASK24);
    }
    s += k;
  }
  if (lane == 0) {
    if (cas_fail) atomicAdd((unsigned long long*)&a.res[c].cas_failures, cas_fail);
    if (room_wait) atomicAdd((unsigned long long*)&a.res[c].room_waits, room_wait);
  }
}

// Consumer c: G CTAs. Each round, a CTA claims the next window of up to
// MPSC_WIN tickets that producers have already reserved (so every one of them
// will be published without waiting for ring space) by advancing the
// consumer's claim counter, and
//   A. warps acquire the tickets' `ready` words and stage their metadata in
//      shared memory;
//   B. each warp digests an equal share of the window's concatenated
//      payloads, streamed through its shared-memory stages by bulk loads;
//   C. warps write the log entries (index = ticket - first ticket), then one
//      thread waits until msg_tail reaches the window's first ticket (the
//      previous window is freed), frees every byte up to the window's last
//      message and advances msg_tail (release stores).
// Windows of one consumer are digested side by side; frees stay in ticket
// order.
static constexpr int MPSC_WIN = 64;

__device__ void mpsc_consumer(const MpscStreamArgs& a, unsigned c, unsigned long long deadline, uint8_t* stage,
                              unsigned long long* bars) {
  unsigned phase = 0;  // parity bits of this warp's stages
  // s_stop / s_done are written only by thread 0 before the first barrier of
  // a round; phase-A waits that give up write s_abort_a, read after the
  // second barrier and cleared by thread 0 at the start of the next round
  // (after the round's last barrier), so no thread can see a flag meant for a
  // later check and leave while others wait at a barrier.
  __shared__ int s_stop, s_abort_a, s_done;
  __shared__ unsigned long long s_avail, s_t;
  __shared__ unsigned long long s_start[MPSC_WIN], s_bpre[MPSC_WIN + 1], s_dig[MPSC_WIN];
  __shared__ unsigned int s_size[MPSC_WIN], s_prod[MPSC_WIN], s_seq[MPSC_WIN];
  const MpscView v = a.chans[c];
  const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, nwarp = blockDim.x >> 5;
  // messages this consumer receives: producers c, c + n_cons, ...
  const unsigned long long nprod = (a.n_prod > c) ? (a.n_prod - c + a.n_cons - 1) / a.n_cons : 0;
  const unsigned long long expect = nprod * a.mpp;
  const unsigned long long win_max = min((unsigned long long)MPSC_WIN, (unsigned long long)(v.M / 2 ? v.M / 2 : 1));
  const unsigned long long base = a.base[c];  // first ticket of the run
  unsigned long long* claim = a.claim + 16ull * c;
  if (tid == 0) s_abort_a = 0;
  unsigned long long consumed = 0, windows = 0, bytes = 0;
  hicr_mpsc_log_t* log = a.log + a.log_stride * c;
  unsigned long long ns_a = 0, ns_b = 0, ns_c = 0, tm = 0;
  int stop_c = 0;  // thread 0: a phase-C wait gave up
  for (;;) {
    if (tid == 0) {
      tm = gtime();
      int stop = stop_c, done = 0;
      unsigned long long t = 0, n = 0;
      while (!stop) {
        t = ld_acq(claim);
        if (t - base >= expect) {
          done = 1;
          break;
        }
        const unsigned long long W = ld_acq(&v.st->reserve.v);
        const unsigned long long avail = ((W >> 40) - t) & MASK24;
        if (avail) {
          n = min(min(avail, win_max), expect - (t - base));
          if (atomicCAS(claim, t, t + n) == t) break;
          continue;
        }
        if (aborted(a.abort) || gtime() > deadline) {
          stop = 1;
          atomicExch(a.abort, 1u);
          break;
        }
        __nanosleep(64);
      }
      s_t = t;
      s_avail = n;
      s_stop = stop;
      s_done = done;
      s_abort_a = 0;
    }
    __syncthreads();
    if (s_stop || s_done) break;
    const unsigned long long t = s_t;
    const unsigned navail = (unsigned)s_avail;
    // A. acquire and stage metadata
    for (unsigned j = warp; j < navail; j += nwarp) {
      const unsigned long long tk = t + j;
      MpscMeta* e = v.meta + (tk & (v.M - 1));
      if (lane == 0) {
        int stop = 0;
        while (ld_acq(&e->ready) != (tk & MASK24) + 1) {
          if (aborted(a.abort) || gtime() > deadline) {
            stop = 1;
            atomicExch(a.abort, 1u);
            break;
          }
          __nanosleep(32);
        }
        if (stop) {
          s_abort_a = 1;
        } else {
          s_start[j] = __ldcg(&e->start);
          s_size[j] = __ldcg(&e->size);
          s_prod[j] = __ldcg(&e->producer);
          s_seq[j] = __ldcg(&e->seq);
          s_dig[j] = 0;
        }
      }
    }
    __syncthreads();
    if (s_abort_a) break;
    if (tid == 0) {
      const unsigned long long x = gtime();
      ns_a += x - tm;
      tm = x;
    }
    if (warp == 0) {
      // exclusive prefix of the messages' bodies (sizes rounded up to 16
      // bytes; navail <= 64: two values per lane)
      const unsigned long long p0 = lane < navail ? round16(s_size[lane]) : 0;
      const unsigned long long p1 = lane + 32 < navail ? round16(s_size[lane + 32]) : 0;
      unsigned long long x0 = p0, x1 = p1;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y0 = __shfl_up_sync(FULLM, x0, o), y1 = __shfl_up_sync(FULLM, x1, o);
        if (lane >= (unsigned)o) {
          x0 += y0;
          x1 += y1;
        }
      }
      const unsigned long long tot0 = __shfl_sync(FULLM, x0, 31);
      s_bpre[lane] = x0 - p0;
      s_bpre[lane + 32] = tot0 + x1 - p1;
      if (lane == 31) s_bpre[64] = tot0 + x1;
    }
    __syncthreads();
    // B. digest: warp w takes the w-th of nwarp equal (16-byte aligned) shares
    // of the window's concatenated bodies and streams it through its stages
    // by bulk loads, adding each message part's digest to the message's
    // shared accumulator.
    {
      const unsigned long long T = s_bpre[navail];
      const unsigned long long lo = (T * warp / nwarp) & ~15ull;
      const unsigned long long hi = warp + 1 == nwarp ? T : (T * (warp + 1) / nwarp) & ~15ull;
      if (hi > lo) {
        unsigned jl = 0, jh = navail;  // largest j < navail with s_bpre[j] <= lo
        while (jh - jl > 1) {
          const unsigned mid = (jl + jh) >> 1;
          if (s_bpre[mid] <= lo) jl = mid;
          else jh = mid;
        }
        auto msg = [&](int j) {
          return DigestMsg{v.ring + (s_start[j] & (v.R - 1)), s_bpre[j + 1] - s_bpre[j], s_size[j]};
        };
        auto sink = [&](int j, unsigned long long d) {
          if (lane == 0) atomicAdd(&s_dig[j], d);
        };
        if (!warp_digest_bulk<PROD_NST, PROD_STG>((int)jl, lo - s_bpre[jl], hi - lo, msg, sink, lane, stage, bars,
                                                  phase, PROD_WAIT_NS)) {
          if (lane == 0) {
            s_abort_a = 1;
            atomicExch(a.abort, 1u);
          }
        }
      }
    }
    __syncthreads();
    if (s_abort_a) break;
    if (tid == 0) {
      const unsigned long long x = gtime();
      ns_b += x - tm;
      tm = x;
    }
    // C. log, then free up to the window's last message once the previous
    // window is freed
    for (unsigned j = tid; j < navail; j += blockDim.x) {
      hicr_mpsc_log_t L;
      L.producer = s_prod[j];
      L.seq = s_seq[j];
      L.size = s_size[j];
      L.reserved = 0;
      L.offset = s_start[j] & (v.R - 1);
      L.digest = s_dig[j];
      log[t - base + j] = L;
    }
    if (tid == 0) {
      unsigned long long b = 0;
      for (unsigned j = 0; j < navail; ++j) b += s_size[j];
      bytes += b;
      while (ld_acq(&v.st->msg_tail.v) != t) {
        if (aborted(a.abort) || gtime() > deadline) {
          stop_c = 1;
          atomicExch(a.abort, 1u);
          break;
        }
        __nanosleep(32);
      }
      if (!stop_c) {
        fence_proxy_async_global();  // the window's bulk reads before the free
        st_rel(&v.st->freed.v, (s_start[navail - 1] + round16(s_size[navail - 1])) & MASK40);
        st_rel(&v.st->msg_tail.v, t + navail);
      }
    }
    consumed += navail;
    ++windows;
    __syncthreads();
    if (tid == 0) ns_c += gtime() - tm;
  }
  if (tid == 0) {
    hicr_mpsc_result_t* r = a.res + c;
    atomicAdd((unsigned long long*)&r->consumed, consumed);
    atomicAdd((unsigned long long*)&r->bytes, bytes);
    atomicAdd((unsigned long long*)&r->windows, windows);
    atomicAdd((unsigned long long*)&r->consumer_ns[0], ns_a);
    atomicAdd((unsigned long long*)&r->consumer_ns[1], ns_b);
    atomicAdd((unsigned long long*)&r->consumer_ns[2], ns_c);
    if (s_stop || s_abort_a || stop_c) r->status = HICR_ERR_TIMEOUT;
  }
}

static constexpr unsigned MPSC_THREADS = 512;
static_assert(MPSC_THREADS / 32 <= PROD_WARPS, "every warp of a producer CTA needs its stages");

__global__ void __launch_bounds__(MPSC_THREADS) k_mpsc_stream(MpscStreamArgs a) {
  if (*(volatile const int*)a.bad) return;  // the check kernel, earlier in the stream, rejected the run
  const unsigned long long deadline = gtime() + a.timeout_ns;
  const unsigned ncta = a.n_cons * a.G;
  extern __shared__ __align__(128) uint8_t prod_smem[];
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint8_t* stage;
  unsigned long long* bars;
  if (blockIdx.x < ncta) {
    prod_stages(prod_smem, warp, lane, &stage, &bars);
    mpsc_consumer(a, blockIdx.x / a.G, deadline, stage, bars);
    return;
  }
  const unsigned p = (blockIdx.x - ncta) * a.pw + warp;
  if (warp < a.pw && p < a.n_prod) {
    prod_stages(prod_smem, warp, lane, &stage, &bars);
    mpsc_producer(a, p, lane, deadline, stage, bars);
  }
}

// Checks run before a stream: every message lies inside the staging slot and
// is at most half its ring (so a reservation always fits an emptied ring).
__global__ void k_mpsc_check(MpscStreamArgs a, unsigned long long staging_size, int* bad) {
  const unsigned long long total = (unsigned long long)a.n_prod * a.mpp;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long n = a.sizes[i], off = a.src_off[i];
    const unsigned c = (unsigned)((i / a.mpp) % a.n_cons);
    if (off > staging_size || n > staging_size - off) atomicCAS(bad, 0, HICR_ERR_BOUNDS);
    else if (round16(n) > a.chans[c].R / 2 || n > 0xffffffffull) atomicCAS(bad, 0, HICR_ERR_TOO_LARGE);
  }
}

// Set-up and wrap-up of a locking stream, one thread per channel: before the
// run, clear the high-water marks and start the consumer's claim counter and
// first ticket at msg_tail (the channels are idle: stream order); after it,
// copy the marks into the results.
__global__ void k_mpsc_stream_prep(const MpscView* v, unsigned n, unsigned long long* claim,
                                   unsigned long long* base) {
  for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
    MpscState* st = v[i].st;
    st->max_bytes.v = 0;
    st->max_msgs.v = 0;
    const unsigned long long mt = st->msg_tail.v;
    claim[16ull * i] = mt;
    base[i] = mt;
  }
}
__global__ void k_mpsc_stream_marks(const MpscView* v, unsigned n, hicr_mpsc_result_t* res) {
  for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
    res[i].max_inflight_bytes = v[i].st->max_bytes.v;
    res[i].max_inflight_msgs = v[i].st->max_msgs.v;
  }
}

// ---------------------------------------------------------------------------
// Non-locking MPSC streaming: CTAs [0, n_cons * G) consume (G per channel),
// the rest hold one producer per warp; producer p uses ring p / n_cons of
// channel p mod n_cons. Consumer warp w of the channel's G * W warps owns its
// rings w, w + G*W, ... (at most 32: lane l keeps the counters of the l-th),
// polls them and drains whichever hold published messages. No CTA barrier
// anywhere, so each warp leaves on its own once its rings are drained.
// ---------------------------------------------------------------------------
struct NlStreamArgs {
  const NlView* chans;
  unsigned int n_cons;
  unsigned int G;  // CTAs per consumer
  unsigned int n_prod;
  unsigned int mpp;
  unsigned int group;
  const unsigned long long* sizes;
  const unsigned long long* src_off;
  const uint8_t* staging;
  unsigned long long timeout_ns;
  hicr_mpsc_log_t* log;
  unsigned long long log_stride;
  unsigned long long* log_count;  // per consumer
  hicr_mpsc_result_t* res;
  unsigned int* abort;
  unsigned int pw;  // producer warps per producer CTA
  const int* bad;   // verdict of the pre-stream check (nonzero: the run does not start)
};

__device__ void nl_producer(const NlStreamArgs& a, unsigned p, unsigned lane, unsigned long long deadline,
                            uint8_t* stage, unsigned long long* bars) {
  unsigned phase = 0;
  const unsigned c = p % a.n_cons, i = p / a.n_cons;
  const NlView v = a.chans[c];
  NlState* st = v.st + i;
  uint8_t* ring = v.ring + (unsigned long long)i * v.R;
  NlMeta* meta = v.meta + (unsigned long long)i * v.M;
  const unsigned long long half = v.R / 2;
  // lane 0 holds the producer's counters; freed / cons are cached and re-read
  // only when the cached copies say "full" (they only grow)
  unsigned long long res = 0, pub = 0, freed = 0, cons = 0, max_b = 0, max_m = 0, room_wait = 0;
  if (lane == 0) {
    res = ld_rlx(&st->reserve.v);
    pub = ld_rlx(&st->pub.v);
    freed = ld_acq(&st->freed.v);
    cons = ld_acq(&st->cons.v);
  }
  for (unsigned s = 0; s < a.mpp;) {
    unsigned long long r[MPSC_MAX_GROUP], sa[MPSC_MAX_GROUP] = {};
    int k = 0;
    unsigned long long sum = 0;
    for (; k < (int)a.group && (unsigned)k < v.M && s + k < a.mpp; ++k) {
      const unsigned long long rk = round16(a.sizes[(unsigned long long)p * a.mpp + s + k]);
      if (k > 0 && sum + rk > half) break;
      r[k] = rk;
      sum += rk;
    }
    unsigned long long end = 0;
    int stop = 0;
    if (lane == 0) {
      end = nl_place(res, r, k, v.R, sa);
      unsigned sleep_ns = 32;
      while (end - freed > v.R || pub + k - cons > v.M) {
        freed = ld_acq(&st->freed.v);
        cons = ld_acq(&st->cons.v);
        if (end - freed <= v.R && pub + k - cons <= v.M) break;
        ++room_wait;
        if (aborted(a.abort) || gtime() > deadline) {
          stop = 1;
          atomicExch(a.abort, 1u);
          break;
        }
        __nanosleep(sleep_ns);
        sleep_ns = min(sleep_ns * 2, 4096u);
      }
      max_b = max(max_b, end - freed);
      max_m = max(max_m, pub + k - cons);
    }
    stop = __shfl_sync(FULLM, stop, 0);
    if (stop) {
      if (lane == 0) a.res[c].status = HICR_ERR_TIMEOUT;
      return;
    }
    const unsigned long long pub0 = __shfl_sync(FULLM, pub, 0);
    // lane j < k takes message j of the group
    unsigned long long my_sa = 0;
#pragma unroll
    for (int j = 0; j < MPSC_MAX_GROUP; ++j) {
      const unsigned long long sj = __shfl_sync(FULLM, sa[j], 0);
      if (lane == (unsigned)j) my_sa = sj;
    }
    const unsigned long long idx = (unsigned long long)p * a.mpp + s + lane;
    const bool mine = lane < (unsigned)k;
    const unsigned long long my_n = mine ? a.sizes[idx] : 0;
    if (!group_copy_bulk<PROD_NST, PROD_STG>(mine ? ring + (my_sa & (v.R - 1)) : nullptr,
                                             mine ? a.staging + a.src_off[idx] : nullptr, my_n, k, lane, stage, bars,
                                             phase, PROD_WAIT_NS)) {
      if (lane == 0) {
        atomicExch(a.abort, 1u);
        a.res[c].status = HICR_ERR_TIMEOUT;
      }
      return;
    }
    if (mine) {
      NlMeta* e = meta + ((pub0 + lane) & (v.M - 1));
      e->start = my_sa;
      e->size = (unsigned int)my_n;
      e->seq = s + lane;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) {
      pub += k;
      res = end;
      st_rel(&st->pub.v, pub);
    }
    s += k;
  }
  if (lane == 0) {
    st_rel(&st->reserve.v, res);
    atomicMax(&v.head->max_bytes.v, max_b);
    atomicMax(&v.head->max_msgs.v, max_m);
    if (room_wait) atomicAdd((unsigned long long*)&a.res[c].room_waits, room_wait);
  }
}

__device__ void nl_consumer_warp(const NlStreamArgs& a, unsigned c, unsigned gw, unsigned nw, unsigned lane,
                                 unsigned long long deadline, uint8_t* stage, unsigned long long* bars) {
  unsigned phase = 0;  // parity bits of this warp's stages
  const NlView v = a.chans[c];
  const unsigned nring = a.n_prod > c ? (a.n_prod - c + a.n_cons - 1) / a.n_cons : 0;
  const unsigned owned = nring > gw ? (nring - gw + nw - 1) / nw : 0;  // <= 32 (host check)
  const bool mine = lane < owned;
  const unsigned ring_l = gw + lane * nw;  // this lane's ring
  NlState* st_l = mine ? v.st + ring_l : nullptr;
  unsigned long long cons = mine ? ld_acq(&st_l->cons.v) : 0, pubc = cons;
  unsigned long long left = mine ? a.mpp : 0;  // messages still to take from this lane's ring
  unsigned long long consumed = 0, bytes = 0, batches = 0, idle_ns = 0;
  hicr_mpsc_log_t* log = a.log + a.log_stride * c;
  int stop = 0;
  for (;;) {
    if (mine && left && pubc == cons) pubc = ld_acq(&st_l->pub.v);
    unsigned ready = __ballot_sync(FULLM, left != 0 && pubc != cons);
    if (!ready) {
      const unsigned pending = __ballot_sync(FULLM, left != 0);
      if (!pending) break;
      if (lane == 0) {
        const unsigned long long t = gtime();
        stop = aborted(a.abort) || t > deadline;
        if (stop) atomicExch(a.abort, 1u);
        __nanosleep(64);
        idle_ns += gtime() - t;
      }
      stop = __shfl_sync(FULLM, stop, 0);
      if (stop) break;
      continue;
    }
    __syncwarp();  // order the lanes' acquire loads before the reads below
    while (ready) {
      const unsigned L = __ffs(ready) - 1;
      ready &= ready - 1;
      const unsigned ring = gw + L * nw;
      const unsigned long long c0 = __shfl_sync(FULLM, cons, L);
      const unsigned long long avail = __shfl_sync(FULLM, min(pubc - cons, left), L);
      const unsigned k = (unsigned)min(avail, 32ull);  // >= 1
      const NlMeta* m = v.meta + (unsigned long long)ring * v.M;
      unsigned long long e_start = 0;
      unsigned int e_size = 0, e_seq = 0;
      if (lane < k) {
        const NlMeta* e = m + ((c0 + lane) & (v.M - 1));
        e_start = __ldcg(&e->start);
        e_size = __ldcg(&e->size);
        e_seq = __ldcg(&e->seq);
      }
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(a.log_count + c, (unsigned long long)k);
      base = __shfl_sync(FULLM, base, 0);
      const uint8_t* rb = v.ring + (unsigned long long)ring * v.R;
      // the batch's bodies, digested by bulk loads; lane j collects message j's
      unsigned long long total = lane < k ? round16(e_size) : 0;
      for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(FULLM, total, o);
      auto msg = [&](int j) {
        const unsigned long long sj = __shfl_sync(FULLM, e_start, j);
        const unsigned long long n = __shfl_sync(FULLM, e_size, j);
        return DigestMsg{rb + (sj & (v.R - 1)), round16(n), n};
      };
      unsigned long long my_d = 0;
      auto sink = [&](int j, unsigned long long d) {
        if (lane == (unsigned)j) my_d += d;
      };
      if (!warp_digest_bulk<PROD_NST, PROD_STG>(0, 0, total, msg, sink, lane, stage, bars, phase, PROD_WAIT_NS)) {
        if (lane == 0) atomicExch(a.abort, 1u);
        stop = 1;
        break;
      }
      if (lane < k) {
        hicr_mpsc_log_t E;
        E.producer = ring * a.n_cons + c;
        E.seq = e_seq;
        E.size = e_size;
        E.reserved = 0;
        E.offset = e_start & (v.R - 1);
        E.digest = my_d;
        log[base + lane] = E;
        bytes += e_size;
      }
      // free every byte up to the batch's last message
      const unsigned long long s_last = __shfl_sync(FULLM, e_start, k - 1);
      const unsigned long long n_last = __shfl_sync(FULLM, e_size, k - 1);
      __syncwarp();
      if (lane == L) {
        fence_proxy_async_global();  // the batch's bulk reads before the free
        st_rel(&st_l->freed.v, s_last + round16(n_last));
        cons += k;
        st_rel(&st_l->cons.v, cons);
        left -= k;
      }
      consumed += k;
      ++batches;
    }
    if (stop) break;  // a bulk-load wait gave up
  }
  for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(FULLM, bytes, o);
  if (lane == 0) {
    hicr_mpsc_result_t* r = a.res + c;
    atomicAdd((unsigned long long*)&r->consumed, consumed);
    atomicAdd((unsigned long long*)&r->bytes, bytes);
    atomicAdd((unsigned long long*)&r->windows, batches);
    atomicAdd((unsigned long long*)&r->consumer_ns[0], idle_ns);
    if (stop) r->status = HICR_ERR_TIMEOUT;
  }
}

__global__ void __launch_bounds__(MPSC_THREADS) k_nl_stream(NlStreamArgs a) {
  if (*(volatile const int*)a.bad) return;  // the check kernel, earlier in the stream, rejected the run
  const unsigned long long deadline = gtime() + a.timeout_ns;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const unsigned ncta = a.n_cons * a.G;
  extern __shared__ __align__(128) uint8_t prod_smem[];
  uint8_t* stage;
  unsigned long long* bars;
  if (blockIdx.x < ncta) {
    const unsigned c = blockIdx.x / a.G, g = blockIdx.x % a.G;
    prod_stages(prod_smem, warp, lane, &stage, &bars);
    nl_consumer_warp(a, c, g * W + warp, a.G * W, lane, deadline, stage, bars);
    return;
  }
  const unsigned p = (blockIdx.x - ncta) * a.pw + warp;
  if (warp < a.pw && p < a.n_prod) {
    prod_stages(prod_smem, warp, lane, &stage, &bars);
    nl_producer(a, p, lane, deadline, stage, bars);
  }
}

// The pre-stream checks of k_mpsc_check against the per-producer rings.
__global__ void k_nl_check(NlStreamArgs a, unsigned long long staging_size, int* bad) {
  const unsigned long long total = (unsigned long long)a.n_prod * a.mpp;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long n = a.sizes[i], off = a.src_off[i];
    const unsigned c = (unsigned)((i / a.mpp) % a.n_cons);
    if (off > staging_size || n > staging_size - off) atomicCAS(bad, 0, HICR_ERR_BOUNDS);
    else if (round16(n) > a.chans[c].R / 2 || n > 0xffffffffull) atomicCAS(bad, 0, HICR_ERR_TOO_LARGE);
  }
}

// The same set-up and wrap-up for a non-locking stream: the channel-wide
// high-water marks live in the channel's head.
__global__ void k_nl_stream_prep(const NlView* v, unsigned n) {
  for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
    v[i].head->max_bytes.v = 0;
    v[i].head->max_msgs.v = 0;
  }
}
__global__ void k_nl_stream_marks(const NlView* v, unsigned n, hicr_mpsc_result_t* res) {
  for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
    res[i].max_inflight_bytes = v[i].head->max_bytes.v;
    res[i].max_inflight_msgs = v[i].head->max_msgs.v;
  }
}

// ---------------------------------------------------------------------------
// Ping-pong: CTAs [0, G) are agent A, [G, 2G) agent B. Round k: A's CTAs copy
// their share of the message into B's buffer and count themselves in
// (arrive_a); B's CTAs wait for arrive_a >= k*G, echo their share into A's
// buffer and count in (arrive_b); A waits for arrive_b >= k*G.
// ---------------------------------------------------------------------------
struct PingArgs {
  const uint8_t* msg;
  uint8_t* buf_a;
  uint8_t* buf_b;
  unsigned long long bytes;
  unsigned int G;
  unsigned int rounds;   // warm-up + timed
  unsigned int warmup;
  unsigned long long timeout_ns;
  unsigned long long* arrive;  // [0] A, [16] B (separate lines)
  unsigned long long* times;   // [0] start of the first timed round, [1] end of the last
  unsigned int* abort;
};

__global__ void __launch_bounds__(512) k_pingpong(PingArgs a) {
  __shared__ int s_stop;
  const unsigned side = blockIdx.x / a.G, g = blockIdx.x % a.G;
  const unsigned long long lo = a.bytes * g / a.G, hi = a.bytes * (g + 1) / a.G;
  unsigned long long* mine = a.arrive + (side ? 16 : 0);
  unsigned long long* peer = a.arrive + (side ? 0 : 16);
  const unsigned long long deadline = gtime() + a.timeout_ns;
  for (unsigned k = 1; k <= a.rounds; ++k) {
    if (side == 0 && g == 0 && threadIdx.x == 0 && k == a.warmup + 1) a.times[0] = gtime();
    if (side == 1) {
      // B: wait for A's k-th message
      if (threadIdx.x == 0) {
        int stop = 0;
        while (ld_acq(peer) < (unsigned long long)k * a.G) {
          if (aborted(a.abort) || gtime() > deadline) {
            stop = 1;
            atomicExch(a.abort, 1u);
            break;
          }
        }
        s_stop = stop;
      }
      __syncthreads();
      if (s_stop) return;
      cta_copy(a.buf_a + lo, a.buf_b + lo, hi - lo);  // echo
    } else {
      cta_copy(a.buf_b + lo, a.msg + lo, hi - lo);  // send
    }
    // barrier, then one cumulative release by thread 0 (no per-thread fence)
    __syncthreads();
    if (threadIdx.x == 0) red_add_rel(mine, 1ull);
    if (side == 0) {
      // A: wait for the echo of round k
      if (threadIdx.x == 0) {
        int stop = 0;
        while (ld_acq(peer) < (unsigned long long)k * a.G) {
          if (aborted(a.abort) || gtime() > deadline) {
            stop = 1;
            atomicExch(a.abort, 1u);
            break;
          }
        }
        s_stop = stop;
      }
      __syncthreads();
      if (s_stop) return;
    }
  }
  if (side == 0 && g == 0 && threadIdx.x == 0) a.times[1] = gtime();
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static Channel* get(Instance* in, hicr_channel_t ch) {
  if (ch >= in->channels.size() || !in->channels[ch] || !in->channels[ch]->live) return nullptr;
  return in->channels[ch];
}

static hicr_status mailbox(Instance* in, Mailbox** host, Mailbox** dev) {
  if (!in->mbox_host) {
    void* p = nullptr;
    HICR_CUDA(in, cudaHostAlloc(&p, 4096, cudaHostAllocMapped));
    void* d = nullptr;
    HICR_CUDA(in, cudaHostGetDevicePointer(&d, p, 0));
    in->mbox_host = p;
    in->mbox_dev = d;
  }
  *host = (Mailbox*)in->mbox_host;
  *dev = (Mailbox*)in->mbox_dev;
  (*host)->status = 1;  // "not written"
  return HICR_OK;
}

static hicr_status finish(Instance* in, Mailbox* mh) {
  HICR_CUDA(in, cudaGetLastError());
  // The kernel posts its status last, behind a system-scope fence, so a
  // posted status means its work is visible. Poll the mapped word; query the
  // stream now and then, so a kernel that failed (status never posted) ends
  // the wait with its error.
  volatile int* st = &mh->status;
  for (uint64_t i = 0;; ++i) {
    if (*st != 1) return *st;
    if ((i & 255) == 255) {
      const cudaError_t e = cudaStreamQuery(in->comm());
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return cuda_fail(in, e, "host channel call");
      if (i > (1u << 20)) std::this_thread::yield();
    }
  }
  // the stream is idle: the status word is final
  if (*st == 1) return HICR_ERR_DEVICE;
  return *st;
}

static hicr_status dev_buffer(Instance* in, size_t bytes, void** out) {
  if (in->chan_buf_cap < bytes) {
    HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
    if (in->chan_buf) cudaFree(in->chan_buf);
    in->chan_buf = nullptr;
    in->chan_buf_cap = 0;
    size_t cap = bytes < 65536 ? 65536 : bytes;
    HICR_CUDA(in, cudaMalloc(&in->chan_buf, cap));
    in->chan_buf_cap = cap;
  }
  *out = in->chan_buf;
  return HICR_OK;
}

static SpscView spsc_view(Channel* c) {
  SpscView v;
  v.ring = c->ring;
  v.st = (SpscState*)c->state;
  v.ts = c->token_size;
  v.cap = c->capacity;
  return v;
}
static MpscView mpsc_view(Channel* c) {
  MpscView v;
  v.ring = c->ring;
  v.st = (MpscState*)c->state;
  v.meta = c->meta;
  v.R = c->ring_bytes;
  v.M = c->max_msgs;
  return v;
}

static NlView nl_view(Channel* c) {
  NlView v;
  v.ring = c->ring;
  v.head = (NlHead*)c->state;
  v.st = (NlState*)((char*)c->state + sizeof(NlHead));
  v.meta = reinterpret_cast<NlMeta*>(c->meta);
  v.R = c->ring_bytes;
  v.M = c->max_msgs;
  v.P = c->n_producers;
  return v;
}

static hicr_status add_channel(hicr_instance_t h, Channel* c, size_t ring_bytes, size_t state_bytes,
                               size_t meta_bytes, hicr_channel_t* out) {
  Instance* in = &h->impl;
  char* p = nullptr;
  const size_t ring_al = (ring_bytes + 255) & ~(size_t)255;
  const size_t st_al = (state_bytes + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(&p, ring_al + st_al + meta_bytes);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    delete c;
    return HICR_ERR_NOMEM;
  }
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(in, e, "cudaMalloc(channel)");
  }
  c->ring = (uint8_t*)p;
  c->state = p + ring_al;
  c->meta = meta_bytes ? (MpscMeta*)(p + ring_al + st_al) : nullptr;
  e = cudaMemsetAsync(p + ring_al, 0, st_al + meta_bytes, in->comm());
  if (e == cudaSuccess) e = cudaStreamSynchronize(in->comm());
  if (e != cudaSuccess) {
    cudaFree(p);
    delete c;
    return cuda_fail(in, e, "channel init");
  }
  hicr_slot_t rs;
  hicr_status st = hicr_slot_register(h, HICR_SPACE_HBM, p, ring_bytes, 0, &rs);
  if (st != HICR_OK) {
    cudaFree(p);
    delete c;
    return st;
  }
  c->ring_slot = rs;
  c->live = true;
  for (size_t i = 0; i < in->channels.size(); ++i) {
    if (!in->channels[i]) {
      in->channels[i] = c;
      *out = (hicr_channel_t)i;
      return HICR_OK;
    }
  }
  in->channels.push_back(c);
  *out = (hicr_channel_t)(in->channels.size() - 1);
  return HICR_OK;
}

void destroy_channels(Instance* in) {
  for (Channel* c : in->channels) {
    if (c) {
      if (c->ring) cudaFree(c->ring);
      delete c;
    }
  }
  in->channels.clear();
  if (in->mbox_host) cudaFreeHost(in->mbox_host);
  in->mbox_host = in->mbox_dev = nullptr;
  if (in->chan_buf) cudaFree(in->chan_buf);
  in->chan_buf = nullptr;
  in->chan_buf_cap = 0;
}

static bool pow2(unsigned long long x) { return x && !(x & (x - 1)); }

}  // namespace hicr

using namespace hicr;

static Instance* I(hicr_instance_t h) { return h ? &h->impl : nullptr; }

extern "C" {

hicr_status hicr_spsc_create(hicr_instance_t h, uint32_t token_size, uint32_t capacity, hicr_channel_t* out) {
  Instance* in = I(h);
  if (!in || !out || token_size == 0 || capacity == 0 || in->capturing) return HICR_ERR_INVALID;
  if ((unsigned long long)token_size * capacity > (1ull << 40)) return HICR_ERR_INVALID;
  Channel* c = new Channel();
  c->kind = 0;
  c->token_size = token_size;
  c->capacity = capacity;
  c->seq.assign(1, 0);
  return add_channel(h, c, (size_t)token_size * capacity, sizeof(SpscState), 0, out);
}

hicr_status hicr_mpsc_create(hicr_instance_t h, uint32_t n_producers, uint64_t ring_bytes, uint32_t max_msgs,
                             hicr_channel_t* out) {
  Instance* in = I(h);
  if (!in || !out || n_producers == 0 || in->capturing) return HICR_ERR_INVALID;
  if (!pow2(ring_bytes) || ring_bytes < 64 || ring_bytes > (1ull << 39)) return HICR_ERR_INVALID;
  if (!pow2(max_msgs) || max_msgs > (1u << 23)) return HICR_ERR_INVALID;
  Channel* c = new Channel();
  c->kind = 1;
  c->n_producers = n_producers;
  c->ring_bytes = ring_bytes;
  c->max_msgs = max_msgs;
  c->seq.assign(n_producers, 0);
  return add_channel(h, c, ring_bytes, sizeof(MpscState), sizeof(MpscMeta) * (size_t)max_msgs, out);
}

hicr_status hicr_mpsc_nl_create(hicr_instance_t h, uint32_t n_producers, uint64_t ring_bytes, uint32_t max_msgs,
                                hicr_channel_t* out) {
  Instance* in = I(h);
  if (!in || !out || n_producers == 0 || in->capturing) return HICR_ERR_INVALID;
  if (!pow2(ring_bytes) || ring_bytes < 64 || ring_bytes > (1ull << 39)) return HICR_ERR_INVALID;
  if (!pow2(max_msgs) || max_msgs > (1u << 23)) return HICR_ERR_INVALID;
  if ((unsigned long long)n_producers * ring_bytes > (1ull << 40)) return HICR_ERR_INVALID;
  Channel* c = new Channel();
  c->kind = 2;
  c->n_producers = n_producers;
  c->ring_bytes = ring_bytes;
  c->max_msgs = max_msgs;
  c->seq.assign(n_producers, 0);
  return add_channel(h, c, (size_t)n_producers * ring_bytes, sizeof(NlHead) + sizeof(NlState) * (size_t)n_producers,
                     sizeof(NlMeta) * (size_t)max_msgs * n_producers, out);
}

hicr_status hicr_channel_device_view(hicr_instance_t h, hicr_channel_t ch, hicr_channel_view_t* out) {
  Instance* in = I(h);
  if (!in || !out) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  hicr_channel_view_t v;
  memset(&v, 0, sizeof(v));
  v.kind = (uint32_t)c->kind;
  v.ring = c->ring;
  if (c->kind == 0) {
    SpscState* st = (SpscState*)c->state;
    v.token_size = c->token_size;
    v.capacity = c->capacity;
    v.ring_bytes = (uint64_t)c->token_size * c->capacity;
    v.head = &st->head.v;
    v.tail = &st->tail.v;
  } else if (c->kind == 1) {
    MpscState* st = (MpscState*)c->state;
    v.max_msgs = c->max_msgs;
    v.ring_bytes = c->ring_bytes;
    v.head = &st->reserve.v;
    v.tail = &st->msg_tail.v;
    v.freed = &st->freed.v;
    v.meta = c->meta;
  } else {
    const NlView nv = nl_view(c);
    v.capacity = nv.P;
    v.max_msgs = nv.M;
    v.ring_bytes = nv.R;
    v.head = &nv.st->reserve.v;
    v.meta = nv.meta;
  }
  *out = v;
  return HICR_OK;
}

hicr_status hicr_channel_destroy(hicr_instance_t h, hicr_channel_t ch) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  hicr_slot_deregister(h, c->ring_slot);
  cudaFree(c->ring);
  delete c;
  in->channels[ch] = nullptr;
  return HICR_OK;
}

hicr_status hicr_channel_ring(hicr_instance_t h, hicr_channel_t ch, hicr_slot_t* ring_slot) {
  Instance* in = I(h);
  if (!in || !ring_slot) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  *ring_slot = c->ring_slot;
  return HICR_OK;
}

hicr_status hicr_channel_push(hicr_instance_t h, hicr_channel_t ch, uint32_t producer, hicr_slot_t src,
                              uint64_t off, uint64_t n) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  void* sp = nullptr;
  uint64_t ssize = 0;
  uint32_t sspace = 0;
  if (hicr_slot_info(h, src, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  Mailbox *mh, *md;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  if ((st = mailbox(in, &mh, &md)) != HICR_OK) return st;
  if (c->kind == 0) {
    if (producer != 0) return HICR_ERR_INVALID;
    if (n > (1ull << 40) / c->token_size) return HICR_ERR_FULL;
    const uint64_t bytes = n * c->token_size;
    if (off > ssize || bytes > ssize - off) return HICR_ERR_BOUNDS;
    if (n > c->capacity) return HICR_ERR_FULL;
    k_spsc_push_host<<<1, 256, 0, in->comm()>>>(spsc_view(c), (const uint8_t*)sp + off, n, md);
    st = finish(in, mh);
  } else {
    if (producer >= c->n_producers) return HICR_ERR_INVALID;
    if (off > ssize || n > ssize - off) return HICR_ERR_BOUNDS;
    if (round16(n) > c->ring_bytes || n > 0xffffffffull) return HICR_ERR_TOO_LARGE;
    if (c->kind == 1)
      k_mpsc_push_host<<<1, 256, 0, in->comm()>>>(mpsc_view(c), producer, c->seq[producer],
                                                 (const uint8_t*)sp + off, n, md);
    else
      k_nl_push_host<<<1, 256, 0, in->comm()>>>(nl_view(c), producer, c->seq[producer], (const uint8_t*)sp + off, n,
                                               md);
    st = finish(in, mh);
    if (st == HICR_OK) c->seq[producer]++;
  }
  if (st == HICR_OK) st = record_done(in);
  return st;
}

static hicr_status ctl(Instance* in, Channel* c, int op, uint64_t k, Mailbox** out) {
  Mailbox *mh, *md;
  hicr_status st = mailbox(in, &mh, &md);
  if (st != HICR_OK) return st;
  if (c->kind == 0) k_spsc_ctl<<<1, 1, 0, in->comm()>>>(spsc_view(c), op, k, md);
  else if (c->kind == 1) k_mpsc_ctl<<<1, 1, 0, in->comm()>>>(mpsc_view(c), op, k, md);
  else k_nl_ctl<<<1, 1, 0, in->comm()>>>(nl_view(c), op, k, md);
  st = finish(in, mh);
  *out = mh;
  return st;
}

hicr_status hicr_channel_peek(hicr_instance_t h, hicr_channel_t ch, uint64_t k, hicr_msg_info_t* out) {
  Instance* in = I(h);
  if (!in || !out || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  Mailbox* mb = nullptr;
  hicr_status st = ctl(in, c, 0, k, &mb);
  if (st != HICR_OK) return st;
  out->offset = mb->v[0];
  out->size = mb->v[1];
  out->producer = (uint32_t)mb->v[2];
  out->reserved = 0;
  out->seq = mb->v[3];
  return HICR_OK;
}

hicr_status hicr_channel_pop(hicr_instance_t h, hicr_channel_t ch, uint64_t count) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  Mailbox* mb = nullptr;
  return ctl(in, c, 1, count, &mb);
}

hicr_status hicr_channel_depth(hicr_instance_t h, hicr_channel_t ch, uint64_t* msgs, uint64_t* bytes) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  Mailbox* mb = nullptr;
  hicr_status st = ctl(in, c, 2, 0, &mb);
  if (st != HICR_OK) return st;
  if (msgs) *msgs = mb->v[0];
  if (bytes) *bytes = mb->v[1];
  return HICR_OK;
}

hicr_status hicr_spsc_stream(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n, uint64_t tokens,
                             uint32_t batch, uint64_t timeout_ns, hicr_spsc_result_t* results) {
  hicr::NvtxRange nvtx_range("hicr_spsc_stream");
  Instance* in = I(h);
  if (!in || !chans || !results || n == 0 || batch == 0 || in->capturing) return HICR_ERR_INVALID;
  std::vector<SpscView> views(n);
  for (uint32_t i = 0; i < n; ++i) {
    Channel* c = get(in, chans[i]);
    if (!c || c->kind != 0 || c->token_size % 16 || batch > c->capacity) return HICR_ERR_INVALID;
    views[i] = spsc_view(c);
  }
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  const size_t vb = ((sizeof(SpscView) * n + 255) / 256) * 256;
  const size_t rb = sizeof(hicr_spsc_result_t) * n;
  void* buf = nullptr;
  if ((st = dev_buffer(in, vb + rb + 256, &buf)) != HICR_OK) return st;
  char* p = (char*)buf;
  cudaStream_t s = in->comm();
  HICR_CUDA(in, cudaMemcpyAsync(p, views.data(), sizeof(SpscView) * n, cudaMemcpyHostToDevice, s));
  HICR_CUDA(in, cudaMemsetAsync(p + vb, 0, rb + 256, s));
  SpscStreamArgs a;
  a.chans = (const SpscView*)p;
  a.n = n;
  a.batch = batch;
  a.tokens = tokens;
  a.timeout_ns = timeout_ns;
  a.res = (hicr_spsc_result_t*)(p + vb);
  a.abort = (unsigned int*)(p + vb + rb);
  void* args[] = {&a};
  HICR_CUDA(in, cudaLaunchCooperativeKernel((const void*)k_spsc_stream, dim3(2 * n), dim3(512), args, 0, s));
  HICR_CUDA(in, cudaMemcpyAsync(results, a.res, rb, cudaMemcpyDeviceToHost, s));
  HICR_CUDA(in, cudaStreamSynchronize(s));
  if ((st = record_done(in)) != HICR_OK) return st;
  for (uint32_t i = 0; i < n; ++i)
    if (results[i].status != HICR_OK) return HICR_ERR_TIMEOUT;
  return HICR_OK;
}

// Grid of a streaming launch: the consumer CTAs first, then the producer
// CTAs (one warp per producer), spread over every CTA slot the consumers leave
// free, so that each SM's memory pipeline serves fewer producer warps. Sets
// *pw to the producer warps per producer CTA; returns 0 when the producers do
// not fit even at `warps` per CTA.
static unsigned long long stream_grid(unsigned long long cons_ctas, unsigned long long n_prod, unsigned warps,
                                      unsigned long long slots, unsigned* pw) {
  const unsigned long long need = (n_prod + warps - 1) / warps;
  if (cons_ctas + need > slots) return 0;
  if (n_prod == 0) {
    *pw = 1;
    return cons_ctas;
  }
  unsigned long long pc = slots - cons_ctas;
  if (pc > n_prod) pc = n_prod;
  *pw = (unsigned)((n_prod + pc - 1) / pc);
  return cons_ctas + (n_prod + *pw - 1) / *pw;
}

hicr_status hicr_mpsc_stream(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                             uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                             const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                             uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                             uint64_t log_stride, hicr_mpsc_result_t* results) {
  hicr::NvtxRange nvtx_range("hicr_mpsc_stream");
  Instance* in = I(h);
  if (!in || !chans || !results || !d_sizes || !d_src_off || !d_log || n_consumers == 0 || n_producers == 0 ||
      group == 0 || group > (uint32_t)MPSC_MAX_GROUP || consumer_ctas == 0 || in->capturing)
    return HICR_ERR_INVALID;
  void* sp = nullptr;
  uint64_t ssize = 0;
  uint32_t sspace = 0;
  if (hicr_slot_info(h, staging, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  std::vector<MpscView> views(n_consumers);
  const uint64_t per = (n_producers + n_consumers - 1) / n_consumers;
  for (uint32_t i = 0; i < n_consumers; ++i) {
    Channel* c = get(in, chans[i]);
    if (!c || c->kind != 1 || c->n_producers < per) return HICR_ERR_INVALID;
    views[i] = mpsc_view(c);
  }
  if (log_stride < per * msgs_per_producer) return HICR_ERR_INVALID;
  const unsigned warps = MPSC_THREADS / 32;
  int per_sm = 0;
  HICR_CUDA(in, cudaFuncSetAttribute((const void*)k_mpsc_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PROD_SMEM));
  HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mpsc_stream, MPSC_THREADS, PROD_SMEM));
  unsigned pw = 0;
  const unsigned long long grid = stream_grid(n_consumers * (unsigned long long)consumer_ctas, n_producers, warps,
                                              (unsigned long long)per_sm * in->sm_count, &pw);
  if (!grid) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  const size_t vb = ((sizeof(MpscView) * n_consumers + 255) / 256) * 256;
  const size_t rb = ((sizeof(hicr_mpsc_result_t) * n_consumers + 255) / 256) * 256;
  const size_t cb = 128 * (size_t)n_consumers;  // claim counters, one 128-byte line each
  const size_t bb = ((8 * (size_t)n_consumers + 255) / 256) * 256;
  void* buf = nullptr;
  if ((st = dev_buffer(in, vb + rb + 256 + cb + bb, &buf)) != HICR_OK) return st;
  char* p = (char*)buf;
  cudaStream_t s = in->comm();
  HICR_CUDA(in, cudaMemcpyAsync(p, views.data(), sizeof(MpscView) * n_consumers, cudaMemcpyHostToDevice, s));
  HICR_CUDA(in, cudaMemsetAsync(p + vb, 0, rb + 256, s));
  unsigned long long* claim = (unsigned long long*)(p + vb + rb + 256);
  unsigned long long* base = (unsigned long long*)(p + vb + rb + 256 + cb);
  // the run starts at each channel's msg_tail (the channels are empty)
  k_mpsc_stream_prep<<<1, 256, 0, s>>>((const MpscView*)p, n_consumers, claim, base);
  MpscStreamArgs a;
  a.chans = (const MpscView*)p;
  a.n_cons = n_consumers;
  a.n_prod = n_producers;
  a.mpp = msgs_per_producer;
  a.group = group;
  a.sizes = (const unsigned long long*)d_sizes;
  a.src_off = (const unsigned long long*)d_src_off;
  a.staging = (const uint8_t*)sp;
  a.timeout_ns = timeout_ns;
  a.log = d_log;
  a.log_stride = log_stride;
  a.res = (hicr_mpsc_result_t*)(p + vb);
  a.abort = (unsigned int*)(p + vb + rb);
  a.G = consumer_ctas;
  a.claim = claim;
  a.base = base;
  a.pw = pw;
  int* bad = (int*)(p + vb + rb + 128);
  a.bad = bad;
  // the check's verdict stays on the device: a rejected run's CTAs leave at
  // once, and the host reads the verdict with the results
  k_mpsc_check<<<in->sm_count * 4, 256, 0, s>>>(a, ssize, bad);
  void* args[] = {&a};
  HICR_CUDA(in, cudaLaunchCooperativeKernel((const void*)k_mpsc_stream, dim3((unsigned)grid), dim3(MPSC_THREADS),
                                            args, PROD_SMEM, s));
  k_mpsc_stream_marks<<<1, 256, 0, s>>>((const MpscView*)p, n_consumers, a.res);
  std::vector<hicr_mpsc_result_t> hres(n_consumers);
  int hbad = 0;
  HICR_CUDA(in, cudaMemcpyAsync(hres.data(), a.res, sizeof(hicr_mpsc_result_t) * n_consumers,
                                cudaMemcpyDeviceToHost, s));
  HICR_CUDA(in, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  HICR_CUDA(in, cudaStreamSynchronize(s));
  if (hbad) return hbad;
  memcpy(results, hres.data(), sizeof(hicr_mpsc_result_t) * n_consumers);
  if ((st = record_done(in)) != HICR_OK) return st;
  for (uint32_t i = 0; i < n_consumers; ++i)
    if (results[i].status != HICR_OK) return HICR_ERR_TIMEOUT;
  return HICR_OK;
}

hicr_status hicr_mpsc_nl_stream(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                                uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                uint64_t log_stride, hicr_mpsc_result_t* results) {
  hicr::NvtxRange nvtx_range("hicr_mpsc_nl_stream");
  Instance* in = I(h);
  if (!in || !chans || !results || !d_sizes || !d_src_off || !d_log || n_consumers == 0 || n_producers == 0 ||
      group == 0 || group > (uint32_t)MPSC_MAX_GROUP || consumer_ctas == 0 || in->capturing)
    return HICR_ERR_INVALID;
  void* sp = nullptr;
  uint64_t ssize = 0;
  uint32_t sspace = 0;
  if (hicr_slot_info(h, staging, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  const unsigned warps = MPSC_THREADS / 32;
  const uint64_t per = (n_producers + n_consumers - 1) / n_consumers;
  // every consumer warp polls at most 32 rings (one per lane)
  if (per > 32ull * warps * consumer_ctas) return HICR_ERR_INVALID;
  std::vector<NlView> views(n_consumers);
  for (uint32_t i = 0; i < n_consumers; ++i) {
    Channel* c = get(in, chans[i]);
    if (!c || c->kind != 2 || c->n_producers < per) return HICR_ERR_INVALID;
    views[i] = nl_view(c);
  }
  if (log_stride < per * msgs_per_producer) return HICR_ERR_INVALID;
  int per_sm = 0;
  HICR_CUDA(in, cudaFuncSetAttribute((const void*)k_nl_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PROD_SMEM));
  HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nl_stream, MPSC_THREADS, PROD_SMEM));
  unsigned pw = 0;
  const unsigned long long grid = stream_grid(n_consumers * (unsigned long long)consumer_ctas, n_producers, warps,
                                              (unsigned long long)per_sm * in->sm_count, &pw);
  if (!grid) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  const size_t vb = ((sizeof(NlView) * n_consumers + 255) / 256) * 256;
  const size_t rb = ((sizeof(hicr_mpsc_result_t) * n_consumers + 255) / 256) * 256;
  const size_t cb = ((sizeof(unsigned long long) * n_consumers + 255) / 256) * 256;
  void* buf = nullptr;
  if ((st = dev_buffer(in, vb + rb + cb + 256, &buf)) != HICR_OK) return st;
  char* p = (char*)buf;
  cudaStream_t s = in->comm();
  HICR_CUDA(in, cudaMemcpyAsync(p, views.data(), sizeof(NlView) * n_consumers, cudaMemcpyHostToDevice, s));
  HICR_CUDA(in, cudaMemsetAsync(p + vb, 0, rb + cb + 256, s));
  NlStreamArgs a;
  a.chans = (const NlView*)p;
  a.n_cons = n_consumers;
  a.G = consumer_ctas;
  a.n_prod = n_producers;
  a.mpp = msgs_per_producer;
  a.group = group;
  a.sizes = (const unsigned long long*)d_sizes;
  a.src_off = (const unsigned long long*)d_src_off;
  a.staging = (const uint8_t*)sp;
  a.timeout_ns = timeout_ns;
  a.log = d_log;
  a.log_stride = log_stride;
  a.res = (hicr_mpsc_result_t*)(p + vb);
  a.log_count = (unsigned long long*)(p + vb + rb);
  a.abort = (unsigned int*)(p + vb + rb + cb);
  a.pw = pw;
  int* bad = (int*)(p + vb + rb + cb + 128);
  a.bad = bad;
  // the check's verdict stays on the device (see hicr_mpsc_stream)
  k_nl_stream_prep<<<1, 256, 0, s>>>((const NlView*)p, n_consumers);
  k_nl_check<<<in->sm_count * 4, 256, 0, s>>>(a, ssize, bad);
  void* args[] = {&a};
  HICR_CUDA(in, cudaLaunchCooperativeKernel((const void*)k_nl_stream, dim3((unsigned)grid), dim3(MPSC_THREADS), args,
                                            PROD_SMEM, s));
  k_nl_stream_marks<<<1, 256, 0, s>>>((const NlView*)p, n_consumers, a.res);
  std::vector<hicr_mpsc_result_t> hres(n_consumers);
  int hbad = 0;
  HICR_CUDA(in, cudaMemcpyAsync(hres.data(), a.res, sizeof(hicr_mpsc_result_t) * n_consumers,
                                cudaMemcpyDeviceToHost, s));
  HICR_CUDA(in, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  HICR_CUDA(in, cudaStreamSynchronize(s));
  if (hbad) return hbad;
  memcpy(results, hres.data(), sizeof(hicr_mpsc_result_t) * n_consumers);
  if ((st = record_done(in)) != HICR_OK) return st;
  for (uint32_t i = 0; i < n_consumers; ++i)
    if (results[i].status != HICR_OK) return HICR_ERR_TIMEOUT;
  return HICR_OK;
}

hicr_status hicr_pingpong(hicr_instance_t h, hicr_slot_t src, uint64_t src_off, uint64_t bytes, uint32_t reps,
                          uint32_t warmup, uint32_t ctas_per_side, uint64_t timeout_ns, hicr_pingpong_result_t* out) {
  Instance* in = I(h);
  if (!in || !out || reps == 0 || ctas_per_side == 0 || ctas_per_side > 256 || bytes == 0 || in->capturing)
    return HICR_ERR_INVALID;
  int per_sm = 0;
  HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pingpong, 512, 0));
  if (2ull * ctas_per_side > (unsigned long long)per_sm * in->sm_count) return HICR_ERR_INVALID;
  void* sp = nullptr;
  uint64_t ssize = 0;
  uint32_t sspace = 0;
  if (hicr_slot_info(h, src, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  if (src_off > ssize || bytes > ssize - src_off) return HICR_ERR_BOUNDS;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  // the two single-message buffers (one allocation, freed at the end)
  uint8_t* bufs = nullptr;
  const uint64_t half = (bytes + 255) & ~255ull;
  cudaError_t e = cudaMalloc(&bufs, 2 * half);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    return HICR_ERR_NOMEM;
  }
  HICR_CUDA(in, e);
  void* buf = nullptr;
  st = dev_buffer(in, 65536, &buf);
  if (st != HICR_OK) {
    cudaFree(bufs);
    return st;
  }
  cudaStream_t cs = in->comm();
  unsigned long long* arrive = (unsigned long long*)buf;  // [0], [16]
  unsigned long long* times = arrive + 32;
  unsigned int* abort_flag = (unsigned int*)(times + 4);
  e = cudaMemsetAsync(buf, 0, 512, cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(bufs, 0, 2 * half, cs);
  PingArgs a;
  a.msg = (const uint8_t*)sp + src_off;
  a.buf_a = bufs;
  a.buf_b = bufs + half;
  a.bytes = bytes;
  a.G = ctas_per_side;
  a.rounds = reps + warmup;
  a.warmup = warmup;
  a.timeout_ns = timeout_ns;
  a.arrive = arrive;
  a.times = times;
  a.abort = abort_flag;
  void* args[] = {&a};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)k_pingpong, dim3(2 * ctas_per_side), dim3(512), args, 0, cs);
  unsigned long long ht[2] = {0, 0};
  unsigned int hab = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(ht, times, 16, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hab, abort_flag, 4, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) {
    cudaFree(bufs);
    return cuda_fail(in, e, "pingpong");
  }
  // digests of both buffers with the library's digest kernel
  hicr_pingpong_result_t r;
  memset(&r, 0, sizeof(r));
  r.bytes = bytes;
  r.reps = reps;
  r.ctas_per_side = ctas_per_side;
  r.status = hab ? HICR_ERR_TIMEOUT : HICR_OK;
  const double dt = (double)(ht[1] - ht[0]);
  r.half_rtt_ns = hab ? 0.0 : dt / (2.0 * reps);
  r.goodput_gbs = r.half_rtt_ns > 0 ? (double)bytes / r.half_rtt_ns : 0.0;
  hicr_slot_t sa = 0, sb = 0;
  st = hicr_slot_register(h, HICR_SPACE_HBM, bufs, bytes, 0, &sa);
  if (st == HICR_OK) st = hicr_slot_register(h, HICR_SPACE_HBM, bufs + half, bytes, 0, &sb);
  if (st == HICR_OK) st = hicr_util_digest(h, sa, 0, bytes, &r.digest_a);
  if (st == HICR_OK) st = hicr_util_digest(h, sb, 0, bytes, &r.digest_b);
  cudaStreamSynchronize(cs);
  hicr_slot_deregister(h, sa);
  hicr_slot_deregister(h, sb);
  cudaFree(bufs);
  if (st != HICR_OK) return st;
  *out = r;
  return r.status;
}

}  // extern "C"
