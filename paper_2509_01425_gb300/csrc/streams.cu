// Streaming runs of the channels (HiCR paper Sec. 4.3): SPSC streams (one
// producer and one consumer CTA per channel) and MPSC streams in locking and
// non-locking mode (one warp per producer, 1-5 CTAs per consumer). Producers
// and consumers run as one cooperative grid, so all of them are resident at
// once; every wait is bounded by the run's %globaltimer deadline and raises a
// shared abort flag on expiry. Payloads of the MPSC streams move by bulk
// copies through per-warp shared-memory stages (group_copy_bulk,
// warp_digest_bulk).
#include <stddef.h>
#include <string.h>

#include <vector>

#include "../../include/hicr_channels.h"
#include "channel_host.h"
#include "splitmix.cuh"

namespace hicr {

// ---------------------------------------------------------------------------
// SPSC streaming: CTA 2i produces into channel i, CTA 2i+1 consumes it.
// Template switches:
//   COPY     the producer pushes by copying token s of channel i from the
//            staging area (token s mod src_tokens of the channel's staged
//            tokens), the channel push the paper defines (a memcpy into the
//            consumer's buffer); otherwise it writes the payload rule's words;
//   VERIFY   the consumer compares every word with the payload rule;
//   CAPTURE  the consumer also stores every token it consumed, in order, to
//            the capture area (token s of channel i at cap + i * cap_stride +
//            s * token_size), so that the tokens can be compared one by one.
// The consumer always folds the consumed words into the digest.
// ---------------------------------------------------------------------------
struct SpscStreamArgs {
  const SpscView* chans;
  unsigned int n;
  unsigned int batch;
  unsigned long long tokens;
  unsigned long long timeout_ns;
  hicr_spsc_result_t* res;
  unsigned int* abort;
  const uint8_t* src;              // COPY: channel i's staged tokens at src + i * src_tokens * ts
  unsigned long long src_tokens;
  uint8_t* cap;                    // CAPTURE
  unsigned long long cap_stride;
};

static constexpr int SPSC_U = 8;

__device__ __forceinline__ uint4 words_to_vec(unsigned long long w0, unsigned long long w1) {
  uint4 x;
  x.x = (unsigned)w0;
  x.y = (unsigned)(w0 >> 32);
  x.z = (unsigned)w1;
  x.w = (unsigned)(w1 >> 32);
  return x;
}

// Load one pass of a copying producer: staged tokens q, q + sstep, ... (mod
// W) of the batch positions tl, tl + tpi, ... below k, vector column jv.
// Returns the staged position after the pass.
__device__ __forceinline__ unsigned long long spsc_load_pass(uint4 (&x)[SPSC_U], const uint8_t* src, unsigned ts,
                                                             unsigned jv, unsigned long long q,
                                                             unsigned long long sstep, unsigned long long W,
                                                             unsigned long long tl, unsigned long long tpi,
                                                             unsigned long long k) {
#pragma unroll
  for (int u = 0; u < SPSC_U; ++u) {
    if (tl + (unsigned long long)u * tpi < k) x[u] = __ldcg(reinterpret_cast<const uint4*>(src + q * ts) + jv);
    q += sstep;
    if (q >= W) q -= W;
  }
  return q;
}

template <bool COPY, bool VERIFY, bool CAPTURE>
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
  const uint8_t* src = COPY ? a.src + (unsigned long long)ci * a.src_tokens * v.ts : nullptr;
  uint8_t* cap = CAPTURE ? a.cap + (unsigned long long)ci * a.cap_stride : nullptr;
  const unsigned long long W = COPY ? a.src_tokens : 1;
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
  const unsigned long long sstep = tpi % W;
  unsigned long long cached = base, max_occ = 0, done = 0, mism = 0, dig = 0;
  int stop = 0;
  // A copying producer's staged tokens do not depend on ring room: each
  // batch's first pass is loaded before the previous batch is published and
  // before the room check, so that one L2 round trip per batch overlaps the
  // hand-off. xp holds the pass to store next.
  uint4 xp[SPSC_U];
  if (COPY && producer && fast)
    spsc_load_pass(xp, src, v.ts, jv, tl0 % W, sstep, W, tl0, tpi, min((unsigned long long)a.batch, a.tokens));
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
      // (and staged positions) advance by `step` (`sstep`) without a
      // division per vector
      unsigned long long slot = (base + s0 + tl0) % v.cap;
      // the staged position of this batch's second pass (the first is in xp)
      unsigned long long sp = COPY ? (s0 + tl0 + (unsigned long long)SPSC_U * tpi) % W : 0;
      for (unsigned long long tl = tl0; tl < k; tl += (unsigned long long)SPSC_U * tpi) {
        if (producer) {
          if (COPY) {
#pragma unroll
            for (int u = 0; u < SPSC_U; ++u) {
              if (tl + (unsigned long long)u * tpi < k) *(reinterpret_cast<uint4*>(v.ring + slot * v.ts) + jv) = xp[u];
              slot += step;
              if (slot >= v.cap) slot -= v.cap;
            }
            // then the next pass: of this batch, or the next batch's first
            const unsigned long long tn = tl + (unsigned long long)SPSC_U * tpi;
            if (tn < k) {
              sp = spsc_load_pass(xp, src, v.ts, jv, sp, sstep, W, tn, tpi, k);
            } else if (s0 + k < a.tokens) {
              const unsigned long long k2 = min((unsigned long long)a.batch, a.tokens - s0 - k);
              spsc_load_pass(xp, src, v.ts, jv, (s0 + k + tl0) % W, sstep, W, tl0, tpi, k2);
            }
          } else {
#pragma unroll
            for (int u = 0; u < SPSC_U; ++u) {
              const unsigned long long t_ = tl + (unsigned long long)u * tpi;
              if (t_ < k) {
                const unsigned long long word = (s0 + t_) * wpt + 2ull * jv;
                uint4* p = reinterpret_cast<uint4*>(v.ring + slot * v.ts) + jv;
                *p = words_to_vec(sm64_first_output(key0 + word), sm64_first_output(key0 + word + 1));
              }
              slot += step;
              if (slot >= v.cap) slot -= v.cap;
            }
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
          if (CAPTURE) {
#pragma unroll
            for (int u = 0; u < SPSC_U; ++u) {
              const unsigned long long t_ = tl + (unsigned long long)u * tpi;
              if (t_ < k) *(reinterpret_cast<uint4*>(cap + (s0 + t_) * v.ts) + jv) = x[u];
            }
          }
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
              const unsigned long long w0 = (unsigned long long)x[u].x | ((unsigned long long)x[u].y << 32);
              const unsigned long long w1 = (unsigned long long)x[u].z | ((unsigned long long)x[u].w << 32);
              if (VERIFY) {
                const unsigned long long word = W0 + (unsigned long long)u * tpi * wpt;
                mism += (w0 != sm64_first_output(key0 + word)) + (w1 != sm64_first_output(key0 + word + 1));
              }
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
          if (COPY) *p = __ldcg(reinterpret_cast<const uint4*>(src + (tok % W) * v.ts) + (q % vpt));
          else *p = words_to_vec(sm64_first_output(key0 + word), sm64_first_output(key0 + word + 1));
        } else {
          const uint4 x = __ldcg(p);
          if (CAPTURE) *(reinterpret_cast<uint4*>(cap + tok * v.ts) + (q % vpt)) = x;
          const unsigned long long w0 = (unsigned long long)x.x | ((unsigned long long)x.y << 32);
          const unsigned long long w1 = (unsigned long long)x.z | ((unsigned long long)x.w << 32);
          if (VERIFY) mism += (w0 != sm64_first_output(key0 + word)) + (w1 != sm64_first_output(key0 + word + 1));
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
// MPSC streaming (locking mode): CTAs [0, n_cons * G) consume (G per
// consumer); the rest hold the producers, pw warps each, one producer per
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
  uint8_t* cap;                    // capture mode: message (p, s) is copied to cap + cap_off[p * mpp + s]
  const unsigned long long* cap_off;
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
      // capture mode: warp w copies messages w, w + nwarp, ... of the window
      // out of the ring (they are freed only after the barrier below); an
      // entry naming no message of the run is skipped (the log shows it)
      if (a.cap) {
        for (unsigned j = warp; j < navail; j += nwarp) {
          if (s_prod[j] >= a.n_prod || s_seq[j] >= a.mpp) continue;
          const unsigned long long idx = (unsigned long long)s_prod[j] * a.mpp + s_seq[j];
          capture_copy(a.cap + a.cap_off[idx], v.ring + (s_start[j] & (v.R - 1)),
                       min((unsigned long long)s_size[j], a.sizes[idx]), lane);
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
  uint8_t* cap;     // capture mode, as in MpscStreamArgs
  const unsigned long long* cap_off;
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
      if (a.cap) {  // capture mode: copy the batch's messages out before they are freed
        const unsigned long long p = (unsigned long long)ring * a.n_cons + c;
        for (unsigned j = 0; j < k; ++j) {
          const unsigned long long sj = __shfl_sync(FULLM, e_start, j);
          const unsigned long long nj = __shfl_sync(FULLM, (unsigned long long)e_size, j);
          const unsigned long long qj = __shfl_sync(FULLM, (unsigned long long)e_seq, j);
          if (p >= a.n_prod || qj >= a.mpp) continue;
          const unsigned long long idx = p * a.mpp + qj;
          capture_copy(a.cap + a.cap_off[idx], rb + (sj & (v.R - 1)), min(nj, a.sizes[idx]), lane);
        }
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

}  // namespace hicr

using namespace hicr;

namespace hicr {

// One SPSC streaming run; opts == nullptr is the generate-and-verify form.
static hicr_status spsc_stream_run(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n, uint64_t tokens,
                                   uint32_t batch, const hicr_spsc_stream_opts_t* opts, uint64_t timeout_ns,
                                   hicr_spsc_result_t* results) {
  hicr::NvtxRange nvtx_range("hicr_spsc_stream");
  Instance* in = I(h);
  if (!in || !chans || !results || n == 0 || batch == 0 || in->capturing) return HICR_ERR_INVALID;
  std::vector<SpscView> views(n);
  uint32_t ts = 0;
  for (uint32_t i = 0; i < n; ++i) {
    Channel* c = get(in, chans[i]);
    if (!c || c->kind != 0 || c->token_size % 16 || batch > c->capacity) return HICR_ERR_INVALID;
    if (i > 0 && c->token_size != ts && opts && (opts->src_tokens || opts->d_capture)) return HICR_ERR_INVALID;
    ts = c->token_size;
    views[i] = spsc_view(c);
  }
  if (opts && (opts->flags & ~HICR_SPSC_DIGEST_ONLY)) return HICR_ERR_INVALID;
  const bool copy = opts && opts->src_tokens > 0;
  const bool capture = opts && opts->d_capture != nullptr;
  const bool verify = !copy && !(opts && (opts->flags & HICR_SPSC_DIGEST_ONLY));
  const uint8_t* src = nullptr;
  if (copy) {
    // the staged tokens of all n channels lie inside the source slot, in HBM,
    // 16-byte aligned (the producers load 16-byte vectors)
    void* sp = nullptr;
    uint64_t ssize = 0;
    uint32_t sspace = 0;
    if (hicr_slot_info(h, opts->src, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
    if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
    const unsigned __int128 need = (unsigned __int128)opts->src_tokens * ts * n;
    if (opts->src_off > ssize || need > (unsigned __int128)(ssize - opts->src_off)) return HICR_ERR_BOUNDS;
    src = (const uint8_t*)sp + opts->src_off;
    if ((uintptr_t)src & 15u) return HICR_ERR_INVALID;
  }
  if (capture) {
    if (((uintptr_t)opts->d_capture & 15u) || (opts->capture_stride & 15u) ||
        (unsigned __int128)tokens * ts > (unsigned __int128)opts->capture_stride)
      return HICR_ERR_INVALID;
  }
  const void* k;
  if (copy) k = capture ? (const void*)k_spsc_stream<true, false, true> : (const void*)k_spsc_stream<true, false, false>;
  else if (verify)
    k = capture ? (const void*)k_spsc_stream<false, true, true> : (const void*)k_spsc_stream<false, true, false>;
  else k = capture ? (const void*)k_spsc_stream<false, false, true> : (const void*)k_spsc_stream<false, false, false>;
  // both CTAs of every channel must be resident at once
  int per_sm = 0;
  HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 512, 0));
  if (2ull * n > (unsigned long long)per_sm * in->sm_count) return HICR_ERR_INVALID;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  // a cooperative grid sized for the whole device: a latency-mode server ends first
  if ((st = lat_stop(in)) != HICR_OK) return st;
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
  a.src = src;
  a.src_tokens = copy ? opts->src_tokens : 0;
  a.cap = capture ? (uint8_t*)opts->d_capture : nullptr;
  a.cap_stride = capture ? opts->capture_stride : 0;
  void* args[] = {&a};
  HICR_CUDA(in, cudaLaunchCooperativeKernel(k, dim3(2 * n), dim3(512), args, 0, s));
  HICR_CUDA(in, cudaMemcpyAsync(results, a.res, rb, cudaMemcpyDeviceToHost, s));
  HICR_CUDA(in, cudaStreamSynchronize(s));
  if ((st = record_done(in)) != HICR_OK) return st;
  for (uint32_t i = 0; i < n; ++i)
    if (results[i].status != HICR_OK) return HICR_ERR_TIMEOUT;
  return HICR_OK;
}

}  // namespace hicr

extern "C" {

hicr_status hicr_spsc_stream(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n, uint64_t tokens,
                             uint32_t batch, uint64_t timeout_ns, hicr_spsc_result_t* results) {
  return spsc_stream_run(h, chans, n, tokens, batch, nullptr, timeout_ns, results);
}

hicr_status hicr_spsc_stream_ex(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n, uint64_t tokens,
                                uint32_t batch, const hicr_spsc_stream_opts_t* opts, uint64_t timeout_ns,
                                hicr_spsc_result_t* results) {
  if (!opts) return HICR_ERR_INVALID;
  return spsc_stream_run(h, chans, n, tokens, batch, opts, timeout_ns, results);
}

}  // extern "C"

namespace hicr {

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

static hicr_status mpsc_stream_run(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                                   uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                   const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                   uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                   uint64_t log_stride, hicr_mpsc_result_t* results, void* d_capture,
                                   const uint64_t* d_cap_off) {
  hicr::NvtxRange nvtx_range("hicr_mpsc_stream");
  Instance* in = I(h);
  if (!in || !chans || !results || !d_sizes || !d_src_off || !d_log || n_consumers == 0 || n_producers == 0 ||
      group == 0 || group > (uint32_t)MPSC_MAX_GROUP || consumer_ctas == 0 || in->capturing)
    return HICR_ERR_INVALID;
  if (d_capture && !d_cap_off) return HICR_ERR_INVALID;
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
  // a cooperative grid sized for the whole device: a latency-mode server ends first
  if ((st = lat_stop(in)) != HICR_OK) return st;
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
  a.cap = (uint8_t*)d_capture;
  a.cap_off = (const unsigned long long*)d_cap_off;
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

static hicr_status nl_stream_run(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                                 uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                 const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                 uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                 uint64_t log_stride, hicr_mpsc_result_t* results, void* d_capture,
                                 const uint64_t* d_cap_off) {
  hicr::NvtxRange nvtx_range("hicr_mpsc_nl_stream");
  Instance* in = I(h);
  if (!in || !chans || !results || !d_sizes || !d_src_off || !d_log || n_consumers == 0 || n_producers == 0 ||
      group == 0 || group > (uint32_t)MPSC_MAX_GROUP || consumer_ctas == 0 || in->capturing)
    return HICR_ERR_INVALID;
  if (d_capture && !d_cap_off) return HICR_ERR_INVALID;
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
  // a cooperative grid sized for the whole device: a latency-mode server ends first
  if ((st = lat_stop(in)) != HICR_OK) return st;
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
  a.cap = (uint8_t*)d_capture;
  a.cap_off = (const unsigned long long*)d_cap_off;
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

}  // namespace hicr

extern "C" {

hicr_status hicr_mpsc_stream(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                             uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                             const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                             uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                             uint64_t log_stride, hicr_mpsc_result_t* results) {
  return mpsc_stream_run(h, chans, n_consumers, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                         consumer_ctas, timeout_ns, d_log, log_stride, results, nullptr, nullptr);
}

hicr_status hicr_mpsc_stream_capture(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                                     uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                     const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                     uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                     uint64_t log_stride, hicr_mpsc_result_t* results, void* d_capture,
                                     const uint64_t* d_cap_off) {
  if (!d_capture) return HICR_ERR_INVALID;
  return mpsc_stream_run(h, chans, n_consumers, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                         consumer_ctas, timeout_ns, d_log, log_stride, results, d_capture, d_cap_off);
}

hicr_status hicr_mpsc_nl_stream(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                                uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                uint64_t log_stride, hicr_mpsc_result_t* results) {
  return nl_stream_run(h, chans, n_consumers, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                       consumer_ctas, timeout_ns, d_log, log_stride, results, nullptr, nullptr);
}

hicr_status hicr_mpsc_nl_stream_capture(hicr_instance_t h, const hicr_channel_t* chans, uint32_t n_consumers,
                                        uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                        const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                        uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                        uint64_t log_stride, hicr_mpsc_result_t* results, void* d_capture,
                                        const uint64_t* d_cap_off) {
  if (!d_capture) return HICR_ERR_INVALID;
  return nl_stream_run(h, chans, n_consumers, n_producers, msgs_per_producer, d_sizes, d_src_off, staging, group,
                       consumer_ctas, timeout_ns, d_log, log_stride, results, d_capture, d_cap_off);
}

}  // extern "C"
