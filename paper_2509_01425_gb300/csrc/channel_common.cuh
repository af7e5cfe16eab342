// Device-side layout and synchronisation primitives of the channels, shared
// by the channel kernels and the serving engine.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include "../../include/hicr_channels.h"
#include "copy.cuh"
#include "tma.cuh"

namespace hicr {

static constexpr unsigned long long MASK40 = (1ull << 40) - 1;
static constexpr unsigned long long MASK24 = (1ull << 24) - 1;
static constexpr unsigned FULLM = 0xffffffffu;

struct alignas(128) Line {
  unsigned long long v;
  unsigned long long pad[15];
};
struct SpscState {
  Line head;
  Line tail;
};
struct MpscState {
  Line reserve;
  Line freed;
  Line msg_tail;
  Line max_bytes;
  Line max_msgs;
};
struct MpscMeta {
  unsigned long long start;
  unsigned int size;
  unsigned int producer;
  unsigned int seq;
  unsigned int flags;
  unsigned long long ready;
};
static_assert(sizeof(MpscMeta) == 32, "metadata entry is 32 bytes");

struct Mailbox {
  int status;
  unsigned int pad;
  unsigned long long v[6];
};

// A host-call kernel's last act: everything it wrote before (results in v[],
// ring bytes, counters) becomes visible system-wide, then the status word,
// which the host polls in mapped memory.
__device__ __forceinline__ void mb_post(Mailbox* mb, int st) {
  __threadfence_system();
  *(volatile int*)&mb->status = st;
}


// ---------------------------------------------------------------------------
// Device primitives.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acq(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_rlx(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_add_rel(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool aborted(const unsigned int* abort) {
  return *(volatile const unsigned int*)abort != 0u;
}
__host__ __device__ __forceinline__ unsigned long long round16(unsigned long long n) { return (n + 15) & ~15ull; }

// Capture mode of the streaming consumers: copy n bytes of a consumed message
// from the ring (written by producers on other SMs, so read at L2) to the
// caller's capture buffer, with the whole warp.
__device__ __forceinline__ void capture_copy(uint8_t* __restrict__ d, const uint8_t* __restrict__ s,
                                             unsigned long long n, unsigned lane) {
  unsigned long long q0 = 0;
  if ((((uintptr_t)d | (uintptr_t)s) & 15u) == 0) {
    const unsigned long long nv = n / 16;
    for (unsigned long long q = lane; q < nv; q += 32)
      reinterpret_cast<uint4*>(d)[q] = __ldcg(reinterpret_cast<const uint4*>(s) + q);
    q0 = nv * 16;
  }
  for (unsigned long long q = q0 + lane; q < n; q += 32) d[q] = __ldcg(s + q);
}

// Register-staged producer copy into a channel ring (the serving engine's
// burst producers; the streaming kernels use group_copy_bulk below): when
// source and destination are both 16-byte aligned, every lane keeps 16 vector
// loads in flight (8 KiB per warp) and the ring is written with
// default-cached stores, so that the consumer, which reads the message soon
// after, can find it in L2. Other alignments use the general warp copy.
__device__ __forceinline__ void ring_copy(uint8_t* __restrict__ d, const uint8_t* __restrict__ s,
                                          unsigned long long n, unsigned lane) {
  if ((((uintptr_t)d | (uintptr_t)s) & 15u) != 0) {
    warp_copy(d, s, n, lane);
    return;
  }
  const unsigned long long nv = n / 16;
  const uint4* sv = reinterpret_cast<const uint4*>(s);
  uint4* dv = reinterpret_cast<uint4*>(d);
  unsigned long long q0 = 0;
  for (; q0 + 512 <= nv; q0 += 512) {
    uint4 x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = __ldcs(sv + q0 + lane + 32 * u);
#pragma unroll
    for (int u = 0; u < 16; ++u) dv[q0 + lane + 32 * u] = x[u];
  }
  for (unsigned long long q = q0 + lane; q < nv; q += 32) dv[q] = __ldcs(sv + q);
  const unsigned long long tb = nv * 16;
  if (tb + lane < n) d[tb + lane] = s[tb + lane];
}

// Producer copy of a group of k (1 .. 32) messages into their ring slots
// through the warp's NST shared-memory stages of STG bytes each (with one
// mbarrier per stage). Lane j < k holds message j: destination d, source s, n
// bytes. The 16-byte-aligned bodies of the messages whose source and
// destination are both 16-byte aligned form one byte sequence that moves by
// bulk copies: it is cut into stage fills of up to STG bytes, so that one fill
// can carry several small messages (one bulk load each, all completing on the
// stage's mbarrier), and every fill, once landed, leaves by one bulk store per
// message part. NST fills are in flight at a time; a stage is refilled only
// after the store that read it has finished reading. Sub-16-byte tails, and
// whole messages with other alignments, use plain warp copies. Lane 0 issues
// every bulk operation; control flow is warp-uniform. `phase` holds one parity
// bit per stage (the same in all lanes). On return the bulk stores have
// completed and are ordered before the caller's later generic-proxy release.
// Returns false if an mbarrier wait gave up after wait_ns; bulk copies still in
// flight are drained first, each wait again bounded.
template <unsigned NST, unsigned STG>
__device__ bool group_copy_bulk(uint8_t* d, const uint8_t* s, unsigned long long n, int k, unsigned lane,
                                uint8_t* stage, unsigned long long* bars, unsigned& phase,
                                unsigned long long wait_ns) {
  const unsigned FM = 0xffffffffu;
  const bool al =
      lane < (unsigned)k && ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(s)) & 15u) == 0;
  const unsigned long long B = al ? (n & ~15ull) : 0ull;
  const unsigned long long du = reinterpret_cast<uintptr_t>(d), su = reinterpret_cast<uintptr_t>(s);
  // the ring bytes were last read by the consumer (ordinary loads, ordered
  // before this producer's acquire of the freed counter): order those before
  // the bulk stores
  if (lane == 0) fence_proxy_async_global();
  int ci = 0;  // load cursor: message ci, byte co of its body
  unsigned long long co = 0;
  // one stage fill from the cursor; returns its bytes (0: nothing left)
  auto fill = [&](unsigned st) -> unsigned {
    int i = ci;
    unsigned long long o = co;
    unsigned used = 0;
    while (i < k && used < STG) {
      const unsigned long long b = __shfl_sync(FM, B, i);
      if (o >= b) {
        ++i;
        o = 0;
        continue;
      }
      const unsigned long long len = min(b - o, (unsigned long long)(STG - used));
      used += (unsigned)len;
      o += len;
    }
    if (used) {
      if (lane == 0) mbar_expect_tx(bars + st, used);
      unsigned off = 0;
      while (off < used) {
        const unsigned long long b = __shfl_sync(FM, B, ci);
        const unsigned long long sp = __shfl_sync(FM, su, ci);
        if (co >= b) {
          ++ci;
          co = 0;
          continue;
        }
        const unsigned long long len = min(b - co, (unsigned long long)(used - off));
        if (lane == 0) tma_load(stage + st * STG + off, reinterpret_cast<const uint8_t*>(sp) + co, (unsigned)len, bars + st);
        off += (unsigned)len;
        co += len;
      }
    }
    return used;
  };
  // lane 0 waits (bounded) for stage st's fill; the verdict goes to all lanes
  auto landed = [&](unsigned st) -> bool {
    int okw = 1;
    if (lane == 0) {
      const unsigned par = (phase >> st) & 1u;
      if (!mbar_try_wait(bars + st, par)) {
        const unsigned long long t0 = tma_now_ns();
        while (!mbar_try_wait(bars + st, par)) {
          if (tma_now_ns() - t0 > wait_ns) {
            okw = 0;
            break;
          }
        }
      }
    }
    okw = __shfl_sync(FM, okw, 0);
    if (okw) phase ^= 1u << st;
    return okw != 0;
  };
  int fi[NST];
  unsigned long long fo[NST];
  unsigned fu[NST];
#pragma unroll
  for (unsigned st = 0; st < NST; ++st) {
    fi[st] = ci;
    fo[st] = co;
    fu[st] = fill(st);
  }
  bool ok = true;
  for (;;) {
    bool any = false;
#pragma unroll
    for (unsigned st = 0; st < NST; ++st) {
      if (!ok || fu[st] == 0) continue;
      any = true;
      if (!landed(st)) {
        ok = false;
        fu[st] = 0;
        continue;
      }
      int i = fi[st];
      unsigned long long o = fo[st];
      unsigned off = 0;
      while (off < fu[st]) {
        const unsigned long long b = __shfl_sync(FM, B, i);
        const unsigned long long dp = __shfl_sync(FM, du, i);
        if (o >= b) {
          ++i;
          o = 0;
          continue;
        }
        const unsigned long long len = min(b - o, (unsigned long long)(fu[st] - off));
        if (lane == 0) tma_store(reinterpret_cast<uint8_t*>(dp) + o, stage + st * STG + off, (unsigned)len);
        off += (unsigned)len;
        o += len;
      }
      if (lane == 0) {
        tma_commit();
        tma_wait_read0();  // the stage may be refilled once its store has read it
      }
      __syncwarp();
      fi[st] = ci;
      fo[st] = co;
      fu[st] = fill(st);
    }
    if (!any || !ok) break;
  }
  if (!ok) {
    // drain the fills still in flight before the stages can be given up
#pragma unroll
    for (unsigned st = 0; st < NST; ++st)
      if (fu[st]) landed(st);
  }
  if (lane == 0) {
    tma_wait_all();
    fence_proxy_async_global();
  }
  __syncwarp();
  // tails and unaligned messages
  for (int j = 0; j < k; ++j) {
    const unsigned long long nj = __shfl_sync(FM, n, j), bj = __shfl_sync(FM, B, j);
    const unsigned long long dj = __shfl_sync(FM, du, j), sj = __shfl_sync(FM, su, j);
    const int aj = __shfl_sync(FM, (int)al, j);
    uint8_t* dd = reinterpret_cast<uint8_t*>(dj);
    const uint8_t* ss = reinterpret_cast<const uint8_t*>(sj);
    if (!aj) warp_copy(dd, ss, nj, lane);
    else if (bj + lane < nj) dd[bj + lane] = ss[bj + lane];
  }
  return ok;
}

// One message as warp_digest_bulk sees it: its ring address, its body (size
// rounded up to 16 bytes: what a bulk load may read) and its size.
struct DigestMsg {
  const uint8_t* addr;
  unsigned long long body;
  unsigned long long n;
};

// Word digest, by bulk loads, of a contiguous share of a list of messages: the
// `bytes` bytes (a multiple of 16) of the messages' concatenated bodies that
// start at byte o0 of message j0's body. msg(j) describes message j (ring
// addresses 16-byte aligned); sink(j, d) receives, in every lane, a part of
// message j's digest (sum_i w_i (2i + 1) over the part's 8-byte words, i
// counted from the message's start, bytes past n as zero); a message's parts
// add up to its digest. The share streams through the warp's NST stages of
// STG bytes (one mbarrier each): a stage fill carries up to STG bytes, one bulk
// load per message part, so that several small messages travel in one fill,
// and NST fills are in flight while the warp digests the oldest one from
// shared memory. Lane 0 issues the loads; control flow is warp-uniform and
// `phase` (one parity bit per stage) is the same in all lanes. Returns false
// if a wait gave up after wait_ns (fills in flight are drained first, each
// wait again bounded).
template <unsigned NST, unsigned STG, class Msg, class Sink>
__device__ bool warp_digest_bulk(int j0, unsigned long long o0, unsigned long long bytes, Msg msg, Sink sink,
                                 unsigned lane, uint8_t* stage, unsigned long long* bars, unsigned& phase,
                                 unsigned long long wait_ns) {
  const unsigned FM = 0xffffffffu;
  int ci = j0;  // load cursor: byte co of message ci's body; `left` bytes to go
  unsigned long long co = o0, left = bytes;
  auto fill = [&](unsigned st) -> unsigned {
    const unsigned used = (unsigned)min(left, (unsigned long long)STG);
    if (used) {
      if (lane == 0) {
        // earlier ordinary reads of this stage come before the bulk writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bars + st, used);
      }
      unsigned off = 0;
      while (off < used) {
        const DigestMsg m = msg(ci);
        if (co >= m.body) {
          ++ci;
          co = 0;
          continue;
        }
        const unsigned long long len = min(m.body - co, (unsigned long long)(used - off));
        if (lane == 0) tma_load(stage + st * STG + off, m.addr + co, (unsigned)len, bars + st);
        off += (unsigned)len;
        co += len;
      }
      left -= used;
    }
    return used;
  };
  // every lane waits (bounded) for stage st's fill: a landed fill's bytes are
  // visible to the threads that observe its mbarrier phase complete
  auto landed = [&](unsigned st) -> bool {
    const unsigned par = (phase >> st) & 1u;
    int okw = 1;
    if (!mbar_try_wait(bars + st, par)) {
      const unsigned long long t0 = tma_now_ns();
      while (!mbar_try_wait(bars + st, par)) {
        if (tma_now_ns() - t0 > wait_ns) {
          okw = 0;
          break;
        }
      }
    }
    okw = __all_sync(FM, okw);
    if (okw) phase ^= 1u << st;
    return okw != 0;
  };
  int fi[NST];
  unsigned long long fo[NST];
  unsigned fu[NST];
#pragma unroll
  for (unsigned st = 0; st < NST; ++st) {
    fi[st] = ci;
    fo[st] = co;
    fu[st] = fill(st);
  }
  // the message being digested and this lane's running share of it
  int jc = -1;
  unsigned long long dc = 0;
  bool ok = true;
  for (;;) {
    bool any = false;
#pragma unroll
    for (unsigned st = 0; st < NST; ++st) {
      if (!ok || fu[st] == 0) continue;
      any = true;
      if (!landed(st)) {
        ok = false;
        fu[st] = 0;
        continue;
      }
      int i = fi[st];
      unsigned long long o = fo[st];
      unsigned off = 0;
      while (off < fu[st]) {
        const DigestMsg m = msg(i);
        if (o >= m.body) {
          ++i;
          o = 0;
          continue;
        }
        if (i != jc) {
          if (jc >= 0) {
            for (int x = 16; x > 0; x >>= 1) dc += __shfl_xor_sync(FM, dc, x);
            sink(jc, dc);
          }
          jc = i;
          dc = 0;
        }
        const unsigned len = (unsigned)min(m.body - o, (unsigned long long)(fu[st] - off));
        const unsigned long long q0 = o / 16, nvm = (m.n + 15) / 16;
        const unsigned tail = (unsigned)(m.n - 16 * (nvm - 1));
        const uint4* sv = reinterpret_cast<const uint4*>(stage + st * STG + off);
        for (unsigned v = lane; v < len / 16; v += 32) {
          const uint4 x = sv[v];
          unsigned long long w0 = (unsigned long long)x.x | ((unsigned long long)x.y << 32);
          unsigned long long w1 = (unsigned long long)x.z | ((unsigned long long)x.w << 32);
          const unsigned long long q = q0 + v;
          if (q + 1 == nvm) {
            if (tail < 8) w0 &= ~0ull >> (64 - 8 * tail);
            if (tail <= 8) w1 = 0;
            else if (tail < 16) w1 &= ~0ull >> (128 - 8 * tail);
          }
          dc += (w0 + w1) * (4ull * q + 1ull) + (w1 << 1);
        }
        off += len;
        o += len;
      }
      __syncwarp();  // every lane has read the stage before it is refilled
      fi[st] = ci;
      fo[st] = co;
      fu[st] = fill(st);
    }
    if (!any || !ok) break;
  }
  if (!ok) {
#pragma unroll
    for (unsigned st = 0; st < NST; ++st)
      if (fu[st]) landed(st);
  }
  if (jc >= 0 && ok) {
    for (int x = 16; x > 0; x >>= 1) dc += __shfl_xor_sync(FM, dc, x);
    sink(jc, dc);
  }
  return ok;
}

// Word digest of one piece of a message (the 16-byte vectors
// [q0, q0 + 32 * NU) of a message of n bytes, src = its first vector), this
// lane's share: lane l holds vectors q = q0 + l + 32u, u < NU, and returns
// sum over them of w0 (4q + 1) + w1 (4q + 3), where w0, w1 are the vector's
// two little-endian words and bytes past n count as zero (so the warp sum over
// all pieces is sum_i w_i (2i + 1) over the message's words). All NU loads
// are issued before any arithmetic. The sum is taken in the equivalent form
//   (4 qb + 1) S + 128 U + 2 W1,  qb = q0 + l,
// with S = sum_u (w0 + w1), U = sum_u u (w0 + w1), W1 = sum_u w1 (all mod
// 2^64), which needs one 64-bit product per piece instead of two per vector.
template <int NU>
__device__ __forceinline__ unsigned long long piece_digest(const uint4* __restrict__ src, unsigned long long q0,
                                                           unsigned long long n, unsigned lane) {
  const unsigned long long nv = (n + 15) / 16;
  const unsigned long long left = nv - q0;  // > 0
  const unsigned rem = left < 32ull * NU ? (unsigned)left : 32u * NU;
  const uint4* sp = src + q0 + lane;
  uint4 x[NU];
#pragma unroll
  for (int u = 0; u < NU; ++u)
    if (lane + 32u * u < rem) x[u] = __ldcg(sp + 32 * u);
  // the message's last vector (in this piece only if left <= 32 NU) keeps
  // only the bytes below n
  const unsigned last = left <= 32ull * NU ? rem - 1 : 0xffffffffu;
  const unsigned tail = (unsigned)(n - 16 * (nv - 1));  // 1..16 bytes
  unsigned long long S = 0, U = 0, W1 = 0;
#pragma unroll
  for (int u = NU - 1; u >= 0; --u) {
    if (lane + 32u * u < rem) {
      unsigned long long w0 = (unsigned long long)x[u].x | ((unsigned long long)x[u].y << 32);
      unsigned long long w1 = (unsigned long long)x[u].z | ((unsigned long long)x[u].w << 32);
      if (lane + 32u * u == last) {
        if (tail < 8) w0 &= ~0ull >> (64 - 8 * tail);
        if (tail <= 8) w1 = 0;
        else if (tail < 16) w1 &= ~0ull >> (128 - 8 * tail);
      }
      S += w0 + w1;
      W1 += w1;
    }
    if (u > 0) U += S;  // after the loop: U = sum_u u (w0 + w1)
  }
  return S * (4ull * (q0 + lane) + 1ull) + (U << 7) + (W1 << 1);
}

struct SpscView {
  uint8_t* ring;
  SpscState* st;
  unsigned int ts;
  unsigned int cap;
};
struct MpscView {
  uint8_t* ring;
  MpscState* st;
  MpscMeta* meta;
  unsigned long long R;
  unsigned int M;
};

// One MPSC reservation attempt for k messages whose rounded sizes are r[0..k)
// starting from reserve word W: fills start[] and returns the end position.
__device__ __forceinline__ unsigned long long mpsc_place(unsigned long long W, const unsigned long long* r, int k,
                                                          unsigned long long R, unsigned long long* start) {
  unsigned long long b = W & MASK40;
  for (int i = 0; i < k; ++i) {
    const unsigned long long pos = b & (R - 1);
    if (pos + r[i] > R) b = (b + (R - pos)) & MASK40;
    start[i] = b;
    b = (b + r[i]) & MASK40;
  }
  return b;
}

// Copy n bytes with every warp of the CTA taking an equal share.
__device__ __forceinline__ void cta_copy(uint8_t* d, const uint8_t* s, unsigned long long n) {
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long a = n * w / nw, b = n * (w + 1) / nw;
  if (b > a) warp_copy(d + a, s + a, b - a, lane);
}

// ---------------------------------------------------------------------------
// Non-locking MPSC layout.
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

}  // namespace hicr
