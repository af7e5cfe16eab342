// Warp-cooperative byte copy shared by the memcpy kernels and the channel
// producers (channel pushes are layered on the same copy).
#pragma once
#include <stdint.h>

namespace hicr {

__device__ __forceinline__ uint4 ld16(const uint4* p) { return __ldcs(p); }
__device__ __forceinline__ void st16(uint4* p, const uint4& v) { __stcs(p, v); }

// Destination is 16-byte aligned, source is k = 4*Q + r/8 bytes past the
// aligned word sa[0] (k in 1..15). Word j of the output is bytes
// [k + 16j, k + 16j + 16) of the aligned source stream, assembled from the
// two aligned words sa[j] and sa[j+1] with funnel shifts. Every aligned
// source word loaded holds at least one byte of the requested range, so the
// loads never leave the 16-byte blocks of the source range.
template <int Q>
__device__ __forceinline__ uint4 shift_pair(const uint4& a, const uint4& b, unsigned r) {
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint4 o;
  o.x = __funnelshift_r(w[Q + 0], w[Q + 1], r);
  o.y = __funnelshift_r(w[Q + 1], w[Q + 2], r);
  o.z = __funnelshift_r(w[Q + 2], w[Q + 3], r);
  o.w = __funnelshift_r(w[Q + 3], w[Q + 4], r);
  return o;
}

template <int Q>
__device__ __forceinline__ void copy_shifted(uint4* __restrict__ dw, const uint4* __restrict__ sa,
                                             unsigned long long nw, unsigned r, unsigned lane) {
  unsigned long long j = lane;
  for (; j + 96 < nw; j += 128) {
    uint4 a0 = ld16(sa + j), b0 = ld16(sa + j + 1);
    uint4 a1 = ld16(sa + j + 32), b1 = ld16(sa + j + 33);
    uint4 a2 = ld16(sa + j + 64), b2 = ld16(sa + j + 65);
    uint4 a3 = ld16(sa + j + 96), b3 = ld16(sa + j + 97);
    st16(dw + j, shift_pair<Q>(a0, b0, r));
    st16(dw + j + 32, shift_pair<Q>(a1, b1, r));
    st16(dw + j + 64, shift_pair<Q>(a2, b2, r));
    st16(dw + j + 96, shift_pair<Q>(a3, b3, r));
  }
  for (; j < nw; j += 32) st16(dw + j, shift_pair<Q>(ld16(sa + j), ld16(sa + j + 1), r));
}

__device__ __forceinline__ void copy_aligned(uint4* __restrict__ dw, const uint4* __restrict__ sw,
                                             unsigned long long nw, unsigned lane) {
  unsigned long long j = lane;
  for (; j + 224 < nw; j += 256) {
    uint4 v0 = ld16(sw + j), v1 = ld16(sw + j + 32), v2 = ld16(sw + j + 64), v3 = ld16(sw + j + 96);
    uint4 v4 = ld16(sw + j + 128), v5 = ld16(sw + j + 160), v6 = ld16(sw + j + 192), v7 = ld16(sw + j + 224);
    st16(dw + j, v0);
    st16(dw + j + 32, v1);
    st16(dw + j + 64, v2);
    st16(dw + j + 96, v3);
    st16(dw + j + 128, v4);
    st16(dw + j + 160, v5);
    st16(dw + j + 192, v6);
    st16(dw + j + 224, v7);
  }
  for (; j < nw; j += 32) st16(dw + j, ld16(sw + j));
}

// Copy n bytes from s to d with all 32 lanes of the warp.
__device__ __forceinline__ void warp_copy(uint8_t* __restrict__ d, const uint8_t* __restrict__ s,
                                          unsigned long long n, unsigned lane) {
  if (n < 64) {
    for (unsigned long long k = lane; k < n; k += 32) d[k] = s[k];
    return;
  }
  const unsigned head = (unsigned)((16u - ((uintptr_t)d & 15u)) & 15u);
  if (lane < head) d[lane] = s[lane];
  d += head;
  s += head;
  n -= head;
  const unsigned long long nw = n >> 4;
  const unsigned tail = (unsigned)(n & 15u);
  uint4* dw = reinterpret_cast<uint4*>(d);
  const unsigned k = (unsigned)((uintptr_t)s & 15u);
  if (k == 0) {
    copy_aligned(dw, reinterpret_cast<const uint4*>(s), nw, lane);
  } else {
    const uint4* sa = reinterpret_cast<const uint4*>(s - k);
    const unsigned r = (k & 3u) * 8u;
    switch (k >> 2) {
      case 0: copy_shifted<0>(dw, sa, nw, r, lane); break;
      case 1: copy_shifted<1>(dw, sa, nw, r, lane); break;
      case 2: copy_shifted<2>(dw, sa, nw, r, lane); break;
      default: copy_shifted<3>(dw, sa, nw, r, lane); break;
    }
  }
  if (lane < tail) d[nw * 16 + lane] = s[nw * 16 + lane];
}

// Largest i < count with cstart[i] <= key (cstart[0] = 0 <= key), found by
// the whole warp: each round the lanes probe 32 evenly spaced positions.
__device__ __forceinline__ unsigned long long find_op(const unsigned long long* __restrict__ cstart,
                                                      unsigned long long count, unsigned long long key,
                                                      unsigned lane) {
  unsigned long long L = 0, R = count;
  while (R - L > 32) {
    const unsigned long long step = (R - L + 31) / 32;
    const unsigned long long pos = L + lane * step;
    const bool le = pos < R && cstart[pos] <= key;
    const unsigned m = __ballot_sync(0xffffffffu, le);
    const unsigned k = 31u - __clz(m);
    const unsigned long long nL = L + k * step;
    R = min(R, nL + step);
    L = nL;
  }
  const unsigned long long pos = L + lane;
  const bool le = pos < R && cstart[pos] <= key;
  const unsigned m = __ballot_sync(0xffffffffu, le);
  return L + (31u - __clz(m));
}

}  // namespace hicr
