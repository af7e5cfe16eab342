// Device-side layout and synchronisation primitives of the channels, shared
// by the channel kernels and the serving engine.
#pragma once
#include <stdint.h>

#include "copy.cuh"

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

// Producer copy into a channel ring: when source and destination are both
// 16-byte aligned (staged payloads and ring positions always are), every lane
// keeps 16 vector loads in flight (8 KiB per warp) and the ring is written
// with default-cached stores, so that the consumer, which reads the message
// soon after, can find it in L2. Other alignments use the general warp copy.
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

}  // namespace hicr
