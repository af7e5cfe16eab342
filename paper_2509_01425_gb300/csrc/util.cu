// Device fill and digest utilities (no counterpart in the HiCR paper): the
// seeded slot contents of the synthetic workloads and a word digest that lets
// large results be compared without copying them to the host.
#include "channel_common.cuh"
#include "hicr_internal.h"
#include "splitmix.cuh"

namespace hicr {

// Byte i of the slot (i in [off, off+n)) = byte (i mod 8), little endian, of
// first_output(key_base + i/8), written over the words that overlap [a, b) by
// threads t, t + st, ...: whole 8-byte words at once when the base is 8-byte
// aligned, bytes elsewhere.
__device__ __forceinline__ void fill_words(uint8_t* base, unsigned long long a, unsigned long long b,
                                           unsigned long long key_base, unsigned long long t, unsigned long long st) {
  const bool aligned = ((uintptr_t)base & 7u) == 0;
  for (unsigned long long w = (a >> 3) + t; w < ((b + 7) >> 3); w += st) {
    const uint64_t v = sm64_first_output(key_base + w);
    const unsigned long long bw = w << 3;
    if (aligned && bw >= a && bw + 8 <= b) {
      *reinterpret_cast<uint64_t*>(base + bw) = v;
    } else {
      for (int k = 0; k < 8; ++k) {
        const unsigned long long i = bw + k;
        if (i >= a && i < b) base[i] = (uint8_t)(v >> (8 * k));
      }
    }
  }
}

// The fill of [off, off+n). With a 16-byte-aligned base, the 16-byte units
// inside the range are written by one vector store each (words 2u and 2u + 1)
// and two threads write the head and tail bytes around them.
__global__ void k_fill(uint8_t* base, unsigned long long off, unsigned long long n, unsigned long long key_base) {
  const unsigned long long end = off + n;
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long u0 = (off + 15) >> 4, u1 = end >> 4;  // full units inside the range
  if (((uintptr_t)base & 15u) != 0 || u1 <= u0) {
    fill_words(base, off, end, key_base, tid, stride);
    return;
  }
  uint4* vb = reinterpret_cast<uint4*>(base);
  for (unsigned long long u = u0 + tid; u < u1; u += stride) {
    const uint64_t lo = sm64_first_output(key_base + 2 * u), hi = sm64_first_output(key_base + 2 * u + 1);
    vb[u] = make_uint4((unsigned)lo, (unsigned)(lo >> 32), (unsigned)hi, (unsigned)(hi >> 32));
  }
  if (tid == 0) fill_words(base, off, u0 << 4, key_base, 0, 1);
  if (tid == 1) fill_words(base, u1 << 4, end, key_base, 0, 1);
}

// out += sum_j w_j * (2j + 1) over the little-endian words of p[0, n), the
// last word zero-padded (*out must start at zero). With a 16-byte-aligned p,
// threads read 16-byte vectors, four independent loads at a time; vector q
// holds words 2q and 2q + 1, whose terms are (w0 + w1)(4q + 1) + 2 w1. The
// words past the last full vector (at most two) go to thread 0.
__global__ void k_digest(const uint8_t* p, unsigned long long n, unsigned long long* out) {
  const unsigned long long nw = (n + 7) >> 3;
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  auto word = [&](unsigned long long j) -> uint64_t {  // word j, zero-padded past n
    const unsigned long long b = j << 3;
    uint64_t w = 0;
    if ((((uintptr_t)p & 7u) == 0) && b + 8 <= n) {
      w = *reinterpret_cast<const uint64_t*>(p + b);
    } else {
      for (int k = 0; k < 8; ++k)
        if (b + k < n) w |= (uint64_t)p[b + k] << (8 * k);
    }
    return w;
  };
  if (((uintptr_t)p & 15u) == 0) {
    const unsigned long long nv = n >> 4;
    const uint4* pv = reinterpret_cast<const uint4*>(p);
    for (unsigned long long q = tid; q < nv; q += 4 * stride) {
      uint4 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (q + u * stride < nv) x[u] = __ldcs(pv + q + u * stride);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned long long qq = q + u * stride;
        if (qq < nv) {
          const uint64_t w0 = (uint64_t)x[u].x | ((uint64_t)x[u].y << 32);
          const uint64_t w1 = (uint64_t)x[u].z | ((uint64_t)x[u].w << 32);
          acc += (w0 + w1) * (4ull * qq + 1ull) + (w1 << 1);
        }
      }
    }
    if (tid == 0)
      for (unsigned long long j = 2 * nv; j < nw; ++j) acc += word(j) * (2ull * j + 1ull);
  } else {
    for (unsigned long long j = tid; j < nw; j += stride) acc += word(j) * (2ull * j + 1ull);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// One warp per segment {off, n, key_base}: byte j of the segment is byte
// (j mod 8) of first_output(key_base + j/8).
__global__ void k_fill_segments(uint8_t* base, unsigned long long size, const unsigned long long* seg,
                                unsigned long long count) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long i = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += warps) {
    const unsigned long long off = seg[3 * i], n = seg[3 * i + 1], key = seg[3 * i + 2];
    if (off > size || n > size - off) continue;  // outside the slot: skipped
    uint8_t* d = base + off;
    const bool aligned = ((uintptr_t)d & 7u) == 0;
    const unsigned long long nw = (n + 7) >> 3;
    for (unsigned long long w = lane; w < nw; w += 32) {
      const uint64_t v = sm64_first_output(key + w);
      if (aligned && 8 * w + 8 <= n) {
        *reinterpret_cast<uint64_t*>(d + 8 * w) = v;
      } else {
        for (unsigned k = 0; k < 8 && 8 * w + k < n; ++k) d[8 * w + k] = (uint8_t)(v >> (8 * k));
      }
    }
  }
}

// Waits on flag[0] (which nothing sets) until the deadline; out[0] = status,
// out[1] = device time waited.
__global__ void k_wait_test(unsigned long long* flag, unsigned long long timeout_ns, unsigned long long* out) {
  const unsigned long long t0 = gtime(), deadline = t0 + timeout_ns;
  int st = HICR_ERR_TIMEOUT;
  for (;;) {
    if (ld_acq(flag) != 0) {
      st = HICR_OK;
      break;
    }
    if (gtime() > deadline) break;
    __nanosleep(1000);
  }
  out[0] = (unsigned long long)(long long)st;
  out[1] = gtime() - t0;
}

// Bandwidth probes (no counterpart in the paper): the bounds the channel and
// host-space measurements are read against. Every thread owns the 16-byte
// vectors tid, tid + stride, ... of the range and keeps U of them in flight;
// loads go to L2 (ld.global.cg), so a range re-read by the same SM is not
// served from its L1.
static constexpr int PROBE_U = 8;

// `reps` passes of dst[0, nv) = src[0, nv) (16-byte vectors).
__global__ void k_copy_loop(uint4* __restrict__ dst, const uint4* __restrict__ src, unsigned long long nv,
                            unsigned reps) {
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned r = 0; r < reps; ++r) {
    for (unsigned long long q = tid; q < nv; q += PROBE_U * stride) {
      uint4 x[PROBE_U];
#pragma unroll
      for (int u = 0; u < PROBE_U; ++u)
        if (q + u * stride < nv) x[u] = __ldcg(src + q + u * stride);
#pragma unroll
      for (int u = 0; u < PROBE_U; ++u)
        if (q + u * stride < nv) dst[q + u * stride] = x[u];
    }
  }
}

// `reps` passes reading p[0, nv) (write = 0) or writing it (write = 1); a
// reading thread folds what it read into one word and stores it only when it
// equals a value no input makes likely, which keeps the loads alive.
__global__ void k_stream(uint4* __restrict__ p, unsigned long long nv, unsigned reps, int write,
                         unsigned long long* sink) {
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  for (unsigned r = 0; r < reps; ++r) {
    for (unsigned long long q = tid; q < nv; q += PROBE_U * stride) {
      if (write) {
#pragma unroll
        for (int u = 0; u < PROBE_U; ++u)
          if (q + u * stride < nv) __stcs(p + q + u * stride, make_uint4((unsigned)q, u, r, 0x5a5a5a5au));
      } else {
        uint4 x[PROBE_U];
#pragma unroll
        for (int u = 0; u < PROBE_U; ++u)
          if (q + u * stride < nv) x[u] = __ldcg(p + q + u * stride);
#pragma unroll
        for (int u = 0; u < PROBE_U; ++u)
          if (q + u * stride < nv) acc ^= ((unsigned long long)x[u].x << 32 | x[u].y) + x[u].z + x[u].w;
      }
    }
  }
  if (acc == 0x0123456789abcdefull) *sink = acc;
}

const void* builtin_fill_kernel() { return (const void*)k_fill; }
const void* builtin_digest_kernel() { return (const void*)k_digest; }

}  // namespace hicr

using namespace hicr;

extern "C" {

hicr_status hicr_util_fill(hicr_instance_t h, hicr_slot_t slot, uint64_t off, uint64_t n, uint64_t key_base) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || slot >= in->slots.size() || !in->slots[slot].live || in->capturing) return HICR_ERR_INVALID;
  const HostSlot& s = in->slots[slot];
  if (off > s.size || n > s.size - off) return HICR_ERR_BOUNDS;
  if (n == 0) return HICR_OK;
  const unsigned grid = (unsigned)in->sm_count * 8;
  k_fill<<<grid, 256, 0, in->comm()>>>((uint8_t*)s.base, off, n, key_base);
  HICR_CUDA(in, cudaGetLastError());
  return record_done(in);
}

hicr_status hicr_util_fill_segments(hicr_instance_t h, hicr_slot_t slot, const uint64_t* d_seg, uint64_t count) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || (count && !d_seg) || slot >= in->slots.size() || !in->slots[slot].live || in->capturing)
    return HICR_ERR_INVALID;
  const HostSlot& s = in->slots[slot];
  if (s.space != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  if (count == 0) return HICR_OK;
  const unsigned grid = (unsigned)in->sm_count * 8;
  k_fill_segments<<<grid, 256, 0, in->comm()>>>((uint8_t*)s.base, s.size, (const unsigned long long*)d_seg, count);
  HICR_CUDA(in, cudaGetLastError());
  return record_done(in);
}

hicr_status hicr_util_wait_test(hicr_instance_t h, uint64_t timeout_ns, hicr_status* status, uint64_t* waited_ns) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || !status || !waited_ns || in->capturing || timeout_ns > 60ull * 1000000000ull) return HICR_ERR_INVALID;
  unsigned long long* d = nullptr;
  HICR_CUDA(in, cudaMalloc(&d, 3 * 8));
  cudaStream_t cs = in->comm();
  unsigned long long out[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(d, 0, 3 * 8, cs);
  if (e == cudaSuccess) {
    k_wait_test<<<1, 1, 0, cs>>>(d, timeout_ns, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 1, 16, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(in, e, "wait test");
  *status = (hicr_status)(long long)out[0];
  *waited_ns = out[1];
  return HICR_OK;
}

hicr_status hicr_util_digest(hicr_instance_t h, hicr_slot_t slot, uint64_t off, uint64_t n, uint64_t* out) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || !out || slot >= in->slots.size() || !in->slots[slot].live || in->capturing) return HICR_ERR_INVALID;
  const HostSlot& s = in->slots[slot];
  if (off > s.size || n > s.size - off) return HICR_ERR_BOUNDS;
  hicr_status st = hicr_flush(h);
  if (st == HICR_OK) st = lat_drain(in);
  if (st != HICR_OK) return st;
  unsigned long long* d = in->dt.sticky + 1;  // spare word next to the sticky error
  cudaStream_t cs = in->comm();
  HICR_CUDA(in, cudaMemsetAsync(d, 0, 8, cs));
  if (n) {
    const unsigned grid = (unsigned)in->sm_count * 8;
    k_digest<<<grid, 256, 0, cs>>>((const uint8_t*)s.base + off, n, d);
    HICR_CUDA(in, cudaGetLastError());
  }
  unsigned long long v = 0;
  HICR_CUDA(in, cudaMemcpyAsync(&v, d, 8, cudaMemcpyDeviceToHost, cs));
  HICR_CUDA(in, cudaStreamSynchronize(cs));
  *out = v;
  return record_done(in);
}

}  // extern "C"

namespace hicr {

static hicr_status probe_range(Instance* in, hicr_slot_t slot, uint64_t off, uint64_t n, uint8_t** p) {
  if (slot >= in->slots.size() || !in->slots[slot].live) return HICR_ERR_INVALID;
  const HostSlot& s = in->slots[slot];
  if (off > s.size || n > s.size - off) return HICR_ERR_BOUNDS;
  *p = (uint8_t*)s.base + off;
  if (((uintptr_t)*p & 15u) || (n & 15u)) return HICR_ERR_INVALID;
  return HICR_OK;
}

// Runs `launch` between two events on the communication stream, waits, and
// returns the device time.
template <class F>
static hicr_status probe_time(Instance* in, F launch, uint64_t* device_ns) {
  cudaStream_t cs = in->comm();
  cudaEvent_t e0, e1;
  HICR_CUDA(in, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(in, e, "cudaEventCreate");
  }
  e = cudaEventRecord(e0, cs);
  if (e == cudaSuccess) {
    launch(cs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(in, e, "bandwidth probe");
  *device_ns = (uint64_t)((double)ms * 1e6);
  return record_done(in);
}

}  // namespace hicr

extern "C" {

hicr_status hicr_util_copy_loop(hicr_instance_t h, hicr_slot_t dst, uint64_t dst_off, hicr_slot_t src,
                                uint64_t src_off, uint64_t n, uint32_t reps, uint32_t ctas, uint64_t* device_ns) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || !device_ns || reps == 0 || ctas == 0 || ctas > 8u * (uint32_t)in->sm_count || in->capturing)
    return HICR_ERR_INVALID;
  uint8_t *d = nullptr, *s = nullptr;
  hicr_status st = probe_range(in, dst, dst_off, n, &d);
  if (st == HICR_OK) st = probe_range(in, src, src_off, n, &s);
  if (st != HICR_OK) return st;
  if (dst == src && dst_off < src_off + n && src_off < dst_off + n) return HICR_ERR_OVERLAP;
  if ((st = hicr_flush(h)) != HICR_OK || (st = lat_drain(in)) != HICR_OK) return st;
  return probe_time(
      in, [&](cudaStream_t cs) { k_copy_loop<<<ctas, 256, 0, cs>>>((uint4*)d, (const uint4*)s, n / 16, reps); },
      device_ns);
}

hicr_status hicr_util_stream(hicr_instance_t h, hicr_slot_t slot, uint64_t off, uint64_t n, int32_t write,
                             uint32_t reps, uint32_t ctas, uint64_t* device_ns) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || !device_ns || reps == 0 || ctas == 0 || ctas > 8u * (uint32_t)in->sm_count || in->capturing)
    return HICR_ERR_INVALID;
  uint8_t* p = nullptr;
  hicr_status st = probe_range(in, slot, off, n, &p);
  if (st != HICR_OK) return st;
  if ((st = hicr_flush(h)) != HICR_OK || (st = lat_drain(in)) != HICR_OK) return st;
  unsigned long long* sink = in->dt.sticky + 1;  // spare word next to the sticky error (never written in practice)
  return probe_time(
      in, [&](cudaStream_t cs) { k_stream<<<ctas, 256, 0, cs>>>((uint4*)p, n / 16, reps, write ? 1 : 0, sink); },
      device_ns);
}

}  // extern "C"
