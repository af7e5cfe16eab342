// Test kernels for the device-side channel calls (include/hicr_device.cuh),
// built into a small shared library by tests/test_gpu_device_api.py. Every
// launcher returns the cudaError_t of its launch; the kernels record the
// first non-OK status of each role in `status`.
#include <cuda_runtime.h>

#include "hicr_device.cuh"

// SPSC. mode 0: warp 0 of block 0 pushes n tokens from src in batches of
// `batch` while warp 0 of block 1 pops them into dst (one cooperative grid);
// mode 1: one warp only pushes; mode 2: one warp only pops.
__global__ void k_spsc(hicr_channel_view_t v, const uint8_t* src, uint8_t* dst, unsigned n, unsigned batch,
                       unsigned long long timeout_ns, int mode, int* status) {
  if (threadIdx.x >= 32) return;
  const bool push = mode == 1 || (mode == 0 && blockIdx.x == 0);
  for (unsigned i = 0; i < n; i += batch) {
    const unsigned k = batch < n - i ? batch : n - i;
    const size_t off = (size_t)i * v.token_size;
    const int st = push ? hicr_dev_spsc_push(v, src + off, k, timeout_ns) : hicr_dev_spsc_pop(v, dst + off, k, timeout_ns);
    if (st != HICR_OK) {
      if (threadIdx.x == 0) status[push ? 0 : 1] = st;
      return;
    }
  }
}

// MPSC (locking). Blocks [0, P) are producers (warp 0 each): producer p pushes
// its M messages (p, 0..M-1) from staging. Block P (warp 0) is the consumer
// when `consume` is set: it pops P*M messages into out (stride out_stride)
// and records each one's description in infos.
__global__ void k_mpsc(hicr_channel_view_t v, const uint8_t* staging, const unsigned long long* offs,
                       const unsigned long long* sizes, unsigned P, unsigned M, int consume, uint8_t* out,
                       unsigned long long out_stride, hicr_msg_info_t* infos, unsigned long long timeout_ns,
                       int* status) {
  if (threadIdx.x >= 32) return;
  if (blockIdx.x < P) {
    const unsigned p = blockIdx.x;
    for (unsigned s = 0; s < M; ++s) {
      const size_t i = (size_t)p * M + s;
      const int st = hicr_dev_mpsc_push(v, p, s, staging + offs[i], (uint32_t)sizes[i], timeout_ns);
      if (st != HICR_OK) {
        if (threadIdx.x == 0) atomicCAS(status, 0, st);
        return;
      }
    }
  } else if (consume) {
    for (unsigned long long j = 0; j < (unsigned long long)P * M; ++j) {
      const int st = hicr_dev_mpsc_pop(v, out + j * out_stride, out_stride, infos + j, timeout_ns);
      if (st != HICR_OK) {
        if (threadIdx.x == 0) status[1] = st;
        return;
      }
    }
  }
}

// MPSC consumer alone: pops `count` messages (pushed by the host).
__global__ void k_mpsc_pop(hicr_channel_view_t v, unsigned long long count, uint8_t* out, unsigned long long out_stride,
                           hicr_msg_info_t* infos, unsigned long long timeout_ns, int* status) {
  if (threadIdx.x >= 32) return;
  for (unsigned long long j = 0; j < count; ++j) {
    const int st = hicr_dev_mpsc_pop(v, out + j * out_stride, out_stride, infos + j, timeout_ns);
    if (st != HICR_OK) {
      if (threadIdx.x == 0) status[1] = st;
      return;
    }
  }
}

extern "C" int devapi_spsc(const hicr_channel_view_t* v, const void* src, void* dst, unsigned n, unsigned batch,
                           unsigned long long timeout_ns, int mode, int* status) {
  hicr_channel_view_t view = *v;
  if (mode == 0) {
    const uint8_t* s = (const uint8_t*)src;
    uint8_t* d = (uint8_t*)dst;
    void* args[] = {&view, &s, &d, &n, &batch, &timeout_ns, &mode, &status};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_spsc, dim3(2), dim3(32), args, 0, 0);
    return e == cudaSuccess ? (int)cudaDeviceSynchronize() : (int)e;
  }
  k_spsc<<<1, 32>>>(view, (const uint8_t*)src, (uint8_t*)dst, n, batch, timeout_ns, mode, status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? (int)cudaDeviceSynchronize() : (int)e;
}

extern "C" int devapi_mpsc(const hicr_channel_view_t* v, const void* staging, const unsigned long long* offs,
                           const unsigned long long* sizes, unsigned P, unsigned M, int consume, void* out,
                           unsigned long long out_stride, hicr_msg_info_t* infos, unsigned long long timeout_ns,
                           int* status) {
  hicr_channel_view_t view = *v;
  const uint8_t* st = (const uint8_t*)staging;
  uint8_t* o = (uint8_t*)out;
  void* args[] = {&view, &st, &offs, &sizes, &P, &M, &consume, &o, &out_stride, &infos, &timeout_ns, &status};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_mpsc, dim3(P + (consume ? 1 : 0)), dim3(32), args, 0, 0);
  return e == cudaSuccess ? (int)cudaDeviceSynchronize() : (int)e;
}

extern "C" int devapi_mpsc_pop(const hicr_channel_view_t* v, unsigned long long count, void* out,
                               unsigned long long out_stride, hicr_msg_info_t* infos, unsigned long long timeout_ns,
                               int* status) {
  k_mpsc_pop<<<1, 32>>>(*v, count, (uint8_t*)out, out_stride, infos, timeout_ns, status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? (int)cudaDeviceSynchronize() : (int)e;
}

// Non-locking MPSC. Blocks [0, P) are producers (warp 0 each), each pushing
// its M messages into its own ring; block P (warp 0) is the consumer when
// `consume` is set and pops P*M messages with pop_any.
__global__ void k_nl(hicr_channel_view_t v, const uint8_t* staging, const unsigned long long* offs,
                     const unsigned long long* sizes, unsigned P, unsigned M, int consume, uint8_t* out,
                     unsigned long long out_stride, hicr_msg_info_t* infos, unsigned long long timeout_ns,
                     int* status) {
  if (threadIdx.x >= 32) return;
  if (blockIdx.x < P) {
    const unsigned p = blockIdx.x;
    for (unsigned s = 0; s < M; ++s) {
      const size_t i = (size_t)p * M + s;
      const int st = hicr_dev_mpsc_nl_push(v, p, s, staging + offs[i], (uint32_t)sizes[i], timeout_ns);
      if (st != HICR_OK) {
        if (threadIdx.x == 0) atomicCAS(status, 0, st);
        return;
      }
    }
  } else if (consume) {
    uint32_t next = 0;
    for (unsigned long long j = 0; j < (unsigned long long)P * M; ++j) {
      const int st = hicr_dev_mpsc_nl_pop_any(v, &next, out + j * out_stride, out_stride, infos + j, timeout_ns);
      if (st != HICR_OK) {
        if (threadIdx.x == 0) status[1] = st;
        return;
      }
    }
  }
}

extern "C" int devapi_nl(const hicr_channel_view_t* v, const void* staging, const unsigned long long* offs,
                         const unsigned long long* sizes, unsigned P, unsigned M, int consume, void* out,
                         unsigned long long out_stride, hicr_msg_info_t* infos, unsigned long long timeout_ns,
                         int* status) {
  hicr_channel_view_t view = *v;
  const uint8_t* st = (const uint8_t*)staging;
  uint8_t* o = (uint8_t*)out;
  void* args[] = {&view, &st, &offs, &sizes, &P, &M, &consume, &o, &out_stride, &infos, &timeout_ns, &status};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_nl, dim3(P + (consume ? 1 : 0)), dim3(32), args, 0, 0);
  return e == cudaSuccess ? (int)cudaDeviceSynchronize() : (int)e;
}
