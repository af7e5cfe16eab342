// The paper's Test Case 1 (Sec. 5.1) restated on one GPU: two agents, each a
// group of CTAs of one cooperative grid, exchange a single message through
// two buffers; the round-trip time gives the one-way latency and goodput.
#include <stddef.h>
#include <string.h>

#include "../../include/hicr_channels.h"
#include "../../include/hicr_util.h"
#include "channel_host.h"

namespace hicr {

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

// The same exchange for large messages when each agent has at most half the
// SMs: every CTA then has an SM to itself and takes PING_SMEM of shared memory
// for two bulk-copy stages per warp, and each warp moves its (16-byte-aligned)
// share of the CTA's part by bulk copies through them (group_copy_bulk). A
// wait on a stage that gives up raises the abort flag; the CTA leaves after
// its barrier.
static constexpr unsigned PING_NST = 2, PING_STG = 6144, PING_WARPS = 16;
static constexpr size_t PING_SMEM = (size_t)PING_WARPS * PING_NST * (PING_STG + 8);
static constexpr unsigned long long PING_WAIT_NS = 2000000000ull;  // bound of one stage wait
static constexpr unsigned long long PING_BULK_MIN = 64u << 10;     // smallest warp share for the bulk form

__global__ void __launch_bounds__(512, 1) k_pingpong_bulk(PingArgs a) {
  extern __shared__ __align__(128) uint8_t ping_smem[];
  __shared__ int s_stop, s_fail;
  const unsigned side = blockIdx.x / a.G, g = blockIdx.x % a.G;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long lo = g == 0 ? 0 : (a.bytes * g / a.G) & ~15ull;
  const unsigned long long hi = g + 1 == a.G ? a.bytes : (a.bytes * (g + 1) / a.G) & ~15ull;
  const unsigned long long n = hi - lo;
  const unsigned long long wa = warp == 0 ? 0 : (n * warp / nw) & ~15ull;
  const unsigned long long wb = warp + 1 == nw ? n : (n * (warp + 1) / nw) & ~15ull;
  uint8_t* stage = ping_smem + (size_t)warp * PING_NST * PING_STG;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(ping_smem + (size_t)PING_WARPS * PING_NST * PING_STG) + warp * PING_NST;
  if (lane == 0) {
    for (unsigned k = 0; k < PING_NST; ++k) mbar_init(bars + k);
    mbar_init_fence();
  }
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  unsigned phase = 0;
  unsigned long long* mine = a.arrive + (side ? 16 : 0);
  unsigned long long* peer = a.arrive + (side ? 0 : 16);
  const unsigned long long deadline = gtime() + a.timeout_ns;
  auto wait_peer = [&](unsigned k) -> bool {
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
    return s_stop == 0;
  };
  for (unsigned k = 1; k <= a.rounds; ++k) {
    if (side == 0 && g == 0 && threadIdx.x == 0 && k == a.warmup + 1) a.times[0] = gtime();
    if (side == 1 && !wait_peer(k)) return;  // B: wait for A's k-th message
    uint8_t* d = (side ? a.buf_a : a.buf_b) + lo;
    const uint8_t* s = (side ? a.buf_b : a.msg) + lo;
    if (wb > wa && !group_copy_bulk<PING_NST, PING_STG>(d + wa, s + wa, wb - wa, 1, lane, stage, bars, phase,
                                                        PING_WAIT_NS)) {
      if (lane == 0) s_fail = 1;
    }
    // barrier, then one cumulative release by thread 0 (no per-thread fence)
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) atomicExch(a.abort, 1u);
      return;
    }
    if (threadIdx.x == 0) red_add_rel(mine, 1ull);
    if (side == 0 && !wait_peer(k)) return;  // A: wait for the echo of round k
  }
  if (side == 0 && g == 0 && threadIdx.x == 0) a.times[1] = gtime();
}

// Capture mode: copies both single-message buffers out after the run (one
// warp per 64 KiB piece of a buffer).
__global__ void k_pp_capture(const uint8_t* buf_a, const uint8_t* buf_b, uint8_t* out_a, uint8_t* out_b,
                             unsigned long long bytes) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long piece = 64ull << 10;
  const unsigned long long np = (bytes + piece - 1) / piece;
  const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  for (unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < 2 * np;
       w += nw) {
    const unsigned long long q = w % np, lo = q * piece, n = min(piece, bytes - lo);
    if (w < np) warp_copy(out_a + lo, buf_a + lo, n, lane);
    else warp_copy(out_b + lo, buf_b + lo, n, lane);
  }
}

static hicr_status pingpong_run(hicr_instance_t h, hicr_slot_t src, uint64_t src_off, uint64_t bytes, uint32_t reps,
                                uint32_t warmup, uint32_t ctas_per_side, uint64_t timeout_ns, void* cap_a,
                                void* cap_b, hicr_pingpong_result_t* out) {
  Instance* in = I(h);
  if (!in || !out || reps == 0 || ctas_per_side == 0 || ctas_per_side > 256 || bytes == 0 || in->capturing)
    return HICR_ERR_INVALID;
  int per_sm = 0;
  HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pingpong, 512, 0));
  if (2ull * ctas_per_side > (unsigned long long)per_sm * in->sm_count) return HICR_ERR_INVALID;
  // large messages, agents of at most half the SMs: the bulk-copy form
  bool bulk = 2ull * ctas_per_side <= (unsigned long long)in->sm_count &&
              bytes / (16ull * ctas_per_side) >= PING_BULK_MIN;
  if (bulk) {
    int per_sm_b = 0;
    HICR_CUDA(in, cudaFuncSetAttribute((const void*)k_pingpong_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)PING_SMEM));
    HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_pingpong_bulk, 512, PING_SMEM));
    bulk = 2ull * ctas_per_side <= (unsigned long long)per_sm_b * in->sm_count;
  }
  void* sp = nullptr;
  uint64_t ssize = 0;
  uint32_t sspace = 0;
  if (hicr_slot_info(h, src, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  if (src_off > ssize || bytes > ssize - src_off) return HICR_ERR_BOUNDS;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  // a cooperative grid sized for the whole device: a latency-mode server ends first
  if ((st = lat_stop(in)) != HICR_OK) return st;
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
    e = bulk ? cudaLaunchCooperativeKernel((const void*)k_pingpong_bulk, dim3(2 * ctas_per_side), dim3(512), args,
                                           PING_SMEM, cs)
             : cudaLaunchCooperativeKernel((const void*)k_pingpong, dim3(2 * ctas_per_side), dim3(512), args, 0, cs);
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
  if (cap_a) {
    k_pp_capture<<<in->sm_count * 2, 512, 0, cs>>>(bufs, bufs + half, (uint8_t*)cap_a, (uint8_t*)cap_b, bytes);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      cudaFree(bufs);
      return cuda_fail(in, e, "pingpong capture");
    }
  }
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

}  // namespace hicr

using namespace hicr;

extern "C" {

hicr_status hicr_pingpong(hicr_instance_t h, hicr_slot_t src, uint64_t src_off, uint64_t bytes, uint32_t reps,
                          uint32_t warmup, uint32_t ctas_per_side, uint64_t timeout_ns, hicr_pingpong_result_t* out) {
  return pingpong_run(h, src, src_off, bytes, reps, warmup, ctas_per_side, timeout_ns, nullptr, nullptr, out);
}

hicr_status hicr_pingpong_capture(hicr_instance_t h, hicr_slot_t src, uint64_t src_off, uint64_t bytes, uint32_t reps,
                                  uint32_t warmup, uint32_t ctas_per_side, uint64_t timeout_ns, void* d_out_a,
                                  void* d_out_b, hicr_pingpong_result_t* out) {
  if (!d_out_a || !d_out_b) return HICR_ERR_INVALID;
  return pingpong_run(h, src, src_off, bytes, reps, warmup, ctas_per_side, timeout_ns, d_out_a, d_out_b, out);
}

}  // extern "C"
