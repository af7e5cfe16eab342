// The TMA engine of the batched copy (batch configuration engine = 1).
//
// Same work distribution as k_copy (warps claim chunks of the cost model and
// copy the byte pieces of the ops a chunk overlaps), but a piece of at least
// tma_min bytes whose source and destination are both in HBM and have the same
// address residue mod 16 moves its 16-byte-aligned body through the Tensor
// Memory Accelerator: lane 0 of the warp streams the body in STG-byte pieces
// through NST shared-memory stages (template parameters: 2, 4 or 8 stages of
// 4, 8 or 16 KiB, chosen by the batch configuration), each a bulk global->shared load
// completed on the stage's mbarrier (cp.async.bulk ... complete_tx) followed
// by a bulk shared->global store (cp.async.bulk ... bulk_group). A stage is
// refilled only after the store that read it has finished reading
// (cp.async.bulk.wait_group.read). The unaligned head and the sub-16-byte tail
// go through the vector warp copy. Every mbarrier wait is bounded; one that
// gives up records HICR_ERR_TIMEOUT for the op in the sticky batch error,
// first waits (each wait bounded again) for the warp's loads still in flight
// so that no bulk copy writes into the stages after the warp has left them,
// and leaves the op uncounted: its sent/recv/tag counters are not bumped and
// its destination bytes are undefined, which the next fence reports as
// TIMEOUT.
#include "copy.cuh"
#include "hicr_internal.h"
#include "tma.cuh"

namespace hicr {

static constexpr unsigned FULLM_COPY = 0xffffffffu;
static constexpr unsigned long long TMA_WAIT_NS = 2000000000ull;  // bound of one mbarrier wait

// Lane 0: copy n bytes (a multiple of 16; d and s 16-byte aligned) through the
// warp's stages. `phase` holds one parity bit per stage. Returns false when a
// wait gave up (the copy is then incomplete).
template <unsigned NST, unsigned STG>
__device__ bool tma_body(uint8_t* d, const uint8_t* s, unsigned long long n, uint8_t* stage,
                         unsigned long long* bars, unsigned& phase) {
  const unsigned long long np = (n + STG - 1) / STG;
  auto piece_bytes = [&](unsigned long long p) -> unsigned {
    const unsigned long long off = p * STG;
    return (unsigned)(n - off < STG ? n - off : STG);
  };
  const unsigned long long pro = np < NST - 1 ? np : NST - 1;
  for (unsigned long long p = 0; p < pro; ++p) {
    const unsigned k = (unsigned)(p % NST);
    mbar_expect_tx(bars + k, piece_bytes(p));
    tma_load(stage + k * STG, s + p * STG, piece_bytes(p), bars + k);
  }
  bool ok = true;
  for (unsigned long long p = 0; p < np; ++p) {
    const unsigned long long q = p + NST - 1;
    if (q < np) {
      // stage q % NST last held piece p - 1: its store must have read it
      tma_wait_read0();
      const unsigned k = (unsigned)(q % NST);
      mbar_expect_tx(bars + k, piece_bytes(q));
      tma_load(stage + k * STG, s + q * STG, piece_bytes(q), bars + k);
    }
    const unsigned k = (unsigned)(p % NST);
    const unsigned par = (phase >> k) & 1u;
    if (!mbar_try_wait(bars + k, par)) {
      const unsigned long long t0 = tma_now_ns();
      while (!mbar_try_wait(bars + k, par)) {
        if (tma_now_ns() - t0 > TMA_WAIT_NS) {
          ok = false;
          break;
        }
      }
    }
    if (!ok) {
      // Pieces p .. last_issued have loads in flight, one per stage; wait
      // for each (bounded) before the stages can be left behind.
      const unsigned long long last = (p + NST - 1 < np ? p + NST - 1 : np - 1);
      for (unsigned long long r = p; r <= last; ++r) {
        const unsigned kr = (unsigned)(r % NST);
        const unsigned long long t1 = tma_now_ns();
        while (!mbar_try_wait(bars + kr, (phase >> kr) & 1u)) {
          if (tma_now_ns() - t1 > TMA_WAIT_NS) break;
        }
        phase ^= 1u << kr;
      }
      break;
    }
    phase ^= 1u << k;
    tma_store(d + p * STG, stage + k * STG, piece_bytes(p));
    tma_commit();
  }
  tma_wait_all();
  // order the async-proxy writes before the generic-proxy completion signal
  fence_proxy_async_global();
  return ok;
}

template <unsigned NST, unsigned STG>
__global__ void __launch_bounds__(1024) k_copy_tma(BatchArgs a) {
  extern __shared__ __align__(128) uint8_t tma_smem[];
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint8_t* stage = tma_smem + (size_t)warp * NST * STG;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(tma_smem + (size_t)nwarp * NST * STG) + warp * NST;
  if (lane == 0) {
    for (unsigned k = 0; k < NST; ++k) mbar_init(bars + k);
    mbar_init_fence();
  }
  __syncwarp();
  unsigned phase = 0;  // lane 0: parity of each stage's next completion
  int tma_ok = 1;      // cleared (warp-uniformly) after a wait gave up: the warp stops using its stages
  const unsigned long long nchunks = *(volatile unsigned long long*)&a.ctrl->nchunks;
  const unsigned long long total = *(volatile unsigned long long*)&a.ctrl->total;
  const unsigned long long chunk = a.chunk;
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(&a.ctrl->claim, 1ull);
    c = __shfl_sync(FULLM_COPY, c, 0);
    if (c >= nchunks) break;
    const unsigned long long lo = c * chunk;
    const unsigned long long hi = min(lo + chunk, total);
    for (unsigned long long i = find_op(a.cstart, a.count, lo, lane); i < a.count; ++i) {
      const unsigned long long cs = a.cstart[i];
      if (cs >= hi) break;
      const hicr_op_t op = a.ops[i];
      const unsigned long long bs = cs + a.op_cost;
      const unsigned long long be = bs + op.n;
      const unsigned long long b0 = lo > bs ? lo - bs : 0ull;
      const unsigned long long b1 = (hi < be ? hi : be) > bs ? (hi < be ? hi : be) - bs : 0ull;
      int piece_done = 1;  // cleared (warp-uniformly) when this piece's bulk copy gave up
      if (b1 > b0) {
        uint8_t* d = reinterpret_cast<uint8_t*>(a.dt.slot_base[op.dst]) + op.dst_off + b0;
        const uint8_t* s = reinterpret_cast<const uint8_t*>(a.dt.slot_base[op.src]) + op.src_off + b0;
        const unsigned long long n = b1 - b0;
        const bool hbm = meta_space(a.dt.slot_meta[op.dst]) == HICR_SPACE_HBM &&
                         meta_space(a.dt.slot_meta[op.src]) == HICR_SPACE_HBM;
        const unsigned long long head = (16 - (reinterpret_cast<uintptr_t>(d) & 15)) & 15;
        if (tma_ok && hbm && n >= a.tma_min && n >= head + 16 &&
            ((reinterpret_cast<uintptr_t>(d) ^ reinterpret_cast<uintptr_t>(s)) & 15) == 0) {
          const unsigned long long body = (n - head) & ~15ull, tail = n - head - body;
          if (head) warp_copy(d, s, head, lane);
          if (tail) warp_copy(d + head + body, s + head + body, tail, lane);
          int ok = 1;
          if (lane == 0) ok = tma_body<NST, STG>(d + head, s + head, body, stage, bars, phase);
          ok = __shfl_sync(FULLM_COPY, ok, 0);
          if (!ok) {
            tma_ok = 0;
            piece_done = 0;
            if (lane == 0) atomicCAS(a.dt.sticky, 0ull, (i << 8) | (unsigned long long)(-HICR_ERR_TIMEOUT));
          }
        } else {
          warp_copy(d, s, n, lane);
        }
      }
      const unsigned pieces = (unsigned)((be - 1) / chunk - cs / chunk + 1);
      __threadfence();
      __syncwarp();
      if (lane == 0 && piece_done) {
        const unsigned prev = atomicAdd(&a.done[i], 1u);
        if (prev + 1 == pieces) {
          __threadfence();
          atomicAdd(&a.dt.sent[op.src], 1ull);
          atomicAdd(&a.dt.recv[op.dst], 1ull);
          const uint32_t ts = meta_tag(a.dt.slot_meta[op.src]);
          const uint32_t td = meta_tag(a.dt.slot_meta[op.dst]);
          atomicAdd(&a.dt.tag_ops[ts], 1ull);
          if (td != ts) atomicAdd(&a.dt.tag_ops[td], 1ull);
        }
      }
    }
  }
  copy_exit(a, lane);
}

// The stage shapes the batch configuration may ask for.
#define HICR_TMA_SHAPES(X) X(2, 4096) X(4, 4096) X(8, 4096) X(2, 8192) X(4, 8192) X(8, 8192) X(2, 16384) X(4, 16384) X(8, 16384)

static void tma_shape(const hicr_batch_config_t& c, unsigned* nst, unsigned* stg) {
  *nst = c.tma_stages ? c.tma_stages : 4;
  *stg = c.tma_stage_bytes ? c.tma_stage_bytes : 4096;
}

static const void* tma_kernel(unsigned nst, unsigned stg) {
#define HICR_TMA_PICK(N, S) \
  if (nst == N && stg == S) return (const void*)k_copy_tma<N, S>;
  HICR_TMA_SHAPES(HICR_TMA_PICK)
#undef HICR_TMA_PICK
  return nullptr;
}

hicr_status copy_tma_load_all(Instance* in) {
  cudaFuncAttributes fa;
#define HICR_TMA_LOAD(N, S) HICR_CUDA(in, cudaFuncGetAttributes(&fa, (const void*)k_copy_tma<N, S>));
  HICR_TMA_SHAPES(HICR_TMA_LOAD)
#undef HICR_TMA_LOAD
  return HICR_OK;
}

bool copy_tma_shape_valid(const hicr_batch_config_t& c) {
  unsigned nst, stg;
  tma_shape(c, &nst, &stg);
  return tma_kernel(nst, stg) != nullptr;
}

size_t copy_tma_smem(const hicr_batch_config_t& c) {
  unsigned nst, stg;
  tma_shape(c, &nst, &stg);
  return (size_t)(c.threads / 32) * ((size_t)nst * stg + nst * 8);
}

hicr_status copy_tma_prepare(Instance* in, const hicr_batch_config_t& c, int* blocks_per_sm) {
  *blocks_per_sm = 0;
  unsigned nst, stg;
  tma_shape(c, &nst, &stg);
  const void* k = tma_kernel(nst, stg);
  const size_t smem = copy_tma_smem(c);
  if (!k || smem > in->prop.sharedMemPerBlockOptin) return HICR_OK;  // cannot be resident at all
  // allow the largest opt-in size once, so that every shape that fits can launch
  HICR_CUDA(in, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)in->prop.sharedMemPerBlockOptin));
  int per_sm = 0;
  HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, c.threads, smem));
  *blocks_per_sm = per_sm;
  return HICR_OK;
}

hicr_status launch_copy_tma(Instance* in, const BatchArgs& a, const hicr_batch_config_t& c, unsigned grid,
                            cudaStream_t st) {
  unsigned nst, stg;
  tma_shape(c, &nst, &stg);
  const void* k = tma_kernel(nst, stg);
  if (!k) return HICR_ERR_INVALID;
  BatchArgs args = a;
  void* params[] = {&args};
  HICR_CUDA(in, cudaLaunchKernel(k, dim3(grid), dim3(c.threads), params, copy_tma_smem(c), st));
  return HICR_OK;
}

}  // namespace hicr
