// hicr_memcpy_batch_noalloc: the device-validated batched memcpy for callers
// that may not allocate GPU memory when they issue copies.
//
// Some callers cannot call cudaMalloc at the point where they issue a batch:
// a host framework that owns all device memory through its own pool and
// forbids allocations outside it, a latency-critical loop that cannot afford
// the implicit device-wide synchronisation cudaMalloc/cudaFree may cause, or a
// process that has already handed nearly all HBM to another allocator. The
// regular entry point (hicr_memcpy_batch_device) grows its per-batch scratch
// with cudaMalloc; this one keeps that scratch in the file-scope array below,
// which every GPU that loads the library holds until the process exits.
//
// The copy work itself is the same: the plan, scan and copy kernels of
// memcpy.cu run unchanged, pointed at this array instead of the instance's
// scratch.
#include <mutex>

#include "hicr_internal.h"

namespace hicr {

// Kernels defined in memcpy.cu.
__global__ void k_plan(BatchArgs a);
__global__ void k_scan(BatchArgs a);
__global__ void k_copy(BatchArgs a);

// Layout of the array, in 8-byte words: the batch control block (padded to
// 256 bytes), per-op costs, the prefix sums (one extra entry), then the
// per-op piece counters (4 bytes each).
static constexpr uint64_t NA_MAX = HICR_NOALLOC_MAX_OPS;
static constexpr uint64_t NA_CTRL_WORDS = 32;
static constexpr uint64_t NA_COST_WORDS = NA_MAX;
static constexpr uint64_t NA_CSTART_WORDS = ((NA_MAX + 1 + 31) / 32) * 32;
static constexpr uint64_t NA_DONE_WORDS = NA_MAX / 2;
static constexpr uint64_t NA_WORDS = NA_CTRL_WORDS + NA_COST_WORDS + NA_CSTART_WORDS + NA_DONE_WORDS;
static_assert(sizeof(BatchCtrl) <= NA_CTRL_WORDS * 8, "control block does not fit");
static_assert(NA_MAX % 2 == 0, "piece counters are packed two per word");

static __device__ __align__(256) unsigned long long hicr_noalloc_scratch[NA_WORDS];

// Device address of the array, resolved once per device. In host code the
// array's name is only a stand-in for the device symbol, never an address a
// kernel could use.
static constexpr int NA_MAX_DEVICES = 64;
static unsigned long long* g_na_ptr[NA_MAX_DEVICES] = {nullptr};
static std::mutex g_na_mutex;

// Set-up, called by hicr_init with the instance's device current: look up
// the array's device address once per device. Under lazy module loading this
// lookup is what loads the module and places the array, so it must not wait
// for the entry point's first call. The kernels the entry point launches are
// loaded here too (cudaFuncGetAttributes loads a function), so that no call
// of it has to load code either.
hicr_status noalloc_setup(Instance* in) {
  if (in->device < 0 || in->device >= NA_MAX_DEVICES) return HICR_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[in->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, hicr_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(in, e, "cudaGetSymbolAddress(hicr_noalloc_scratch)");
    if (!p) return HICR_ERR_DEVICE;
    cudaFuncAttributes fa;
    const void* fns[] = {(const void*)k_plan, (const void*)k_scan, (const void*)k_copy};
    for (const void* f : fns) HICR_CUDA(in, cudaFuncGetAttributes(&fa, f));
    hicr_status s = copy_tma_load_all(in);
    if (s != HICR_OK) return s;
    g_na_ptr[in->device] = (unsigned long long*)p;
  }
  return HICR_OK;
}

static hicr_status noalloc_scratch(Instance* in, unsigned long long** out) {
  if (in->device < 0 || in->device >= NA_MAX_DEVICES) return HICR_ERR_INVALID;
  unsigned long long* p = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    p = g_na_ptr[in->device];
  }
  // hicr_init resolved it; an instance whose set-up failed never reaches here
  if (!p) return HICR_ERR_INVALID;
  *out = p;
  return HICR_OK;
}

}  // namespace hicr

using namespace hicr;

extern "C" hicr_status hicr_memcpy_batch_noalloc(hicr_instance_t h, const hicr_op_t* d_ops, uint64_t count) {
  Instance* in = h ? &h->impl : nullptr;
  if (!in || (count && !d_ops) || ((uintptr_t)d_ops & 7u)) return HICR_ERR_INVALID;
  if (count > NA_MAX) return HICR_ERR_TOO_LARGE;
  if (count == 0) return HICR_OK;
  // Flushing queued single ops could allocate staging memory: refuse instead.
  if (!in->queue.empty()) return HICR_ERR_BUSY;
  unsigned long long* base = nullptr;
  hicr_status s = noalloc_scratch(in, &base);
  if (s != HICR_OK) return s;

  BatchArgs a;
  a.ops = d_ops;
  a.count = count;
  a.dt = in->dt;
  a.ctrl = reinterpret_cast<BatchCtrl*>(base);
  a.cost = base + NA_CTRL_WORDS;
  a.cstart = a.cost + NA_COST_WORDS;
  a.done = reinterpret_cast<unsigned int*>(a.cstart + NA_CSTART_WORDS);
  a.chunk = in->cfg.chunk_bytes;
  a.op_cost = in->cfg.op_cost_bytes;
  a.support = in->support;
  a.engine = in->cfg.engine;
  a.tma_min = in->cfg.tma_min_bytes;
  a.tma_stage = 0;

  cudaStream_t st = in->comm();
  // The array keeps whatever the previous call left. The plan kernel zeroes
  // the piece counters and the scan kernel rewrites the prefix sums, the
  // chunk count and the claim counter; only the "first bad op" word must be
  // reset to its empty value (all ones) before the plan kernel min-reduces
  // into it.
  HICR_CUDA(in, cudaMemsetAsync(&a.ctrl->bad, 0xFF, sizeof(a.ctrl->bad), st));
  const unsigned pb = (unsigned)((count + 255) / 256);
  k_plan<<<pb, 256, 0, st>>>(a);
  k_scan<<<1, 1024, 0, st>>>(a);
  const unsigned grid = (unsigned)in->sm_count * in->cfg.blocks_per_sm;
  if (in->cfg.engine == 1) {  // the TMA engine's stages are shared memory, not an allocation
    if ((s = launch_copy_tma(in, a, in->cfg, grid, st)) != HICR_OK) return s;
  } else {
    k_copy<<<grid, in->cfg.threads, 0, st>>>(a);
  }
  HICR_CUDA(in, cudaGetLastError());
  note_signal(in, nullptr);  // the copy kernel's last warp signals; the table's tags are not read here
  return record_signalled(in);
}
