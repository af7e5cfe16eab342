// Internal declarations shared by the translation units of libhicr_gb300.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hicr.h"
#include "../../include/hicr_util.h"
#include "host_pool.h"

namespace hicr {

// NVTX range around a library call (visible in Nsight timelines; a no-op when
// no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// -------------------------------------------------------------------------
// Device-resident tables. Slot metadata word: bit 0 live, bits 1..3 memory
// space, bits 8..31 tag.
// -------------------------------------------------------------------------
struct DevTables {
  uint64_t* slot_base;             // [HICR_MAX_SLOTS] device-usable address
  uint64_t* slot_size;             // [HICR_MAX_SLOTS]
  uint32_t* slot_meta;             // [HICR_MAX_SLOTS]
  unsigned long long* sent;        // [HICR_MAX_SLOTS]
  unsigned long long* recv;        // [HICR_MAX_SLOTS]
  unsigned long long* tag_ops;     // [HICR_MAX_TAGS]
  unsigned long long* sticky;      // [2]: packed (first_bad << 8 | -status), 0 = none
  unsigned long long* sig;         // [2]: completion signals emitted, CTA tickets of the small-batch kernel
  unsigned long long* sig_host;    // device address of the mapped host mirror: [0] last signal, [1] sticky then
};

// Completion signal of one memcpy launch (a batch's copy kernel, a small
// batch): called once, by the thread that finished the launch's last piece
// of work after every other thread had finished (an exit counter). It counts
// the signal on the device and writes its number, after the sticky batch
// error as of now, into mapped host memory, where fences poll it. Launches
// on the one communication stream finish in order, so the mirrored number
// only grows.
__device__ __forceinline__ void emit_signal(const DevTables& dt) {
  __threadfence();
  const unsigned long long v = atomicAdd(&dt.sig[0], 1ull) + 1ull;
  const unsigned long long sticky = atomicAdd(dt.sticky, 0ull);
  asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(dt.sig_host + 1), "l"(sticky) : "memory");
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(dt.sig_host), "l"(v) : "memory");
}

__host__ __device__ inline uint32_t meta_pack(uint32_t live, uint32_t space, uint32_t tag) {
  return (live & 1u) | ((space & 7u) << 1) | (tag << 8);
}
__host__ __device__ inline uint32_t meta_live(uint32_t m) { return m & 1u; }
__host__ __device__ inline uint32_t meta_space(uint32_t m) { return (m >> 1) & 7u; }
__host__ __device__ inline uint32_t meta_tag(uint32_t m) { return m >> 8; }

// Supported (dst space, src space) pairs as a bit mask: bit (dst * 8 + src).
__host__ __device__ inline bool pair_supported(uint32_t mask, uint32_t dsp, uint32_t ssp) {
  return (mask >> (dsp * 8u + ssp)) & 1u;
}

// Control block of one batch (device memory).
struct BatchCtrl {
  unsigned long long claim;      // next chunk to hand out
  unsigned long long nchunks;    // chunks in this batch (0 when invalid)
  unsigned long long total;      // summed cost
  unsigned long long bad;        // packed (index << 8 | -status) of the first bad op; ~0 = none
  unsigned long long exited;     // copy-kernel warps that have finished (the last one signals)
};

// Per-batch scratch, sized for `cap` ops.
struct Scratch {
  uint64_t cap = 0;
  unsigned long long* cost = nullptr;    // [cap]
  unsigned long long* cstart = nullptr;  // [cap + 1]
  unsigned int* done = nullptr;          // [cap]
  BatchCtrl* ctrl = nullptr;
  unsigned long long* tiles = nullptr;   // look-back words of the fused plan+scan, then a tile counter
  uint64_t n_tiles = 0;                  // capacity of `tiles` (excluding the counter)
};

struct BatchArgs {
  const hicr_op_t* ops;
  unsigned long long count;
  DevTables dt;
  unsigned long long* cost;
  unsigned long long* cstart;
  unsigned int* done;
  BatchCtrl* ctrl;
  unsigned int chunk;
  unsigned int op_cost;
  unsigned int support;
  unsigned int engine;
  unsigned int tma_min;
  unsigned int tma_stage;
};

// The end of a copy-kernel warp (k_copy, k_copy_tma): the last warp of the
// launch to finish emits the batch's completion signal; every op completed
// in the launch is counted by then.
__device__ __forceinline__ void copy_exit(const BatchArgs& a, unsigned lane) {
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&a.ctrl->exited, 1ull) + 1 == warps) emit_signal(a.dt);
  }
}

struct HostSlot {
  uint64_t base = 0;     // device-usable address
  void* host_ptr = nullptr;
  uint64_t size = 0;
  uint32_t space = 0;
  uint32_t tag = 0;
  bool live = false;
  bool owned = false;    // allocated by hicr_mem_alloc
};

struct Pu {
  cudaStream_t stream = nullptr;
  bool owned = false;
  bool live = false;
};

struct GraphRec {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool live = false;
  uint64_t sigs = 0;  // completion signals one launch of the graph emits
};

// Latency mode (latency.cu): the ring of small-batch ops a short-lived
// persistent server kernel takes from mapped host memory. head is written by
// the host, done and exit_epoch by the server, stop by the host.
static constexpr unsigned LAT_RING_OPS = 256;
struct LatOp {
  unsigned long long dst, src, n;  // copy: device-usable addresses, bytes
  uint32_t dslot, sslot, dtag, stag;
  uint32_t kind;                   // LAT_COPY, or LAT_CHANNEL: a channel host call
  uint32_t pad;
  unsigned long long call[12];     // LAT_CHANNEL: the call (ChanCall, channel_calls.cuh)
};
static constexpr uint32_t LAT_COPY = 0, LAT_CHANNEL = 1;
struct LatRing {
  alignas(128) unsigned long long head;        // ops published
  alignas(128) unsigned long long done;        // ops completed (counters bumped)
  alignas(128) unsigned long long exit_epoch;  // epoch of the last server that announced its exit
  alignas(128) unsigned long long stop;        // ask a running server to end
  alignas(128) LatOp ops[LAT_RING_OPS];
};

struct Channel;  // channel_host.h

struct Instance {
  int device = 0;
  cudaDeviceProp prop{};
  int sm_count = 0;
  std::vector<HostSlot> slots;
  std::vector<uint32_t> free_ids;
  DevTables dt{};
  uint32_t support = 0;
  std::vector<Pu> pus;
  uint32_t comm_pu = 0;

  // hicr_memcpy queue and host-batch upload
  std::vector<hicr_op_t> queue;
  std::unique_ptr<HostPool> pool;  // host workers for large op tables (created on first use)
  hicr_op_t* pinned[2] = {nullptr, nullptr};
  uint64_t pinned_cap[2] = {0, 0};
  cudaEvent_t pinned_ev[2] = {nullptr, nullptr};
  int pinned_idx = 0;
  hicr_op_t* d_ops = nullptr;
  uint64_t d_ops_cap = 0;

  Scratch scratch;
  hicr_batch_config_t cfg{};
  int checked = 0;

  cudaEvent_t done_ev = nullptr;  // recorded after the last issued work
  // Completion signals (fence): every memcpy launch emits one; sig_mirror is
  // the mapped host pair the device writes (last signal, sticky error then).
  unsigned long long* sig_mirror = nullptr;
  uint64_t sig_issued = 0;      // signals of the launches issued so far
  uint64_t any_sig = 0;         // signal of the last launch whose tags the host does not know
  uint64_t small_tickets = 0;   // CTAs of the small-batch kernel launched so far
  uint64_t cap_sigs = 0;        // signals of the graph being captured
  std::vector<uint64_t> tag_sig;  // per tag: signal of the last launch with an op of that tag
  bool opaque = false;          // other work issued on the communication stream since the last full wait
  // latency mode (latency.cu)
  LatRing* lat_ring = nullptr;      // mapped host ring
  LatRing* lat_ring_dev = nullptr;  // its device address
  cudaStream_t lat_stream = nullptr;
  uint64_t lat_head = 0, lat_epoch = 0, lat_idle_ns = 0;  // idle_ns 0 = latency mode off
  std::vector<uint64_t> tag_lat;    // per tag: server op count to wait for
  bool capturing = false;
  std::vector<GraphRec> graphs;

  std::unordered_map<uint64_t, cudaEvent_t> execs;
  std::vector<cudaEvent_t> exec_events;  // completion events of awaited executions, reused
  uint64_t next_exec = 1;

  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs
  size_t prof_used = 0;

  std::vector<Channel*> channels;
  void* mbox_host = nullptr;  // mapped page-locked mailbox for channel host calls
  void* mbox_dev = nullptr;
  void* chan_buf = nullptr;   // device buffer for streaming-run arguments/results
  size_t chan_buf_cap = 0;
  std::string last_err;

  cudaStream_t comm() const { return pus[comm_pu].stream; }
};

// Record a CUDA error on the instance and return HICR_ERR_DEVICE.
hicr_status cuda_fail(Instance* in, cudaError_t e, const char* what);

#define HICR_CUDA(in, call)                                   \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::hicr::cuda_fail((in), _e, #call); \
  } while (0)

// Validation shared by the host entry points (same rules the device plan
// kernel applies).
hicr_status validate_op(const Instance* in, const hicr_op_t& op);
hicr_status first_hazard(const Instance* in, const hicr_op_t* ops, uint64_t count, uint64_t* bad);

// memcpy.cu
hicr_status ensure_scratch(Instance* in, uint64_t count);
// `tags`: HICR_MAX_TAGS bits of the ops' tags, or nullptr when unknown.
hicr_status launch_batch(Instance* in, const hicr_op_t* d_ops, uint64_t count, cudaStream_t st,
                         const uint64_t* tags);
// The TMA engine of the copy kernel (copy_tma.cu): dynamic shared memory per
// CTA, one-time attribute set-up + resident CTAs per SM, launch.
bool copy_tma_shape_valid(const hicr_batch_config_t& c);
size_t copy_tma_smem(const hicr_batch_config_t& c);
hicr_status copy_tma_prepare(Instance* in, const hicr_batch_config_t& c, int* blocks_per_sm);
hicr_status launch_copy_tma(Instance* in, const BatchArgs& a, const hicr_batch_config_t& c, unsigned grid,
                            cudaStream_t st);
// Loads every stage shape of the TMA engine (cudaFuncGetAttributes).
hicr_status copy_tma_load_all(Instance* in);
// latency.cu: submit validated small ops to the server (launching one when
// needed), wait until it has completed `target` ops, stop it, free it.
hicr_status lat_submit(Instance* in, const hicr_op_t* ops, uint64_t count);
hicr_status lat_wait(Instance* in, uint64_t target, uint64_t timeout_ns);
hicr_status lat_stop(Instance* in);
// Wait (bounded) until the server has completed every op published to it:
// calls that read or write slot bytes on the communication stream after a
// flush (a channel push's source, a digest) see those copies as they would
// with the copies launched on that stream.
hicr_status lat_drain(Instance* in);
// Channel host calls in latency mode: whether the server may take one now
// (latency mode on, nothing pending on the communication stream), and the
// call itself (published to the server; waits for the status it posts).
struct ChanCall;
bool lat_takes_calls(Instance* in);
hicr_status lat_channel_call(Instance* in, const ChanCall& c, volatile int* status);
void lat_destroy(Instance* in);
// memcpy_noalloc.cu: per-device set-up of the allocation-free entry point
// (device address of its static scratch array, kernels loaded); hicr_init.
hicr_status noalloc_setup(Instance* in);
// Record the instance's done event after work on the communication stream
// that emits no completion signal (fences then wait for all of it once).
hicr_status record_done(Instance* in);
// The same after a memcpy launch accounted for by note_signal.
hicr_status record_signalled(Instance* in);
// One more completion signal issued; `mask` (HICR_MAX_TAGS bits) holds the
// tags of the launch's ops, or nullptr when the host does not know them.
void note_signal(Instance* in, const uint64_t* mask);
// Sets the bits of both slots' tags of ops[0, count) in mask (validated ops).
void tag_mask(const Instance* in, const hicr_op_t* ops, uint64_t count, uint64_t* mask);
static constexpr int TAG_WORDS = HICR_MAX_TAGS / 64;
hicr_status wait_event(Instance* in, cudaEvent_t ev, uint64_t timeout_ns);
void default_config(Instance* in, hicr_batch_config_t* c);
hicr_status check_config(const Instance* in, const hicr_batch_config_t* c);

// channels.cu
void destroy_channels(Instance* in);
void destroy_servers(Instance* in);  // serve.cu
// Records the instance's last error message (and prints it when HICR_LOG is set).
void log_error(Instance* in, const std::string& msg);

// dataobject.cu
void forget_data_objects(const Instance* in);

inline uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}
// Host waits on device progress spin for WAIT_SPIN_NS, then yield the core
// until WAIT_YIELD_NS, then sleep in short steps. A timed sleep wakes up a
// timer slack late (tens of microseconds), so the yielding phase covers the
// waits of the hot path (a fence on an epoch of a few milliseconds).
static constexpr uint64_t WAIT_SPIN_NS = 50000, WAIT_YIELD_NS = 50000000;

}  // namespace hicr

struct hicr_instance_s {
  hicr::Instance impl;
};
