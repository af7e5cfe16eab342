/*
 * hicr.h -- C ABI of the GB300 HiCR communication library (libhicr_gb300.so).
 *
 * One instance drives one GPU. The calls follow the abstract operations of
 * the HiCR model (Sec. 3.1 of "HiCR, an Abstract Model for Distributed
 * Heterogeneous Programming"): topology query, memory-slot allocation and
 * registration, memcpy between slots with fence and per-slot message
 * counters, processing units / execution units / execution states of the
 * compute manager, and (hicr_channels.h) the SPSC and MPSC channels of the
 * Channels frontend.
 *
 * Conventions (all calls):
 *  - every call returns hicr_status: HICR_OK (0) or a negative error code;
 *    nothing throws across the ABI;
 *  - out-parameters are written only on success;
 *  - a rejected call has no side effect and increments no counter;
 *  - one host thread per instance (thread-compatible, not thread-safe);
 *  - all pointers are plain host pointers unless the name says "device"
 *    (a device pointer is a CUDA global-memory address on the instance's GPU);
 *  - the library never takes ownership of caller memory; memory it allocates
 *    (hicr_mem_alloc, channel rings) it frees itself.
 */
#ifndef HICR_H
#define HICR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes                                                              */
/* ------------------------------------------------------------------------ */
typedef int32_t hicr_status;
#define HICR_OK 0
#define HICR_ERR_INVALID (-1)     /* bad handle or argument */
#define HICR_ERR_UNSUPPORTED (-2) /* memory-space pair not supported (Sec. 3.1.4: "rejected") */
#define HICR_ERR_BOUNDS (-3)      /* off + n exceeds the slot (overflow-safe) */
#define HICR_ERR_OVERLAP (-4)     /* same-slot source and destination ranges intersect */
#define HICR_ERR_HAZARD (-5)      /* checked mode: ops of one epoch touch each other's ranges */
#define HICR_ERR_NOMEM (-6)       /* memory space exhausted (Sec. 3.1.3) */
#define HICR_ERR_FULL (-7)        /* channel has no room for the push */
#define HICR_ERR_EMPTY (-8)       /* channel holds fewer messages than asked */
#define HICR_ERR_TOO_LARGE (-9)   /* message larger than the channel ring */
#define HICR_ERR_TIMEOUT (-10)    /* fence, await or a device-side wait gave up */
#define HICR_ERR_BUSY (-11)       /* object still in use by outstanding work */
#define HICR_ERR_DEVICE (-12)     /* CUDA error; see hicr_last_error_string */

/* Human-readable name of a status code (static storage; never NULL). */
const char* hicr_status_str(hicr_status s);

/* ------------------------------------------------------------------------ */
/* Handles and limits                                                        */
/* ------------------------------------------------------------------------ */
typedef struct hicr_instance_s* hicr_instance_t; /* opaque */
typedef uint32_t hicr_slot_t;                    /* index into the slot table */
typedef uint32_t hicr_pu_t;                      /* processing unit (a CUDA stream) */
typedef uint64_t hicr_exec_t;                    /* execution state */
typedef uint64_t hicr_graph_t;                   /* captured batch graph */

#define HICR_MAX_SLOTS 65536u
#define HICR_MAX_TAGS 1024u
#define HICR_MAX_SPACES 4u
#define HICR_MAX_RESOURCES 4u
#define HICR_MAX_PUS 64u

#define HICR_SPACE_HBM 0u  /* the GPU's HBM3e */
#define HICR_SPACE_HOST 1u /* page-locked host (Grace) memory, device-accessible */

#define HICR_RESOURCE_GPU 0u /* a GPU: streams run kernels on its SMs */

/* ------------------------------------------------------------------------ */
/* Instance (Sec. 3.1.1). Reduced to one instance on one GPU; it is the root  */
/* instance (the first created), which is the model's tie-break.             */
/* ------------------------------------------------------------------------ */

/* Create the instance for CUDA device `cuda_device`. Creates the default
 * processing unit (a non-blocking stream, pu 0) used by communication calls
 * and the device-resident slot table and counters.
 * Errors: INVALID (bad device or NULL out), DEVICE (CUDA failure). */
hicr_status hicr_init(int cuda_device, hicr_instance_t* out);

/* Wait for outstanding work, free every library-owned allocation and stream,
 * then the instance. Registered caller memory is left untouched. */
hicr_status hicr_finalize(hicr_instance_t inst);

/* 1 when this is the root instance (always, with a single instance). */
hicr_status hicr_is_root(hicr_instance_t inst, int32_t* out);

/* ------------------------------------------------------------------------ */
/* Topology (Sec. 3.1.2; Fig. 5 queries it first).                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t id;        /* memory-space id passed to hicr_mem_alloc */
  uint32_t kind;      /* HICR_SPACE_* */
  int32_t device;     /* CUDA device, or -1 for host memory */
  uint32_t peak_mbps; /* device spaces: theoretical bandwidth in MB/s from the
                         memory clock and bus width the driver reports
                         (2 transfers per clock); 0 when unknown or host */
  uint64_t phys_size; /* physical capacity in bytes (not the virtual size) */
  uint64_t free_size; /* bytes free when queried (device spaces), else 0 */
} hicr_memory_space_t;

typedef struct {
  uint32_t id;
  uint32_t kind;      /* HICR_RESOURCE_GPU */
  int32_t device;
  uint32_t sm_count;
  uint32_t max_threads_per_sm;
  uint32_t cc_major, cc_minor;
  uint32_t reserved;
  uint64_t l2_bytes;
  uint64_t smem_per_block_optin;
} hicr_compute_resource_t;

typedef struct {
  int32_t device;
  uint32_t n_spaces;
  uint32_t n_resources;
  uint32_t reserved;
  char name[128];
  hicr_memory_space_t spaces[HICR_MAX_SPACES];
  hicr_compute_resource_t resources[HICR_MAX_RESOURCES];
} hicr_topology_t;

/* Fill *out with the instance's device: its HBM space (id 0), the host space
 * (id 1) and the GPU compute resource. Errors: INVALID, DEVICE. */
hicr_status hicr_topology_query(hicr_instance_t inst, hicr_topology_t* out);

/* ------------------------------------------------------------------------ */
/* Memory manager (Sec. 3.1.3): local memory slots.                          */
/* A slot is {space, base address, size, tag}. The tag groups slots for      */
/* fence(tag); it defaults to 0 and must be < HICR_MAX_TAGS.                 */
/* ------------------------------------------------------------------------ */

/* Allocate `size` bytes (size > 0) in memory space `space` (HBM: cudaMalloc;
 * HOST: page-locked, mapped). Errors: INVALID (unknown space, size 0, tag out
 * of range, slot table full), NOMEM (space exhausted), DEVICE. */
hicr_status hicr_mem_alloc(hicr_instance_t inst, uint32_t space, uint64_t size, uint32_t tag,
                           hicr_slot_t* out);

/* Free a slot made by hicr_mem_alloc. Waits for outstanding work first.
 * Errors: INVALID (not a live allocated slot). */
hicr_status hicr_mem_free(hicr_instance_t inst, hicr_slot_t slot);

/* Register caller memory [ptr, ptr+size) in `space` as a slot (e.g. a torch
 * tensor's storage). The library borrows it: the caller keeps it alive until
 * hicr_slot_deregister. size may be 0. Errors: INVALID (NULL ptr with size >
 * 0, unknown space, tag out of range, table full). */
hicr_status hicr_slot_register(hicr_instance_t inst, uint32_t space, void* ptr, uint64_t size,
                               uint32_t tag, hicr_slot_t* out);

/* Forget a registered slot; does not free memory. Errors: INVALID (not a live
 * registered slot), BUSY (work issued on this instance has not completed). */
hicr_status hicr_slot_deregister(hicr_instance_t inst, hicr_slot_t slot);

/* Describe a live slot; any out pointer may be NULL. Errors: INVALID. */
hicr_status hicr_slot_info(hicr_instance_t inst, hicr_slot_t slot, void** ptr, uint64_t* size,
                           uint32_t* space, uint32_t* tag);

/* ------------------------------------------------------------------------ */
/* Communication manager (Sec. 3.1.4; Fig. 5): memcpy, fence, counters.      */
/* ------------------------------------------------------------------------ */

/* One copy: n bytes from src at src_off to dst at dst_off. 32 bytes, little
 * endian, no padding. dst/src are hicr_slot_t values. */
typedef struct {
  uint32_t dst;
  uint32_t src;
  uint64_t dst_off;
  uint64_t src_off;
  uint64_t n;
} hicr_op_t;

/* Queue one local-to-local memcpy. Validation is synchronous, the copy is
 * not: completion is only guaranteed after a fence (Sec. 3.1.4). Queued ops
 * are launched when the queue fills, at hicr_flush and at every fence.
 * Ops between two fences are unordered: an op must not write a range that
 * another op of the same epoch reads or writes.
 * Errors (no effect): INVALID (dead/unknown slot), UNSUPPORTED (space pair
 * not supported), BOUNDS (off + n > size, overflow-safe), OVERLAP (dst == src
 * with intersecting ranges). n == 0 is accepted and counts as one message. */
hicr_status hicr_memcpy(hicr_instance_t inst, hicr_slot_t dst, uint64_t dst_off, hicr_slot_t src,
                        uint64_t src_off, uint64_t n);

/* Launch every op queued by hicr_memcpy on the communication stream. */
hicr_status hicr_flush(hicr_instance_t inst);

/* Validate `count` host-resident ops, all-or-nothing, then launch them as one
 * batch (persistent size-binned copy kernel). On a validation error nothing is
 * launched and *first_bad (if not NULL) receives the index of the first bad op.
 * With checked mode on (hicr_set_checked) cross-op hazards are rejected too
 * (HAZARD). The op array may be reused when the call returns. Tables of
 * 8,192 ops or more are validated and staged by the instance's host worker
 * threads (up to 8 with the caller, started on first use); they spin, yielding,
 * for up to 5 ms after each such call before they block, so that batches
 * issued one fence apart find them awake. */
hicr_status hicr_memcpy_batch(hicr_instance_t inst, const hicr_op_t* ops, uint64_t count,
                              uint64_t* first_bad);

/* Launch a batch whose op table is already in device memory (`d_ops`,
 * 8-byte aligned, count ops; it must stay unchanged until the next fence).
 * Validation runs on the device: if any op is invalid the batch copies
 * nothing, and the next fence returns the error (hicr_batch_error gives the
 * first bad index). May be called while a graph is being captured.
 * Errors: INVALID (NULL/unaligned pointer, count > capacity reserved with
 * hicr_batch_reserve while capturing), DEVICE. */
hicr_status hicr_memcpy_batch_device(hicr_instance_t inst, const hicr_op_t* d_ops, uint64_t count);

/* Largest op count hicr_memcpy_batch_noalloc accepts. */
#define HICR_NOALLOC_MAX_OPS 32768u

/* hicr_memcpy_batch_device for callers that must not allocate GPU memory at
 * the moment they issue copies: a host framework that owns all device memory
 * through its own pool and forbids allocations outside it, a latency-critical
 * loop that cannot absorb the implicit device-wide synchronisation of
 * cudaMalloc/cudaFree, or a process whose HBM is already handed to another
 * allocator. The HiCR paper has no counterpart to this call; it only changes
 * where this library keeps its per-batch scratch.
 *  - This call allocates nothing: no cudaMalloc, cudaFree or allocating
 *    library routine. Its scratch is one file-scope device array of 640.5 KiB
 *    that every GPU which loads the library holds until the process exits.
 *  - count <= HICR_NOALLOC_MAX_OPS, otherwise HICR_ERR_TOO_LARGE and nothing
 *    is launched.
 *  - hicr_init looks up the array's device address (cudaGetSymbolAddress,
 *    with the instance's device current) and loads the kernels this call
 *    launches, so that under lazy module loading neither the array's
 *    placement nor a kernel load falls on a call of this function.
 *  - Every call, from every instance on the device, shares the one array,
 *    which keeps the last call's contents: calls whose work overlaps on the
 *    GPU race. Issue them on one stream, or order them with events.
 *  - Same validation, copies, counters and error reporting at the next fence
 *    as hicr_memcpy_batch_device; also BUSY while single ops queued by
 *    hicr_memcpy wait for a flush (flushing may allocate): call hicr_flush
 *    first. */
hicr_status hicr_memcpy_batch_noalloc(hicr_instance_t inst, const hicr_op_t* d_ops, uint64_t count);

/* Status and first bad op index of the last failed device-validated batch;
 * reading clears it. *status is HICR_OK when none failed. */
hicr_status hicr_batch_error(hicr_instance_t inst, hicr_status* status, uint64_t* first_bad);

/* Pre-size the per-batch scratch for batches of up to `max_ops` ops (needed
 * before capturing graphs; grows automatically otherwise). */
hicr_status hicr_batch_reserve(hicr_instance_t inst, uint64_t max_ops);

/* Memory-space pairs the communication manager accepts (Sec. 3.1.4: a
 * memcpy is initiated when the manager supports the pair of spaces and
 * rejected otherwise). Default: HBM <- HBM only. With host copies on, every
 * pair of HBM and HOST (page-locked Grace memory, reached by the copy
 * kernels over NVLink-C2C) is accepted. Errors: INVALID. */
hicr_status hicr_set_host_copies(hicr_instance_t inst, int32_t on);

/* Latency mode for small synchronous copies. With idle_us > 0, host
 * batches of at most 8 ops of at most 256 KiB each (what single hicr_memcpy
 * calls before a fence, Data Object gets and small hicr_memcpy_batch tables
 * give) are not launched as kernels: a persistent server kernel of one CTA,
 * on a stream of its own, takes them from a ring in mapped host memory and
 * publishes their completion there, where fences poll it. The server ends
 * after idle_us microseconds without work (at most 1 s) and the next small
 * batch starts a new one; while it runs it holds one CTA slot of one SM, and
 * device-wide synchronisations (cudaDeviceSynchronize, cudaFree) wait for it
 * to end. This library's cooperative runs (channel streams, ping-pong,
 * serving) and hicr_mem_free end a running server first; digests and the
 * bandwidth probes wait for the copies it holds, so they see them as they
 * would see copies launched on the communication stream. The ops keep the
 * model's semantics: unordered within an epoch, complete at the fence of
 * their tag, counters exact. The channel host calls (hicr_channel_push, peek,
 * pop, depth; hicr_channels.h) go to the server too while nothing is pending
 * on the communication stream, after the copies published to it before them;
 * otherwise they wait for those copies and launch as usual. Either way a
 * call sees everything issued before it, and returns the same results.
 * idle_us = 0 (the default) turns the mode off after the server's pending
 * ops complete.
 * Errors: INVALID (idle_us > 1,000,000 or capturing), DEVICE, TIMEOUT. */
hicr_status hicr_set_latency_mode(hicr_instance_t inst, uint32_t idle_us);

/* Checked mode: hicr_memcpy_batch and the hicr_memcpy queue also reject
 * cross-op hazards within one epoch (O(k log k) host check). Default off. */
hicr_status hicr_set_checked(hicr_instance_t inst, int32_t on);

/* fence(tag): flush the queue, then wait until every op issued before this
 * call that touches a slot of `tag` has completed, or `timeout_ns` elapsed
 * (TIMEOUT; the work keeps running and a later fence can succeed). When a
 * device-validated batch failed, returns its error (INVALID/BOUNDS/...).
 * On success the slot counters are final for those ops.
 * Only those ops are waited for: each memcpy launch ends with a completion
 * signal that the device writes into mapped host memory, and the fence polls
 * for the signal of the last launch holding an op of `tag`, so copies of
 * other tags issued later may still run when it returns. Device-resident
 * batches and graph launches (whose tables the host does not read) count as
 * holding every tag; other work issued on the communication stream since the
 * last fence (fills, channel calls, launches on that processing unit) is
 * waited for in full by the next fence, whatever its tag. */
hicr_status hicr_fence(hicr_instance_t inst, uint32_t tag, uint64_t timeout_ns);

/* Wait until slot's sent counter >= expect_sent and received counter >=
 * expect_recv ("the expected number of incoming and outgoing transfers",
 * Sec. 3.1.4), or TIMEOUT. It waits, as hicr_fence does, for the ops of the
 * slot's tag issued before the call, then reads the counters once; counts
 * that are still short then cannot be reached by any issued op, and the
 * call returns TIMEOUT at once. */
hicr_status hicr_fence_slot(hicr_instance_t inst, hicr_slot_t slot, uint64_t expect_sent,
                            uint64_t expect_recv, uint64_t timeout_ns);

/* Current device counters of a slot: ops completed that read it (sent) and
 * that wrote it (recv). Monotonic, never reset. Synchronous read. */
hicr_status hicr_slot_counters(hicr_instance_t inst, hicr_slot_t slot, uint64_t* sent,
                               uint64_t* recv);

/* Counters of the `count` consecutive slot handles starting at `first`
 * (arrays of count entries; either may be NULL). One synchronous read. */
hicr_status hicr_slot_counters_range(hicr_instance_t inst, hicr_slot_t first, uint32_t count,
                                     uint64_t* sent, uint64_t* recv);

/* Ops completed that touch tag (an op counts once per distinct tag of its
 * two slots). Synchronous read. */
hicr_status hicr_tag_counter(hicr_instance_t inst, uint32_t tag, uint64_t* ops);

/* The plain form: one cudaMemcpyAsync per op on the communication stream,
 * after the same host validation as hicr_memcpy_batch. No counters. */
hicr_status hicr_memcpy_batch_plain(hicr_instance_t inst, const hicr_op_t* ops, uint64_t count,
                                    uint64_t* first_bad);

/* ------------------------------------------------------------------------ */
/* Batching: copy-kernel configuration, autotuner, CUDA graphs.              */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t chunk_bytes;    /* bytes-equivalent of work per claim (multiple of 1024) */
  uint32_t op_cost_bytes;  /* per-op overhead charged in the cost model */
  uint32_t blocks_per_sm;  /* persistent grid = SMs x blocks_per_sm */
  uint32_t threads;        /* threads per block (multiple of 32, <= 1024) */
  uint32_t engine;         /* 0 = vector load/store, 1 = TMA bulk for co-aligned pieces */
  uint32_t tma_min_bytes;  /* engine 1: smallest piece copied by TMA bulk */
  uint32_t tma_stage_bytes; /* engine 1: bytes per shared-memory stage: 4096, 8192 or 16384 (0 = 4096) */
  uint32_t tma_stages;      /* engine 1: stages per warp: 2, 4 or 8 (0 = 4); warps x stages x stage
                               bytes of shared memory must fit blocks_per_sm CTAs on an SM */
} hicr_batch_config_t;

hicr_status hicr_batch_get_config(hicr_instance_t inst, hicr_batch_config_t* out);
/* Errors: INVALID when a field is out of range. */
hicr_status hicr_batch_set_config(hicr_instance_t inst, const hicr_batch_config_t* cfg);

/* Time candidate configurations on a device-resident op table (which must be
 * safe to execute repeatedly: hazard-free, sources not written) and install
 * the fastest. Each candidate is run `reps` times after one warm-up; the
 * median is compared. *best (may be NULL) receives the winner, *best_ms its
 * median time (may be NULL). Candidates cover both copy engines.
 * Tuning cache: with the environment variable HICR_TUNE_CACHE naming a file,
 * the call first runs the table once with the current configuration to learn
 * its payload bytes. It then looks up the key (device name, SM count,
 * floor(log2(ops)), floor(log2(bytes))) in that file, one JSON object per
 * line. On a hit it installs the cached configuration without trials; on a
 * miss it tunes and appends a line. */
hicr_status hicr_batch_autotune(hicr_instance_t inst, const hicr_op_t* d_ops, uint64_t count,
                                uint32_t reps, hicr_batch_config_t* best, float* best_ms);

/* Capture every communication call between begin and end into a CUDA graph
 * (stream capture of the communication stream). Only device-resident batches
 * may be issued while capturing. */
hicr_status hicr_graph_begin(hicr_instance_t inst);
hicr_status hicr_graph_end(hicr_instance_t inst, hicr_graph_t* out);
/* Launch a captured graph on the communication stream. */
hicr_status hicr_graph_launch(hicr_instance_t inst, hicr_graph_t g);
hicr_status hicr_graph_destroy(hicr_instance_t inst, hicr_graph_t g);

/* Kernel timing of batches: while enabled, each batch records CUDA events
 * around its copy kernel (also inside captured graphs).
 * hicr_profile_read synchronises and returns the summed copy-kernel time and
 * number of copy-kernel launches since the last reset. */
hicr_status hicr_profile_enable(hicr_instance_t inst, int32_t on);
hicr_status hicr_profile_reset(hicr_instance_t inst);
hicr_status hicr_profile_read(hicr_instance_t inst, float* copy_ms, uint32_t* launches);

/* ------------------------------------------------------------------------ */
/* Compute manager (Sec. 3.1.5; Fig. 6).                                     */
/* A processing unit is a CUDA stream; an execution unit is a __global__     */
/* function with its launch shape; an execution state is one launch of it    */
/* on a processing unit, awaitable with a timeout.                           */
/* ------------------------------------------------------------------------ */

/* Wrap `cuda_stream` (a cudaStream_t, e.g. torch's current stream; borrowed)
 * or, when NULL, create a new non-blocking stream owned by the library.
 * Errors: INVALID (table full), DEVICE. */
hicr_status hicr_pu_create(hicr_instance_t inst, void* cuda_stream, hicr_pu_t* out);
/* Waits for the stream, destroys it if owned. pu 0 cannot be destroyed. */
hicr_status hicr_pu_destroy(hicr_instance_t inst, hicr_pu_t pu);
/* The cudaStream_t of a processing unit. */
hicr_status hicr_pu_stream(hicr_instance_t inst, hicr_pu_t pu, void** stream);
/* Choose the processing unit communication calls are issued on (default 0).
 * Flushes the queue first. */
hicr_status hicr_comm_set_pu(hicr_instance_t inst, hicr_pu_t pu);

typedef struct {
  const void* func;   /* __global__ function (host stub address) */
  uint32_t grid[3];
  uint32_t block[3];
  uint32_t smem_bytes;
  uint32_t n_args;    /* number of kernel parameters */
} hicr_exec_unit_t;

/* Built-in execution units of this library, by name:
 *   "fill_seeded"  args (u8* slot_base, u64 off, u64 n, u64 key_base): the
 *                  seeded fill of hicr_util_fill on bytes [off, off+n);
 *   "digest_words" args (const u8* p, u64 n, u64* out): adds the word digest
 *                  of hicr_util_digest of p[0, n) to *out.
 * grid/block are set to defaults the caller may change.
 * Errors: INVALID (unknown name). */
hicr_status hicr_exec_unit_builtin(const char* name, hicr_exec_unit_t* out);

/* Launch `unit` with kernel parameters `args` (array of n_args pointers to
 * the values, as cudaLaunchKernel takes them) on processing unit `pu`.
 * Returns an execution state that completes when the kernel does.
 * Errors: INVALID (NULL unit/func, bad pu, zero grid/block), DEVICE. */
hicr_status hicr_exec_launch(hicr_instance_t inst, hicr_pu_t pu, const hicr_exec_unit_t* unit,
                             void** args, hicr_exec_t* out);
/* Non-blocking query: *done = 1 when finished. */
hicr_status hicr_exec_query(hicr_instance_t inst, hicr_exec_t e, int32_t* done);
/* Wait for completion or TIMEOUT; on success the state is finished and its
 * handle is released (it cannot be awaited again: INVALID). */
hicr_status hicr_exec_await(hicr_instance_t inst, hicr_exec_t e, uint64_t timeout_ns);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */
/* Copy the last error text recorded by this instance (a CUDA error, a
 * serving-engine timeout or self-check) into buf. With the environment
 * variable HICR_LOG set (to anything but "0"), every such message is also
 * printed to stderr when it is recorded. */
hicr_status hicr_last_error_string(hicr_instance_t inst, char* buf, uint64_t len);

#ifdef __cplusplus
}
#endif

#endif /* HICR_H */
