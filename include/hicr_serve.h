/*
 * hicr_serve.h -- continuous-batching request loop of libhicr_gb300.so.
 *
 * The HiCR paper's Channels frontend targets request-driven applications with
 * a low-latency turnaround (Sec. 4.3); this module serves such requests on
 * one GPU. A request is either a memcpy batch (a template of ops whose
 * destinations are offsets inside the request's own destination region) or an
 * MPSC burst (a template of messages pushed, in order, into one of the
 * engine's MPSC channels and drained by its consumer).
 *
 * hicr_serve_run runs a host admission loop in the calling thread and one
 * persistent device kernel:
 *  - requests are admitted in arrival order as the destination arena (the
 *    device-memory budget minus the channel rings) has room for their region;
 *  - admitted requests are published through a doorbell in mapped host memory;
 *    a dispatcher warp moves them into a device-side request table and cuts
 *    them into work units (memcpy: cost chunks, small enough to occupy the
 *    idle worker warps; burst: groups of up to 2 messages or 32 KiB, whose
 *    channel tickets and ring bytes the first group reserves for the whole
 *    burst when it takes at most half the ring); worker warps claim units
 *    from the 32 oldest requests that
 *    still have unclaimed units, taking the one with the fewest unclaimed
 *    units first (continuous batching with shortest-remaining-first order
 *    inside that window: work of requests admitted at different times
 *    overlaps on the device, and a small request is not queued behind the
 *    units of a large one);
 *  - the unit that finishes a request writes its completion into mapped host
 *    memory; the host frees the request's region and records the latency from
 *    arrival to the moment it saw the completion.
 * Every device wait is bounded by the run's deadline.
 *
 * Conventions as in hicr.h.
 */
#ifndef HICR_SERVE_H
#define HICR_SERVE_H

#include <stdint.h>

#include "hicr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef uint64_t hicr_serve_t;

typedef struct {
  uint64_t budget_bytes;  /* device-memory budget: destination arena + channel rings */
  uint32_t n_channels;    /* MPSC channels (one consumer CTA each), >= 1 */
  uint32_t max_msgs;      /* metadata entries per channel (power of two) */
  uint64_t ring_bytes;    /* per channel ring (power of two) */
  uint32_t chunk_bytes;   /* largest memcpy work unit (cost bytes, multiple of 1024). When a request
                             is published it is cut into enough units (of at least 16 KiB) to
                             occupy the worker warps that no published work waits for, so that on
                             an idle engine it spreads over many warps; with every warp busy its
                             units are chunk_bytes */
  uint32_t op_cost_bytes; /* per-op charge of the cost model */
  uint32_t verify;        /* 1: never reuse destination regions, so that results
                             can be digested after the run (tests) */
  uint32_t reserved;
} hicr_serve_config_t;

typedef struct {
  uint64_t arrival_ns; /* offset from the start of the run */
  uint32_t kind;       /* 0 = memcpy batch, 1 = MPSC burst */
  uint32_t tmpl;       /* template index of that kind */
} hicr_serve_request_t;

typedef struct {
  uint64_t latency_ns;  /* host-observed completion minus arrival */
  uint64_t admit_ns;    /* admission minus arrival (queueing for the budget) */
  uint64_t digest;      /* MPSC burst: sum over messages m of (2m+1) * word digest
                           of message m as consumed; memcpy: see hicr_serve_digests */
  uint64_t dst_offset;  /* memcpy: offset of the request's region in the arena */
  uint64_t device_done_ns; /* engine mode: the device clock (%globaltimer, ns) when the request
                              completed, which the host's latency_ns observes later; it shares
                              no origin with the host clock, so only its differences mean
                              anything. Plain mode: 0 */
} hicr_serve_result_t;

typedef struct {
  uint64_t completed;
  uint64_t bytes_moved;      /* memcpy payload bytes + burst payload bytes */
  uint64_t wall_ns;          /* first arrival to last completion */
  uint64_t max_inflight;     /* most requests admitted and not complete at once */
  uint64_t max_region_bytes; /* high-water mark of the arena */
  uint64_t admitted;         /* requests published to the device */
  uint64_t dev_units;        /* work units the dispatcher published */
  uint64_t dev_claimed;      /* work units claimed by workers */
  uint64_t dev_requests;     /* requests the dispatcher took over */
  uint64_t dev_flags;        /* bit 0 stop seen, bit 1 abort (deadline), bit 2 self-check */
  int32_t status;            /* HICR_OK or HICR_ERR_TIMEOUT */
  uint32_t reserved;
  uint64_t burst_bytes;      /* the burst part of bytes_moved (the rest is memcpy payload): each burst
                                byte is read from staging, written to a ring and read by the consumer
                                (3 bytes of traffic), each memcpy byte read and written once (2) */
  uint64_t max_poll_gap_ns;    /* longest interval between two passes of the host's admission and
                                  completion loop (a thread the OS did not run meanwhile shows here) */
  uint64_t max_poll_gap_at_ns; /* when that interval ended, from the start of the run */
} hicr_serve_stats_t;

/* Create a serving engine: allocates the destination arena and the channel
 * rings (together budget_bytes) in HBM. Errors: INVALID, NOMEM, DEVICE. */
hicr_status hicr_serve_create(hicr_instance_t inst, const hicr_serve_config_t* cfg, hicr_serve_t* out);
hicr_status hicr_serve_destroy(hicr_instance_t inst, hicr_serve_t srv);

/* Add a memcpy template: `count` ops (host array) whose `dst` field is
 * ignored (0 = the request's region) and whose dst_off must lie inside
 * region_bytes; src/src_off name live HBM slots. Templates are added before
 * the first run. Errors: INVALID, BOUNDS (an op outside its source slot or
 * region), UNSUPPORTED (a source not in HBM). */
hicr_status hicr_serve_add_memcpy_template(hicr_instance_t inst, hicr_serve_t srv, const hicr_op_t* ops,
                                           uint64_t count, uint64_t region_bytes, uint32_t* tmpl);

/* Add an MPSC burst template: `count` messages of sizes[i] bytes read from
 * slot `staging` at staging_off[i] (host arrays). A burst request of this
 * template is pushed into channel (request index mod n_channels) as
 * producer = request index, seq = message index. Each message must be at most
 * half a ring. Errors: INVALID, BOUNDS, TOO_LARGE. */
hicr_status hicr_serve_add_burst_template(hicr_instance_t inst, hicr_serve_t srv, const uint64_t* sizes,
                                          const uint64_t* staging_off, uint64_t count, hicr_slot_t staging,
                                          uint32_t* tmpl);

/* Serve `n` requests (host array, sorted by arrival). mode 0 = by arrival
 * time (the trace), mode 1 = alone (request i+1 is admitted only after
 * request i completed). results: host array of n (may be NULL), zeroed
 * before the run starts (so a freshly mapped array takes its page faults
 * outside the run); an entry stays zero if its request did not complete.
 * stats may be NULL. Synchronous. The engine checks itself while it runs: an entry
 * outside the run, or a burst message consumed out of its request's order,
 * stops it with DEVICE (stats.dev_flags bit 2; the message names the request).
 * Errors: INVALID (unknown template, unsorted), NOMEM (a
 * request's region exceeds the arena), DEVICE, TIMEOUT (not finished within
 * timeout_ns; the engine stops, and if its kernel has not ended 10 s later
 * the call returns anyway and leaves the run's buffers allocated). */
hicr_status hicr_serve_run(hicr_instance_t inst, hicr_serve_t srv, const hicr_serve_request_t* reqs, uint64_t n,
                           uint32_t mode, uint64_t timeout_ns, hicr_serve_result_t* results,
                           hicr_serve_stats_t* stats);

/* hicr_serve_run with two checking aids (tests, sampled checks of long runs):
 *  - keep: NULL or a host array of n flags; the destination region of every
 *    memcpy request r with keep[r] != 0 is not reused after the request
 *    completes (as every region is in verify mode), so that its bytes can be
 *    read after the run (hicr_serve_arena, result dst_offset) or digested
 *    (hicr_serve_digests). Kept regions stay taken for the rest of the run;
 *  - d_capture, d_cap_off: NULL, or a device buffer and a device array of n
 *    u64 offsets: the consumer copies message m of burst request r, as it
 *    consumed it from the channel ring, to d_capture + d_cap_off[r] + (sum of
 *    the sizes of the template's messages before m), unless d_cap_off[r] is
 *    UINT64_MAX. The caller sizes the buffer.
 * Errors: as hicr_serve_run, plus INVALID (d_capture without d_cap_off). */
hicr_status hicr_serve_run_ex(hicr_instance_t inst, hicr_serve_t srv, const hicr_serve_request_t* reqs, uint64_t n,
                              uint32_t mode, uint64_t timeout_ns, const uint8_t* keep, void* d_capture,
                              const uint64_t* d_cap_off, hicr_serve_result_t* results, hicr_serve_stats_t* stats);

/* The engine's destination arena as a (library-owned) HBM slot: the region of
 * memcpy request r starts at result[r].dst_offset. Errors: INVALID. */
hicr_status hicr_serve_arena(hicr_instance_t inst, hicr_serve_t srv, hicr_slot_t* out);

/* The plain form on the same requests: one cudaMemcpyAsync per op (memcpy
 * requests) or per message into the channel ring space (bursts; no consumer),
 * in arrival order on one stream, with the same admission budget. Requests
 * with arrival time beyond `horizon_ns` are not served. */
hicr_status hicr_serve_run_plain(hicr_instance_t inst, hicr_serve_t srv, const hicr_serve_request_t* reqs,
                                 uint64_t n, uint64_t horizon_ns, uint64_t timeout_ns,
                                 hicr_serve_result_t* results, hicr_serve_stats_t* stats);

/* After a run that kept regions (verify mode, or keep flags of
 * hicr_serve_run_ex; reqs and n as in that run): result[i].digest of every
 * memcpy request i whose region was kept becomes sum over its ops k of
 * (2k+1) * word digest of op k's destination bytes; other results are left
 * as they are. Errors: INVALID (no region kept, or n differs from the last
 * run), DEVICE. */
hicr_status hicr_serve_digests(hicr_instance_t inst, hicr_serve_t srv, const hicr_serve_request_t* reqs,
                               uint64_t n, hicr_serve_result_t* results);

#ifdef __cplusplus
}
#endif

#endif /* HICR_SERVE_H */
