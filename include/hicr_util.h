/*
 * hicr_util.h -- workload and checking utilities of libhicr_gb300.so.
 *
 * The HiCR paper has no counterpart to these calls: they produce synthetic
 * slot contents on the device and digest slot bytes so that large results can
 * be compared without copying them back. Conventions as in hicr.h.
 */
#ifndef HICR_UTIL_H
#define HICR_UTIL_H

#include <stdint.h>

#include "hicr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Fill bytes [off, off+n) of `slot` so that byte i of the slot (counted from
 * the slot start) is byte (i mod 8), little endian, of SplitMix64's first
 * output for state key_base + floor(i/8), i.e. finalise(key_base + i/8 +
 * 0x9E3779B97F4A7C15) with the published SplitMix64 finaliser (Steele, Lea
 * and Flood, OOPSLA 2014). Runs on the communication stream (asynchronous).
 * Errors: INVALID (dead slot), BOUNDS (off + n > size), UNSUPPORTED (host
 * slot), DEVICE. */
hicr_status hicr_util_fill(hicr_instance_t inst, hicr_slot_t slot, uint64_t off, uint64_t n,
                           uint64_t key_base);

/* Seeded fill of `count` segments of `slot`. d_seg is a device array of
 * count triples {off, n, key_base} (u64): byte j of segment [off, off+n) is
 * byte (j mod 8), little endian, of the SplitMix64 first output for state
 * key_base + floor(j/8) -- each segment restarts its own word count.
 * Asynchronous on the communication stream. A segment that does not lie
 * inside the slot is skipped.
 * Errors: INVALID, UNSUPPORTED (host slot), DEVICE. */
hicr_status hicr_util_fill_segments(hicr_instance_t inst, hicr_slot_t slot, const uint64_t* d_seg,
                                    uint64_t count);

/* Word digest of bytes [off, off+n) of `slot`: with w_j the little-endian
 * 8-byte words of that range (last word zero-padded), D = sum_j w_j * (2j+1)
 * mod 2^64. Synchronous (waits for the communication stream first).
 * Errors: INVALID, BOUNDS, DEVICE. */
hicr_status hicr_util_digest(hicr_instance_t inst, hicr_slot_t slot, uint64_t off, uint64_t n,
                             uint64_t* out);

/* Self-test of the bounded device waits that every spin in this library
 * uses: launches one thread that waits on a device flag nothing sets, giving up
 * after timeout_ns of %globaltimer time, and reports what happened:
 * *status = HICR_ERR_TIMEOUT when the wait gave up (expected), HICR_OK if the
 * flag was seen; *waited_ns = device time spent waiting. Synchronous.
 * Errors: INVALID, DEVICE. */
hicr_status hicr_util_wait_test(hicr_instance_t inst, uint64_t timeout_ns, hicr_status* status,
                                uint64_t* waited_ns);

/* Bandwidth probes: the bounds that channel and host-space measurements are
 * read against. Both run `ctas` CTAs of 256 threads (1 .. 8 per SM of the
 * device in all; the scheduler spreads them over the SMs) on the
 * communication stream, each thread with eight 16-byte accesses in flight,
 * loads at L2 (bypassing L1), and return the device time (CUDA events) in
 * *device_ns. Synchronous. Ranges are 16-byte aligned with
 * n a multiple of 16; slots of either memory space (host slots through
 * their device-visible address).
 *  - hicr_util_copy_loop: `reps` passes copying n bytes from src to dst
 *    (2 n bytes moved per pass); a range small enough to stay in L2 (e.g. 8
 *    MiB each way) gives the L2 copy rate;
 *  - hicr_util_stream: `reps` passes reading (write == 0) or writing
 *    (write != 0) n bytes; on a host slot, the link's one-way rate.
 * Errors: INVALID (bad slot, alignment, reps or ctas), BOUNDS,
 * OVERLAP (copy ranges of one slot intersect), DEVICE. */
hicr_status hicr_util_copy_loop(hicr_instance_t inst, hicr_slot_t dst, uint64_t dst_off, hicr_slot_t src,
                                uint64_t src_off, uint64_t n, uint32_t reps, uint32_t ctas, uint64_t* device_ns);
hicr_status hicr_util_stream(hicr_instance_t inst, hicr_slot_t slot, uint64_t off, uint64_t n, int32_t write,
                             uint32_t reps, uint32_t ctas, uint64_t* device_ns);

#ifdef __cplusplus
}
#endif

#endif /* HICR_UTIL_H */
