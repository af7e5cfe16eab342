/*
 * hicr_channels.h -- SPSC and MPSC channels of libhicr_gb300.so.
 *
 * HiCR paper Sec. 4.3 (Built-in Frontends, Channels): a channel is a
 * pre-allocated circular buffer at the consumer; a producer pushes while it is
 * not full and otherwise waits until the consumer reports consumption.
 * Single-producer/single-consumer (SPSC) channels carry fixed-size tokens;
 * multiple-producer/single-consumer (MPSC) channels in "locking" mode share one
 * buffer that an exclusive access keeps from overflowing.
 *
 * Here the buffer (ring), its head/tail counters and the MPSC metadata live in
 * HBM and are updated with release/acquire atomics, so producers and
 * consumers can be device threads. The host calls below run one small kernel
 * each and return when it has finished (synchronous, non-blocking semantics:
 * FULL / EMPTY instead of waiting).
 *
 * Conventions as in hicr.h.
 */
#ifndef HICR_CHANNELS_H
#define HICR_CHANNELS_H

#include <stdint.h>

#include "hicr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef uint32_t hicr_channel_t;

/* Description of one buffered message (peek). */
typedef struct {
  uint64_t offset;   /* byte offset of the payload in the channel ring */
  uint64_t size;     /* payload bytes */
  uint32_t producer; /* producer index (0 for SPSC) */
  uint32_t reserved;
  uint64_t seq;      /* per-producer sequence number (SPSC: token index) */
} hicr_msg_info_t;

/* SPSC channel of `capacity` tokens of `token_size` bytes (both >= 1,
 * capacity * token_size <= 2^40). head and tail are 64-bit monotonic token
 * counts; token t sits at ring offset (t mod capacity) * token_size.
 * Errors: INVALID, NOMEM, DEVICE. */
hicr_status hicr_spsc_create(hicr_instance_t inst, uint32_t token_size, uint32_t capacity,
                             hicr_channel_t* out);

/* MPSC channel (locking-mode semantics) with `n_producers` producers, a
 * payload ring of `ring_bytes` (a power of two, 64 B .. 2^39) and at most
 * `max_msgs` (a power of two, 1 .. 2^23) messages in flight.
 * Placement rule: each message reserves its size rounded up to 16 bytes; a
 * message that would cross the ring end skips to the ring start and the
 * skipped bytes count as reserved; reservations happen in ticket order and the
 * consumer frees in that order. A push succeeds only if reserved-but-unfreed
 * bytes stay <= ring_bytes and in-flight messages <= max_msgs.
 * Errors: INVALID (not powers of two, zero producers), NOMEM, DEVICE. */
hicr_status hicr_mpsc_create(hicr_instance_t inst, uint32_t n_producers, uint64_t ring_bytes,
                             uint32_t max_msgs, hicr_channel_t* out);

/* MPSC channel in non-locking mode (Sec. 4.3: a dedicated buffer per
 * producer, no collective exclusive access, more memory): `n_producers`
 * rings of `ring_bytes` each (power of two) with `max_msgs` metadata entries
 * each (power of two, 1 .. 2^23), ring_bytes 64 B .. 2^39 and n_producers
 * * ring_bytes <= 2^40. Ring p starts at byte p * ring_bytes of the channel's
 * ring slot and follows the placement rule of the locking mode on its own.
 * Host pops and peeks see the consumer order "producers in index order, each
 * producer's messages oldest first"; peek reports offsets within the
 * producer's ring. Device consumers poll the rings (hicr_mpsc_nl_stream).
 * Errors: INVALID, NOMEM, DEVICE. */
hicr_status hicr_mpsc_nl_create(hicr_instance_t inst, uint32_t n_producers, uint64_t ring_bytes,
                                uint32_t max_msgs, hicr_channel_t* out);

/* Free a channel's device memory. Errors: INVALID. */
hicr_status hicr_channel_destroy(hicr_instance_t inst, hicr_channel_t ch);

/* The channel ring as a (library-owned) HBM memory slot, so a consumer can
 * copy payloads out with hicr_memcpy using the offsets peek reports.
 * Errors: INVALID. */
hicr_status hicr_channel_ring(hicr_instance_t inst, hicr_channel_t ch, hicr_slot_t* ring_slot);

/* Push from slot `src` at byte `off`:
 *  SPSC: `n` tokens (n * token_size bytes), all or nothing; FULL when fewer
 *        than n tokens are free. `producer` must be 0.
 *  MPSC: one message of `n` bytes from producer `producer`; FULL when the
 *        placement rule finds no room (non-locking: in the producer's own
 *        ring), TOO_LARGE when the rounded size exceeds the ring.
 * Errors: INVALID (bad channel/producer/slot), BOUNDS (off + bytes > slot
 * size), UNSUPPORTED (source not in HBM), FULL, TOO_LARGE, DEVICE. */
hicr_status hicr_channel_push(hicr_instance_t inst, hicr_channel_t ch, uint32_t producer, hicr_slot_t src,
                              uint64_t off, uint64_t n);

/* Describe the k-th oldest unpopped message (k = 0 is the next to pop)
 * without changing state. EMPTY when k >= depth (for MPSC: or when that
 * message has been reserved but not yet published by a device producer). */
hicr_status hicr_channel_peek(hicr_instance_t inst, hicr_channel_t ch, uint64_t k, hicr_msg_info_t* out);

/* Consume the `count` oldest messages (SPSC: tokens), freeing their ring
 * space. All or nothing: EMPTY when fewer are buffered. */
hicr_status hicr_channel_pop(hicr_instance_t inst, hicr_channel_t ch, uint64_t count);

/* Messages (tokens) buffered and ring bytes held (MPSC: reserved, including
 * skipped bytes, minus freed). */
hicr_status hicr_channel_depth(hicr_instance_t inst, hicr_channel_t ch, uint64_t* msgs, uint64_t* bytes);

/* Device view of a channel for kernels that push or pop on the device
 * (the functions of hicr_device.cuh). Filled by hicr_channel_device_view,
 * passed to a kernel by value; valid until the channel is destroyed. */
typedef struct {
  uint32_t kind;             /* 0 SPSC, 1 MPSC (locking mode), 2 MPSC (non-locking mode) */
  uint32_t token_size;       /* SPSC token bytes */
  uint32_t capacity;         /* SPSC tokens; non-locking: number of producer rings */
  uint32_t max_msgs;         /* MPSC metadata entries (power of two; non-locking: per ring) */
  uint64_t ring_bytes;       /* ring size in bytes (non-locking: per ring; ring p at ring + p * ring_bytes) */
  uint8_t* ring;             /* the ring (the channel's ring slot) */
  unsigned long long* head;  /* SPSC: tokens published; MPSC: reserve word; non-locking: the
                                counter blocks, HICR_NL_STATE_WORDS words per producer ring */
  unsigned long long* tail;  /* SPSC: tokens consumed; MPSC: messages freed (NULL for non-locking) */
  unsigned long long* freed; /* MPSC: ring bytes freed (NULL for SPSC and non-locking) */
  void* meta;                /* MPSC: metadata ring of hicr_mpsc_meta_t; non-locking: max_msgs
                                hicr_nl_meta_t per ring, ring p's at meta + p * max_msgs */
} hicr_channel_view_t;

/* Non-locking counter block of producer ring p: head + p * HICR_NL_STATE_WORDS,
 * with the bytes reserved and the messages published (written by the
 * producer) and the bytes freed and messages consumed (written by the
 * consumer) at these word offsets, each on its own 128-byte line. */
#define HICR_NL_STATE_WORDS 64u
#define HICR_NL_RESERVE 0u
#define HICR_NL_PUB 16u
#define HICR_NL_FREED 32u
#define HICR_NL_CONS 48u

/* One non-locking metadata entry: absolute reservation start, size and
 * sequence number (the producer is the ring's index). */
typedef struct {
  unsigned long long start;
  uint32_t size;
  uint32_t seq;
} hicr_nl_meta_t;

/* One MPSC metadata entry (the library's layout). `ready` holds
 * (ticket mod 2^24) + 1 once the message of that ticket is published. */
typedef struct {
  unsigned long long start; /* absolute reservation start (mod 2^40) */
  uint32_t size;
  uint32_t producer;
  uint32_t seq;
  uint32_t flags;
  unsigned long long ready;
} hicr_mpsc_meta_t;

/* Fill *out with the device view of an SPSC, MPSC (locking) or MPSC
 * (non-locking) channel. Errors: INVALID (unknown channel). */
hicr_status hicr_channel_device_view(hicr_instance_t inst, hicr_channel_t ch, hicr_channel_view_t* out);

/* ------------------------------------------------------------------------ */
/* Device-driven streaming (producers and consumers are device threads).     */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t pushed;        /* tokens the producer published */
  uint64_t popped;        /* tokens the consumer consumed */
  uint64_t mismatches;    /* consumed 8-byte words that differ from the payload rule */
  uint64_t digest;        /* sum_j w_j * (2j + 1) mod 2^64 over the consumed word stream */
  uint64_t max_occupancy; /* largest head - tail a push had to respect (<= capacity) */
  int32_t status;         /* HICR_OK or HICR_ERR_TIMEOUT */
  uint32_t reserved;
} hicr_spsc_result_t;

/* Stream `tokens` tokens through each of the `n` SPSC channels `chans`
 * (token_size a multiple of 16, all starting empty) with one producer CTA and
 * one consumer CTA per channel, launched together as one cooperative grid so
 * both sides are resident at once. Word w of token s on the i-th channel of
 * the call is the SplitMix64 first output for state i * 2^40 + s *
 * (token_size / 8) + w. The producer publishes `batch` tokens per head update
 * (1 .. capacity); the consumer checks every word, accumulates the digest and
 * releases the tail per batch. Every wait gives up after `timeout_ns`
 * (result status TIMEOUT). Synchronous; `results` is a host array of n.
 * Both CTAs of every channel must be resident at once: one CTA of 512
 * threads fits an SM (about 128 registers a thread), so n is at most half
 * the SM count (76 on a GB300).
 * Errors: INVALID (bad channel, token size, batch, empty list, more channels
 * than can be resident), DEVICE, TIMEOUT (any channel timed out; the results
 * say which). */
hicr_status hicr_spsc_stream(hicr_instance_t inst, const hicr_channel_t* chans, uint32_t n, uint64_t tokens,
                             uint32_t batch, uint64_t timeout_ns, hicr_spsc_result_t* results);

/* Options of hicr_spsc_stream_ex. */
typedef struct {
  hicr_slot_t src;         /* HBM slot the producers copy tokens from (when src_tokens > 0) */
  uint32_t flags;          /* HICR_SPSC_DIGEST_ONLY, or 0 */
  uint64_t src_off;        /* byte offset in src of channel 0's staged tokens (16-byte aligned address) */
  uint64_t src_tokens;     /* tokens staged per channel: channel i's at src_off + i * src_tokens *
                              token_size; 0 = the producers write the payload rule instead */
  void* d_capture;         /* device buffer (16-byte aligned), or NULL: token s consumed from the
                              i-th channel of the call is stored at d_capture + i * capture_stride +
                              s * token_size */
  uint64_t capture_stride; /* multiple of 16, >= tokens * token_size */
} hicr_spsc_stream_opts_t;

/* With producers that write the payload rule: the consumer does not check the
 * words against the rule (mismatches is 0) and only digests the consumed
 * stream, as with copy producers. */
#define HICR_SPSC_DIGEST_ONLY 1u

/* hicr_spsc_stream with two more forms, chosen by `opts`:
 *  - copy producers (src_tokens > 0): a push is what Sec. 4.3 makes it, a
 *    copy from a memory slot into the consumer's ring; token s of the i-th
 *    channel is token (s mod src_tokens) of that channel's staged tokens. The
 *    consumer does not check words against the payload rule (mismatches is
 *    0); it digests the consumed stream as always;
 *  - capture (d_capture != NULL): the consumer also stores every token it
 *    consumed, in consumption order, so that a caller can compare the
 *    delivered stream token by token (tests; it adds a write per token);
 *  - digest only (flags HICR_SPSC_DIGEST_ONLY, payload-rule producers): the
 *    consumer skips the per-word check, so the run measures the channel
 *    rather than the check; its digest still identifies the stream.
 * All channels must have the same token size when either form is used.
 * Errors: as hicr_spsc_stream, plus INVALID (NULL opts, unknown flags, unaligned
 * or short capture area, unaligned staged tokens), UNSUPPORTED (src not in HBM), BOUNDS
 * (staged tokens outside src). */
hicr_status hicr_spsc_stream_ex(hicr_instance_t inst, const hicr_channel_t* chans, uint32_t n, uint64_t tokens,
                                uint32_t batch, const hicr_spsc_stream_opts_t* opts, uint64_t timeout_ns,
                                hicr_spsc_result_t* results);

/* One consumed MPSC message, as the consumer logs it in ticket order. */
typedef struct {
  uint32_t producer;
  uint32_t seq;
  uint32_t size;
  uint32_t reserved;
  uint64_t offset;  /* ring offset */
  uint64_t digest;  /* word digest of the payload (last word zero-padded) */
} hicr_mpsc_log_t;

typedef struct {
  uint64_t consumed;           /* messages consumed */
  uint64_t bytes;              /* payload bytes consumed */
  uint64_t max_inflight_bytes; /* largest reserved-minus-freed bytes at a reservation (<= ring) */
  uint64_t max_inflight_msgs;  /* largest in-flight message count at a reservation */
  uint64_t windows;            /* consumer rounds (consumed / windows = mean window) */
  uint64_t room_waits;         /* producer polls that found no room */
  uint64_t cas_failures;       /* producer reservations lost to another producer */
  uint64_t consumer_ns[3];     /* consumer time in: waiting for/acquiring tickets, digesting, logging+freeing */
  int32_t status;              /* HICR_OK or HICR_ERR_TIMEOUT */
  uint32_t reserved;
} hicr_mpsc_result_t;

/* Stream messages from `n_producers` producers into `n_consumers` MPSC
 * channels `chans` (all empty, each created with at least
 * ceil(n_producers / n_consumers) producers); producer p feeds channel
 * p mod n_consumers and sends `msgs_per_producer` messages in order.
 * Message (p, s) has d_sizes[p * msgs_per_producer + s] bytes (device array,
 * u64) taken from slot `staging` at byte d_src_off[p * msgs_per_producer + s]
 * (device array, u64). Each producer is one warp and reserves up to `group`
 * consecutive messages (1 .. 8) per exclusive access. Consumer c runs on
 * `consumer_ctas` CTAs that claim successive windows of reserved tickets,
 * digest their windows' payloads side by side and free them strictly in
 * ticket order (a CTA frees its window once the previous one is freed); the
 * log entry of ticket t goes to d_log + c * log_stride + (t - t0), t0 the
 * channel's first ticket of the run (device array, at least as many entries
 * as the consumer receives), so logs are in ticket order.
 * One cooperative grid: the consumer CTAs plus producer CTAs of 512
 * threads; the producer warps are spread evenly over every CTA slot that the
 * consumer CTAs leave free on the device. Every wait gives up after
 * `timeout_ns`. Synchronous; `results` is a host array of n_consumers.
 * Errors: INVALID (also when the grid cannot be co-resident), BOUNDS (a
 * message outside the staging slot), TOO_LARGE (a message larger than half
 * its ring), DEVICE, TIMEOUT. */
hicr_status hicr_mpsc_stream(hicr_instance_t inst, const hicr_channel_t* chans, uint32_t n_consumers,
                             uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                             const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                             uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                             uint64_t log_stride, hicr_mpsc_result_t* results);

/* The streaming run of hicr_mpsc_stream for non-locking channels (created
 * with hicr_mpsc_nl_create with at least ceil(n_producers / n_consumers)
 * producers each). Producer p (one warp) uses ring p / n_consumers of channel
 * p mod n_consumers; it reserves up to `group` messages (rounded sizes
 * summing to at most half a ring) at a time in its own ring, copies them and
 * publishes them with one release store, without any shared reservation.
 * Consumer c runs on `consumer_ctas` CTAs whose warps each own a fixed
 * subset of the channel's rings (at most 32 per warp) and drain whichever of
 * them hold published messages. Logs are in consumption order (each
 * producer's messages in push order; the interleaving of producers is
 * arbitrary). Other arguments, results and errors as hicr_mpsc_stream
 * (cas_failures is 0). */
hicr_status hicr_mpsc_nl_stream(hicr_instance_t inst, const hicr_channel_t* chans, uint32_t n_consumers,
                                uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                uint64_t log_stride, hicr_mpsc_result_t* results);

/* Capture forms of the two streaming runs: the same run, and each consumer
 * also copies every message it consumed, before freeing its ring space, to
 * d_capture + d_cap_off[p * msgs_per_producer + s] (device buffer and device
 * array of u64 offsets chosen by the caller; message (p, s)'s bytes must fit
 * there), so that the delivered payloads can be compared byte by byte (tests;
 * each message is read once more). Errors: as the plain forms, plus INVALID
 * (NULL d_capture or d_cap_off). */
hicr_status hicr_mpsc_stream_capture(hicr_instance_t inst, const hicr_channel_t* chans, uint32_t n_consumers,
                                     uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                     const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                     uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                     uint64_t log_stride, hicr_mpsc_result_t* results, void* d_capture,
                                     const uint64_t* d_cap_off);
hicr_status hicr_mpsc_nl_stream_capture(hicr_instance_t inst, const hicr_channel_t* chans, uint32_t n_consumers,
                                        uint32_t n_producers, uint32_t msgs_per_producer, const uint64_t* d_sizes,
                                        const uint64_t* d_src_off, hicr_slot_t staging, uint32_t group,
                                        uint32_t consumer_ctas, uint64_t timeout_ns, hicr_mpsc_log_t* d_log,
                                        uint64_t log_stride, hicr_mpsc_result_t* results, void* d_capture,
                                        const uint64_t* d_cap_off);

/* ------------------------------------------------------------------------ */
/* Ping-pong over two opposing single-message SPSC channels (HiCR paper      */
/* Sec. 5.1, Test Case 1, restated for one GPU).                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t bytes;          /* message size */
  uint32_t reps;           /* timed round trips */
  uint32_t ctas_per_side;  /* CTAs of each agent */
  double half_rtt_ns;      /* device time of one direction (round trip / 2) */
  double goodput_gbs;      /* bytes / half_rtt, GB/s (the paper's G(s)) */
  uint64_t digest_a;       /* word digest of agent A's buffer after the run */
  uint64_t digest_b;       /* word digest of agent B's buffer after the run */
  int32_t status;          /* HICR_OK or HICR_ERR_TIMEOUT */
  uint32_t reserved;
} hicr_pingpong_result_t;

/* Agent A sends bytes [src_off, src_off+bytes) of slot `src` into agent B's
 * single-message buffer; B echoes the message into A's buffer; repeat. Each
 * buffer holds exactly one message at the consumer, so a sender never has
 * more than one message outstanding. Each agent is `ctas_per_side` CTAs (1 ..
 * 256, both agents co-resident) of one cooperative grid that copy equal
 * shares with vector loads and stores; when each agent has at most half the
 * SMs and every warp's share is at least 64 KiB, the CTAs run one per SM and
 * copy by bulk copies (TMA) through shared memory instead. A side's arrival
 * count is the channel head the other side acquires. `warmup` untimed round trips
 * come first. After the run both buffers must hold the message (the digests
 * let the caller check). Every wait gives up after timeout_ns.
 * Errors: INVALID, BOUNDS, NOMEM, DEVICE, TIMEOUT. */
hicr_status hicr_pingpong(hicr_instance_t inst, hicr_slot_t src, uint64_t src_off, uint64_t bytes, uint32_t reps,
                          uint32_t warmup, uint32_t ctas_per_side, uint64_t timeout_ns, hicr_pingpong_result_t* out);

/* hicr_pingpong, then both agents' buffers (`bytes` each) are copied to the
 * device buffers d_out_a and d_out_b, so that a caller can compare what each
 * agent last received byte by byte. Errors: as hicr_pingpong, plus INVALID
 * (a NULL output buffer). */
hicr_status hicr_pingpong_capture(hicr_instance_t inst, hicr_slot_t src, uint64_t src_off, uint64_t bytes,
                                  uint32_t reps, uint32_t warmup, uint32_t ctas_per_side, uint64_t timeout_ns,
                                  void* d_out_a, void* d_out_b, hicr_pingpong_result_t* out);

#ifdef __cplusplus
}
#endif

#endif /* HICR_CHANNELS_H */
