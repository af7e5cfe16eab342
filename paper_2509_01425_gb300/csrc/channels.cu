// SPSC and MPSC channels (HiCR paper Sec. 4.3, Channels frontend).
//
// A channel is a circular buffer (ring) in HBM at the consumer plus 64-bit
// coordination counters, each on its own 128-byte line:
//   SPSC  head = tokens published, tail = tokens consumed;
//         token t lives at ring offset (t mod capacity) * token_size.
//   MPSC  reserve = (ticket mod 2^24) << 40 | (reserved bytes mod 2^40),
//         freed   = bytes freed (mod 2^40), msg_tail = messages freed,
//         plus a metadata ring of max_msgs entries {start, size, producer,
//         seq, ready}. The "locking" mode's exclusive access is one
//         compare-and-swap of `reserve`, taken only when the placement rule
//         (16-byte rounding, skip to the ring start instead of crossing its
//         end, reserved-minus-freed <= ring bytes, in-flight <= max_msgs)
//         finds room; a producer then copies its payload into the ring and
//         publishes the entry with a release store of `ready`. The consumer
//         drains tickets in order and frees with release stores.
//   MPSC non-locking (a dedicated ring per producer): producer i of the
//         channel owns ring i, its metadata ring and the counters reserve
//         (bytes reserved), pub (messages published) -- written only by the
//         producer -- and freed / cons, written only by the consumer. No
//         compare-and-swap: a producer places its messages with the same
//         rule in its own ring and publishes them with one release store of
//         pub; 64-bit absolute counters.
// Ring bytes and max_msgs are powers of two, so positions modulo 2^40 and
// tickets modulo 2^24 map consistently onto the rings.
//
// This file holds channel creation and the host calls (push, peek, pop,
// depth): each runs a one-CTA kernel that posts its result to a mapped host
// mailbox. The streaming runs are in streams.cu, the ping-pong in
// pingpong.cu.
#include <stddef.h>
#include <string.h>

#include <thread>
#include <vector>

#include "../../include/hicr_channels.h"
#include "channel_calls.cuh"
#include "channel_host.h"

namespace hicr {


// ---------------------------------------------------------------------------
// Host-call kernels (one CTA, result in the mailbox); the bodies are in
// channel_calls.cuh, which the latency-mode server shares.
// ---------------------------------------------------------------------------
__global__ void k_spsc_push_host(SpscView v, const uint8_t* src, unsigned long long k, Mailbox* mb) {
  spsc_push_call(v, src, k, mb);
}
__global__ void k_spsc_ctl(SpscView v, int op, unsigned long long k, Mailbox* mb) { spsc_ctl_call(v, op, k, mb); }
__global__ void k_mpsc_push_host(MpscView v, unsigned int producer, unsigned int seq, const uint8_t* src,
                                 unsigned long long n, Mailbox* mb) {
  mpsc_push_call(v, producer, seq, src, n, mb);
}
__global__ void k_mpsc_ctl(MpscView v, int op, unsigned long long k, Mailbox* mb) { mpsc_ctl_call(v, op, k, mb); }
__global__ void k_nl_push_host(NlView v, unsigned int producer, unsigned int seq, const uint8_t* src,
                               unsigned long long n, Mailbox* mb) {
  nl_push_call(v, producer, seq, src, n, mb);
}
__global__ void k_nl_ctl(NlView v, int op, unsigned long long k, Mailbox* mb) { nl_ctl_call(v, op, k, mb); }

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static hicr_status mailbox(Instance* in, Mailbox** host, Mailbox** dev) {
  if (!in->mbox_host) {
    void* p = nullptr;
    HICR_CUDA(in, cudaHostAlloc(&p, 4096, cudaHostAllocMapped));
    void* d = nullptr;
    HICR_CUDA(in, cudaHostGetDevicePointer(&d, p, 0));
    in->mbox_host = p;
    in->mbox_dev = d;
  }
  *host = (Mailbox*)in->mbox_host;
  *dev = (Mailbox*)in->mbox_dev;
  (*host)->status = 1;  // "not written"
  return HICR_OK;
}

static hicr_status finish(Instance* in, Mailbox* mh) {
  HICR_CUDA(in, cudaGetLastError());
  // The kernel posts its status last, behind a system-scope fence, so a
  // posted status means its work is visible. Poll the mapped word; query the
  // stream now and then, so a kernel that failed (status never posted) ends
  // the wait with its error.
  volatile int* st = &mh->status;
  for (uint64_t i = 0;; ++i) {
    if (*st != 1) return *st;
    if ((i & 255) == 255) {
      const cudaError_t e = cudaStreamQuery(in->comm());
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return cuda_fail(in, e, "host channel call");
      if (i > (1u << 20)) std::this_thread::yield();
    }
  }
  // the stream is idle: the status word is final
  if (*st == 1) return HICR_ERR_DEVICE;
  return *st;
}

static hicr_status add_channel(hicr_instance_t h, Channel* c, size_t ring_bytes, size_t state_bytes,
                               size_t meta_bytes, hicr_channel_t* out) {
  Instance* in = &h->impl;
  char* p = nullptr;
  const size_t ring_al = (ring_bytes + 255) & ~(size_t)255;
  const size_t st_al = (state_bytes + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(&p, ring_al + st_al + meta_bytes);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    delete c;
    return HICR_ERR_NOMEM;
  }
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(in, e, "cudaMalloc(channel)");
  }
  c->ring = (uint8_t*)p;
  c->state = p + ring_al;
  c->meta = meta_bytes ? (MpscMeta*)(p + ring_al + st_al) : nullptr;
  e = cudaMemsetAsync(p + ring_al, 0, st_al + meta_bytes, in->comm());
  if (e == cudaSuccess) e = cudaStreamSynchronize(in->comm());
  if (e != cudaSuccess) {
    cudaFree(p);
    delete c;
    return cuda_fail(in, e, "channel init");
  }
  hicr_slot_t rs;
  hicr_status st = hicr_slot_register(h, HICR_SPACE_HBM, p, ring_bytes, 0, &rs);
  if (st != HICR_OK) {
    cudaFree(p);
    delete c;
    return st;
  }
  c->ring_slot = rs;
  c->live = true;
  for (size_t i = 0; i < in->channels.size(); ++i) {
    if (!in->channels[i]) {
      in->channels[i] = c;
      *out = (hicr_channel_t)i;
      return HICR_OK;
    }
  }
  in->channels.push_back(c);
  *out = (hicr_channel_t)(in->channels.size() - 1);
  return HICR_OK;
}

void destroy_channels(Instance* in) {
  for (Channel* c : in->channels) {
    if (c) {
      if (c->ring) cudaFree(c->ring);
      delete c;
    }
  }
  in->channels.clear();
  if (in->mbox_host) cudaFreeHost(in->mbox_host);
  in->mbox_host = in->mbox_dev = nullptr;
  if (in->chan_buf) cudaFree(in->chan_buf);
  in->chan_buf = nullptr;
  in->chan_buf_cap = 0;
}

static bool pow2(unsigned long long x) { return x && !(x & (x - 1)); }

}  // namespace hicr

using namespace hicr;

extern "C" {

hicr_status hicr_spsc_create(hicr_instance_t h, uint32_t token_size, uint32_t capacity, hicr_channel_t* out) {
  Instance* in = I(h);
  if (!in || !out || token_size == 0 || capacity == 0 || in->capturing) return HICR_ERR_INVALID;
  if ((unsigned long long)token_size * capacity > (1ull << 40)) return HICR_ERR_INVALID;
  Channel* c = new Channel();
  c->kind = 0;
  c->token_size = token_size;
  c->capacity = capacity;
  c->seq.assign(1, 0);
  return add_channel(h, c, (size_t)token_size * capacity, sizeof(SpscState), 0, out);
}

hicr_status hicr_mpsc_create(hicr_instance_t h, uint32_t n_producers, uint64_t ring_bytes, uint32_t max_msgs,
                             hicr_channel_t* out) {
  Instance* in = I(h);
  if (!in || !out || n_producers == 0 || in->capturing) return HICR_ERR_INVALID;
  if (!pow2(ring_bytes) || ring_bytes < 64 || ring_bytes > (1ull << 39)) return HICR_ERR_INVALID;
  if (!pow2(max_msgs) || max_msgs > (1u << 23)) return HICR_ERR_INVALID;
  Channel* c = new Channel();
  c->kind = 1;
  c->n_producers = n_producers;
  c->ring_bytes = ring_bytes;
  c->max_msgs = max_msgs;
  c->seq.assign(n_producers, 0);
  return add_channel(h, c, ring_bytes, sizeof(MpscState), sizeof(MpscMeta) * (size_t)max_msgs, out);
}

hicr_status hicr_mpsc_nl_create(hicr_instance_t h, uint32_t n_producers, uint64_t ring_bytes, uint32_t max_msgs,
                                hicr_channel_t* out) {
  Instance* in = I(h);
  if (!in || !out || n_producers == 0 || in->capturing) return HICR_ERR_INVALID;
  if (!pow2(ring_bytes) || ring_bytes < 64 || ring_bytes > (1ull << 39)) return HICR_ERR_INVALID;
  if (!pow2(max_msgs) || max_msgs > (1u << 23)) return HICR_ERR_INVALID;
  if ((unsigned long long)n_producers * ring_bytes > (1ull << 40)) return HICR_ERR_INVALID;
  Channel* c = new Channel();
  c->kind = 2;
  c->n_producers = n_producers;
  c->ring_bytes = ring_bytes;
  c->max_msgs = max_msgs;
  c->seq.assign(n_producers, 0);
  return add_channel(h, c, (size_t)n_producers * ring_bytes, sizeof(NlHead) + sizeof(NlState) * (size_t)n_producers,
                     sizeof(NlMeta) * (size_t)max_msgs * n_producers, out);
}

hicr_status hicr_channel_device_view(hicr_instance_t h, hicr_channel_t ch, hicr_channel_view_t* out) {
  Instance* in = I(h);
  if (!in || !out) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  hicr_channel_view_t v;
  memset(&v, 0, sizeof(v));
  v.kind = (uint32_t)c->kind;
  v.ring = c->ring;
  if (c->kind == 0) {
    SpscState* st = (SpscState*)c->state;
    v.token_size = c->token_size;
    v.capacity = c->capacity;
    v.ring_bytes = (uint64_t)c->token_size * c->capacity;
    v.head = &st->head.v;
    v.tail = &st->tail.v;
  } else if (c->kind == 1) {
    MpscState* st = (MpscState*)c->state;
    v.max_msgs = c->max_msgs;
    v.ring_bytes = c->ring_bytes;
    v.head = &st->reserve.v;
    v.tail = &st->msg_tail.v;
    v.freed = &st->freed.v;
    v.meta = c->meta;
  } else {
    const NlView nv = nl_view(c);
    v.capacity = nv.P;
    v.max_msgs = nv.M;
    v.ring_bytes = nv.R;
    v.head = &nv.st->reserve.v;
    v.meta = nv.meta;
  }
  *out = v;
  return HICR_OK;
}

hicr_status hicr_channel_destroy(hicr_instance_t h, hicr_channel_t ch) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  // a latency-mode server may still hold calls on this channel: end it (it
  // completes what it took first), so the ring is idle when it is freed
  hicr_status st = hicr_flush(h);
  if (st == HICR_OK) st = lat_stop(in);
  if (st != HICR_OK) return st;
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  if ((st = hicr_slot_deregister(h, c->ring_slot)) != HICR_OK) return st;
  cudaFree(c->ring);
  delete c;
  in->channels[ch] = nullptr;
  return HICR_OK;
}

hicr_status hicr_channel_ring(hicr_instance_t h, hicr_channel_t ch, hicr_slot_t* ring_slot) {
  Instance* in = I(h);
  if (!in || !ring_slot) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  *ring_slot = c->ring_slot;
  return HICR_OK;
}

hicr_status hicr_channel_push(hicr_instance_t h, hicr_channel_t ch, uint32_t producer, hicr_slot_t src,
                              uint64_t off, uint64_t n) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  void* sp = nullptr;
  uint64_t ssize = 0;
  uint32_t sspace = 0;
  if (hicr_slot_info(h, src, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  Mailbox *mh, *md;
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  if (c->kind == 0) {
    if (producer != 0) return HICR_ERR_INVALID;
    if (n > (1ull << 40) / c->token_size) return HICR_ERR_FULL;
    const uint64_t bytes = n * c->token_size;
    if (off > ssize || bytes > ssize - off) return HICR_ERR_BOUNDS;
    if (n > c->capacity) return HICR_ERR_FULL;
  } else {
    if (producer >= c->n_producers) return HICR_ERR_INVALID;
    if (off > ssize || n > ssize - off) return HICR_ERR_BOUNDS;
    if (round16(n) > c->ring_bytes || n > 0xffffffffull) return HICR_ERR_TOO_LARGE;
  }
  // latency mode: the running server takes the call (after the copies
  // published to it before); otherwise a one-CTA launch on the
  // communication stream, after the server's copies have drained
  const bool served = lat_takes_calls(in);
  if (!served && (st = lat_drain(in)) != HICR_OK) return st;
  if ((st = mailbox(in, &mh, &md)) != HICR_OK) return st;
  const uint8_t* src_p = (const uint8_t*)sp + off;
  const unsigned seq = c->kind == 0 ? 0u : c->seq[producer];
  if (served) {
    ChanCall cc{};
    cc.kind = (unsigned)c->kind;
    cc.op = -1;
    cc.producer = producer;
    cc.seq = seq;
    cc.src = src_p;
    cc.k = n;
    cc.mb = md;
    if (c->kind == 0) cc.v.s = spsc_view(c);
    else if (c->kind == 1) cc.v.m = mpsc_view(c);
    else cc.v.l = nl_view(c);
    st = lat_channel_call(in, cc, &mh->status);
  } else {
    if (c->kind == 0) k_spsc_push_host<<<1, 256, 0, in->comm()>>>(spsc_view(c), src_p, n, md);
    else if (c->kind == 1) k_mpsc_push_host<<<1, 256, 0, in->comm()>>>(mpsc_view(c), producer, seq, src_p, n, md);
    else k_nl_push_host<<<1, 256, 0, in->comm()>>>(nl_view(c), producer, seq, src_p, n, md);
    st = finish(in, mh);
    if (st == HICR_OK) st = record_done(in);
  }
  if (st == HICR_OK && c->kind != 0) c->seq[producer]++;
  return st;
}

static hicr_status ctl(Instance* in, Channel* c, int op, uint64_t k, Mailbox** out) {
  Mailbox *mh, *md;
  const bool served = lat_takes_calls(in);
  hicr_status st;
  if (!served && (st = lat_drain(in)) != HICR_OK) return st;
  if ((st = mailbox(in, &mh, &md)) != HICR_OK) return st;
  if (served) {
    ChanCall cc{};
    cc.kind = (unsigned)c->kind;
    cc.op = op;
    cc.k = k;
    cc.mb = md;
    if (c->kind == 0) cc.v.s = spsc_view(c);
    else if (c->kind == 1) cc.v.m = mpsc_view(c);
    else cc.v.l = nl_view(c);
    st = lat_channel_call(in, cc, &mh->status);
  } else {
    if (c->kind == 0) k_spsc_ctl<<<1, 1, 0, in->comm()>>>(spsc_view(c), op, k, md);
    else if (c->kind == 1) k_mpsc_ctl<<<1, 1, 0, in->comm()>>>(mpsc_view(c), op, k, md);
    else k_nl_ctl<<<1, 1, 0, in->comm()>>>(nl_view(c), op, k, md);
    st = finish(in, mh);
  }
  *out = mh;
  return st;
}

hicr_status hicr_channel_peek(hicr_instance_t h, hicr_channel_t ch, uint64_t k, hicr_msg_info_t* out) {
  Instance* in = I(h);
  if (!in || !out || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  Mailbox* mb = nullptr;
  hicr_status st = ctl(in, c, 0, k, &mb);
  if (st != HICR_OK) return st;
  out->offset = mb->v[0];
  out->size = mb->v[1];
  out->producer = (uint32_t)mb->v[2];
  out->reserved = 0;
  out->seq = mb->v[3];
  return HICR_OK;
}

hicr_status hicr_channel_pop(hicr_instance_t h, hicr_channel_t ch, uint64_t count) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  Mailbox* mb = nullptr;
  return ctl(in, c, 1, count, &mb);
}

hicr_status hicr_channel_depth(hicr_instance_t h, hicr_channel_t ch, uint64_t* msgs, uint64_t* bytes) {
  Instance* in = I(h);
  if (!in || in->capturing) return HICR_ERR_INVALID;
  Channel* c = get(in, ch);
  if (!c) return HICR_ERR_INVALID;
  Mailbox* mb = nullptr;
  hicr_status st = ctl(in, c, 2, 0, &mb);
  if (st != HICR_OK) return st;
  if (msgs) *msgs = mb->v[0];
  if (bytes) *bytes = mb->v[1];
  return HICR_OK;
}

}  // extern "C"
