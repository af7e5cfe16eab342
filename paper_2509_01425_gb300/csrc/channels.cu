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
#include "channel_host.h"

namespace hicr {


// ---------------------------------------------------------------------------
// Host-call kernels (one CTA, result in the mailbox).
// ---------------------------------------------------------------------------

__global__ void k_spsc_push_host(SpscView v, const uint8_t* src, unsigned long long k, Mailbox* mb) {
  __shared__ unsigned long long s_head;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned long long h = ld_rlx(&v.st->head.v), t = ld_acq(&v.st->tail.v);
    s_ok = (h - t + k <= v.cap);
    s_head = h;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) mb_post(mb, HICR_ERR_FULL);
    return;
  }
  // at most two contiguous runs: up to the ring end, then from its start
  const unsigned long long first = s_head % v.cap;
  const unsigned long long run1 = min(k, (unsigned long long)v.cap - first);
  cta_copy(v.ring + first * v.ts, src, run1 * v.ts);
  if (k > run1) cta_copy(v.ring, src + run1 * v.ts, (k - run1) * v.ts);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    st_rel(&v.st->head.v, s_head + k);
    mb->v[0] = s_head;
    mb_post(mb, HICR_OK);
  }
}

// op 0 = peek(k), 1 = pop(k), 2 = depth
__global__ void k_spsc_ctl(SpscView v, int op, unsigned long long k, Mailbox* mb) {
  const unsigned long long h = ld_acq(&v.st->head.v), t = ld_acq(&v.st->tail.v);
  const unsigned long long depth = h - t;
  if (op == 2) {
    mb->v[0] = depth;
    mb->v[1] = depth * v.ts;
    mb_post(mb, HICR_OK);
  } else if (op == 0) {
    if (k >= depth) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    mb->v[0] = ((t + k) % v.cap) * v.ts;
    mb->v[1] = v.ts;
    mb->v[2] = 0;
    mb->v[3] = t + k;
    mb_post(mb, HICR_OK);
  } else {
    if (k > depth) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    st_rel(&v.st->tail.v, t + k);
    mb_post(mb, HICR_OK);
  }
}

__global__ void k_mpsc_push_host(MpscView v, unsigned int producer, unsigned int seq, const uint8_t* src,
                                 unsigned long long n, Mailbox* mb) {
  __shared__ unsigned long long s_start, s_ticket;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned long long r = round16(n);
    int ok = 0;
    for (int attempt = 0; attempt < 1000; ++attempt) {
      const unsigned long long W = ld_rlx(&v.st->reserve.v);
      unsigned long long start;
      const unsigned long long end = mpsc_place(W, &r, 1, v.R, &start);
      const unsigned long long freed = ld_acq(&v.st->freed.v);
      const unsigned long long mt = ld_acq(&v.st->msg_tail.v);
      const unsigned long long t0 = W >> 40;
      const unsigned long long inflight = (end - freed) & MASK40;
      const unsigned long long msgs = ((t0 + 1) - mt) & MASK24;
      if (inflight > v.R || msgs > v.M) break;  // FULL under the placement rule
      const unsigned long long nw = (((t0 + 1) & MASK24) << 40) | end;
      if (atomicCAS(&v.st->reserve.v, W, nw) == W) {
        ok = 1;
        s_start = start;
        s_ticket = t0;
        atomicMax(&v.st->max_bytes.v, inflight);
        atomicMax(&v.st->max_msgs.v, msgs);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) mb_post(mb, HICR_ERR_FULL);
    return;
  }
  cta_copy(v.ring + (s_start & (v.R - 1)), src, n);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    MpscMeta* e = v.meta + (s_ticket & (v.M - 1));
    e->start = s_start;
    e->size = (unsigned int)n;
    e->producer = producer;
    e->seq = seq;
    e->flags = 0;
    st_rel(&e->ready, (s_ticket & MASK24) + 1);
    mb->v[0] = s_start & (v.R - 1);
    mb->v[1] = s_ticket;
    mb_post(mb, HICR_OK);
  }
}

// op 0 = peek(k), 1 = pop(k), 2 = depth
__global__ void k_mpsc_ctl(MpscView v, int op, unsigned long long k, Mailbox* mb) {
  const unsigned long long W = ld_acq(&v.st->reserve.v);
  const unsigned long long mt = ld_acq(&v.st->msg_tail.v);
  const unsigned long long freed = ld_acq(&v.st->freed.v);
  const unsigned long long depth = ((W >> 40) - mt) & MASK24;
  if (op == 2) {
    mb->v[0] = depth;
    mb->v[1] = ((W & MASK40) - freed) & MASK40;
    mb_post(mb, HICR_OK);
    return;
  }
  if (op == 0) {
    if (k >= depth) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    const unsigned long long t = mt + k;
    MpscMeta* e = v.meta + (t & (v.M - 1));
    if (ld_acq(&e->ready) != (t & MASK24) + 1) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
    mb->v[0] = __ldcg(&e->start) & (v.R - 1);
    mb->v[1] = __ldcg(&e->size);
    mb->v[2] = __ldcg(&e->producer);
    mb->v[3] = __ldcg(&e->seq);
    mb_post(mb, HICR_OK);
    return;
  }
  if (k > depth) {
    mb_post(mb, HICR_ERR_EMPTY);
    return;
  }
  if (k == 0) {
    mb_post(mb, HICR_OK);
    return;
  }
  for (unsigned long long i = 0; i < k; ++i) {
    const unsigned long long t = mt + i;
    if (ld_acq(&v.meta[t & (v.M - 1)].ready) != (t & MASK24) + 1) {
      mb_post(mb, HICR_ERR_EMPTY);
      return;
    }
  }
  const MpscMeta* last = v.meta + ((mt + k - 1) & (v.M - 1));
  const unsigned long long end = (__ldcg(&last->start) + round16(__ldcg(&last->size))) & MASK40;
  st_rel(&v.st->freed.v, end);
  st_rel(&v.st->msg_tail.v, mt + k);
  mb_post(mb, HICR_OK);
}

__global__ void k_nl_push_host(NlView v, unsigned int producer, unsigned int seq, const uint8_t* src,
                               unsigned long long n, Mailbox* mb) {
  __shared__ unsigned long long s_start, s_pub;
  __shared__ int s_ok;
  NlState* st = v.st + producer;
  if (threadIdx.x == 0) {
    const unsigned long long r = round16(n);
    unsigned long long start;
    const unsigned long long end = nl_place(ld_rlx(&st->reserve.v), &r, 1, v.R, &start);
    const unsigned long long pub = ld_rlx(&st->pub.v);
    const unsigned long long freed = ld_acq(&st->freed.v), cons = ld_acq(&st->cons.v);
    s_ok = end - freed <= v.R && pub + 1 - cons <= v.M;
    s_start = start;
    s_pub = pub;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) mb_post(mb, HICR_ERR_FULL);
    return;
  }
  uint8_t* ring = v.ring + (unsigned long long)producer * v.R;
  cta_copy(ring + (s_start & (v.R - 1)), src, n);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    NlMeta* e = v.meta + (unsigned long long)producer * v.M + (s_pub & (v.M - 1));
    e->start = s_start;
    e->size = (unsigned int)n;
    e->seq = seq;
    st_rel(&st->reserve.v, s_start + round16(n));
    __threadfence();
    st_rel(&st->pub.v, s_pub + 1);
    mb->v[0] = s_start & (v.R - 1);
    mb->v[1] = s_pub;
    mb_post(mb, HICR_OK);
  }
}

// op 0 = peek(k), 1 = pop(k), 2 = depth; the consumer order is "producers in
// index order, each producer's messages oldest first". One thread.
__global__ void k_nl_ctl(NlView v, int op, unsigned long long k, Mailbox* mb) {
  unsigned long long msgs = 0, bytes = 0;
  for (unsigned p = 0; p < v.P; ++p) {
    const NlState* st = v.st + p;
    msgs += ld_acq(&st->pub.v) - ld_acq(&st->cons.v);
    bytes += ld_acq(&st->reserve.v) - ld_acq(&st->freed.v);
  }
  if (op == 2) {
    mb->v[0] = msgs;
    mb->v[1] = bytes;
    mb_post(mb, HICR_OK);
    return;
  }
  if (op == 0 ? k >= msgs : k > msgs) {
    mb_post(mb, HICR_ERR_EMPTY);
    return;
  }
  unsigned long long left = k;
  for (unsigned p = 0; p < v.P; ++p) {
    NlState* st = v.st + p;
    const unsigned long long cons = ld_rlx(&st->cons.v);
    const unsigned long long d = ld_acq(&st->pub.v) - cons;
    const NlMeta* m = v.meta + (unsigned long long)p * v.M;
    if (op == 0) {
      if (left < d) {
        const NlMeta* e = m + ((cons + left) & (v.M - 1));
        mb->v[0] = __ldcg(&e->start) & (v.R - 1);
        mb->v[1] = __ldcg(&e->size);
        mb->v[2] = p;
        mb->v[3] = __ldcg(&e->seq);
        mb_post(mb, HICR_OK);
        return;
      }
      left -= d;
    } else {
      const unsigned long long take = left < d ? left : d;
      if (take) {
        const NlMeta* e = m + ((cons + take - 1) & (v.M - 1));
        st_rel(&st->freed.v, __ldcg(&e->start) + round16(__ldcg(&e->size)));
        st_rel(&st->cons.v, cons + take);
        left -= take;
      }
      if (!left) break;
    }
  }
  mb_post(mb, HICR_OK);
}

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
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  hicr_slot_deregister(h, c->ring_slot);
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
  if ((st = lat_drain(in)) != HICR_OK) return st;
  if ((st = mailbox(in, &mh, &md)) != HICR_OK) return st;
  if (c->kind == 0) {
    if (producer != 0) return HICR_ERR_INVALID;
    if (n > (1ull << 40) / c->token_size) return HICR_ERR_FULL;
    const uint64_t bytes = n * c->token_size;
    if (off > ssize || bytes > ssize - off) return HICR_ERR_BOUNDS;
    if (n > c->capacity) return HICR_ERR_FULL;
    k_spsc_push_host<<<1, 256, 0, in->comm()>>>(spsc_view(c), (const uint8_t*)sp + off, n, md);
    st = finish(in, mh);
  } else {
    if (producer >= c->n_producers) return HICR_ERR_INVALID;
    if (off > ssize || n > ssize - off) return HICR_ERR_BOUNDS;
    if (round16(n) > c->ring_bytes || n > 0xffffffffull) return HICR_ERR_TOO_LARGE;
    if (c->kind == 1)
      k_mpsc_push_host<<<1, 256, 0, in->comm()>>>(mpsc_view(c), producer, c->seq[producer],
                                                 (const uint8_t*)sp + off, n, md);
    else
      k_nl_push_host<<<1, 256, 0, in->comm()>>>(nl_view(c), producer, c->seq[producer], (const uint8_t*)sp + off, n,
                                               md);
    st = finish(in, mh);
    if (st == HICR_OK) c->seq[producer]++;
  }
  if (st == HICR_OK) st = record_done(in);
  return st;
}

static hicr_status ctl(Instance* in, Channel* c, int op, uint64_t k, Mailbox** out) {
  Mailbox *mh, *md;
  hicr_status st = mailbox(in, &mh, &md);
  if (st != HICR_OK) return st;
  if (c->kind == 0) k_spsc_ctl<<<1, 1, 0, in->comm()>>>(spsc_view(c), op, k, md);
  else if (c->kind == 1) k_mpsc_ctl<<<1, 1, 0, in->comm()>>>(mpsc_view(c), op, k, md);
  else k_nl_ctl<<<1, 1, 0, in->comm()>>>(nl_view(c), op, k, md);
  st = finish(in, mh);
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
