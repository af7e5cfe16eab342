// The channel host calls (push, peek, pop, depth; HiCR paper Sec. 4.3) as
// device functions. Two callers run them: the one-CTA kernels of
// channels.cu, launched per call on the communication stream, and the
// latency-mode server (latency.cu), which takes them from its ring in mapped
// host memory while it runs. A push is CTA-wide (every thread calls it); the
// other calls run on one thread. Each posts its status, and its results
// before it, to the caller's mailbox in mapped host memory.
#pragma once

#include "channel_common.cuh"

namespace hicr {


__device__ inline void spsc_push_call(SpscView v, const uint8_t* src, unsigned long long k, Mailbox* mb) {
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
__device__ inline void spsc_ctl_call(SpscView v, int op, unsigned long long k, Mailbox* mb) {
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

__device__ inline void mpsc_push_call(MpscView v, unsigned int producer, unsigned int seq, const uint8_t* src,
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
__device__ inline void mpsc_ctl_call(MpscView v, int op, unsigned long long k, Mailbox* mb) {
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

__device__ inline void nl_push_call(NlView v, unsigned int producer, unsigned int seq, const uint8_t* src,
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
__device__ inline void nl_ctl_call(NlView v, int op, unsigned long long k, Mailbox* mb) {
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

// One channel call as the latency-mode server receives it.
struct ChanCall {
  unsigned int kind;      // 0 SPSC, 1 MPSC (locking), 2 MPSC (non-locking)
  int op;                 // -1 push; 0 peek, 1 pop, 2 depth
  unsigned int producer;  // push (MPSC): producer index and its next sequence number
  unsigned int seq;
  const uint8_t* src;     // push: the payload (device-usable address)
  unsigned long long k;   // push: tokens (SPSC) or bytes (MPSC); peek / pop: k
  Mailbox* mb;            // device address of the caller's mailbox
  union {
    SpscView s;
    MpscView m;
    NlView l;
  } v;
};

// Run call c. Every thread of the CTA calls this; the one-thread calls run on
// thread 0.
__device__ inline void chan_call(const ChanCall& c) {
  if (c.op < 0) {
    if (c.kind == 0) spsc_push_call(c.v.s, c.src, c.k, c.mb);
    else if (c.kind == 1) mpsc_push_call(c.v.m, c.producer, c.seq, c.src, c.k, c.mb);
    else nl_push_call(c.v.l, c.producer, c.seq, c.src, c.k, c.mb);
  } else if (threadIdx.x == 0) {
    if (c.kind == 0) spsc_ctl_call(c.v.s, c.op, c.k, c.mb);
    else if (c.kind == 1) mpsc_ctl_call(c.v.m, c.op, c.k, c.mb);
    else nl_ctl_call(c.v.l, c.op, c.k, c.mb);
  }
}

}  // namespace hicr
