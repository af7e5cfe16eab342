// Continuous-batching request engine (see include/hicr_serve.h).
//
// Host side (hicr_serve_run, calling thread): arrivals -> FIFO admission under
// the arena budget (first-fit allocator) -> descriptor + doorbell in mapped
// host memory -> poll per-request completion words the device writes into
// mapped host memory -> free the region, record latency.
//
// Device side: one cooperative persistent kernel, all CTAs resident:
//   CTA 0, warp 0   dispatcher: acquires the doorbell, copies each new request
//                   into the per-request device table, gives it a contiguous range
//                   of work units (memcpy: one unit per cost chunk of its
//                   template, cut into enough chunks of SRV_MIN_UNIT to
//                   chunk_bytes to occupy the idle worker warps; burst: one
//                   unit per message group) and
//                   publishes units_pub;
//   CTAs 1..C       one MPSC consumer per channel (windowed drain as in the
//                   channel stream kernel); completes burst requests;
//   other CTAs      worker warps share the work of the requests in flight
//                   (shortest remaining first): each claim takes the next unit of the
//                   request with the fewest unclaimed units among the SRV_PS_WINDOW oldest
//                   published requests that still have unclaimed units, so a
//                   small request does not wait behind the units of a large
//                   one. A unit either
//                   copies one cost chunk of the template's ops (same warp copy
//                   and chunking as the batch path) or pushes one group of the burst's
//                   messages: group k reserves its tickets only after group
//                   k-1 has reserved (a per-request chain), so a burst's
//                   messages keep their order in the channel while the groups
//                   are copied side by side.
// Every wait is bounded by the run deadline (%globaltimer).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <thread>
#include <vector>

#include "../../include/hicr_serve.h"
#include "channel_common.cuh"
#include "copy.cuh"
#include "hicr_internal.h"

namespace hicr {

static constexpr unsigned SRV_THREADS = 512;
static constexpr unsigned SRV_MAX_CH = 64;
static constexpr int SRV_WIN = 64;
static constexpr int SRV_PIECE = 512;
// While worker warps are idle, a memcpy request is cut into enough work units
// to occupy them, of at least SRV_MIN_UNIT cost bytes (at most chunk_bytes).
static constexpr unsigned long long SRV_MIN_UNIT = 16ull << 10;

struct SrvReq {
  unsigned long long U;       // first unit
  unsigned long long id;      // request index
  unsigned long long dst;     // destination region base (memcpy)
  unsigned long long done;    // completed chunks / consumed messages
  unsigned long long digest;  // burst digest accumulator
  unsigned int N, need, kind, tmpl;
  unsigned int unit, pad;     // memcpy: cost bytes per work unit, chosen at dispatch
  unsigned long long gres;    // burst: message groups that have reserved their tickets (whole
                              // reservation: 1 once the burst's reservation is made)
  unsigned long long wbase;   // burst, whole reservation: the channel's reserve word before it
  unsigned long long claimed; // units handed out (may pass N by failed claims)
};

// A burst's messages are cut into groups of at most SRV_GROUP_MSGS
// consecutive messages whose rounded sizes sum to at most SRV_GROUP_BYTES
// (a larger message is a group of its own); one work unit per group.
static constexpr unsigned SRV_GROUP_MSGS = 2;
// Workers claim among at most this many of the oldest requests that may have
// unclaimed units, the one with the fewest unclaimed units first (under
// overload the requests behind the window wait in order; there the units
// are all chunk_bytes, so fewest units is least work).
static constexpr unsigned long long SRV_PS_WINDOW = 32;
static constexpr unsigned long long SRV_GROUP_BYTES = 32ull << 10;

struct SrvHostDesc {
  unsigned int kind, tmpl;
  unsigned long long dst;
};

struct SrvCtl {
  Line claim, units_pub, req_pub, stop, final_units, abort, bad, exited;
  Line lo;  // requests below lo have no unclaimed unit
  Line rr;  // round-robin ticket of the claims
  unsigned long long final_msgs[SRV_MAX_CH];
};

struct SrvArgs {
  SrvCtl* ctl;
  SrvReq* req;                          // per-request state, indexed by request id
  const SrvHostDesc* hdesc;             // mapped host memory
  const unsigned long long* hdoor;      // mapped: requests published
  const unsigned long long* hstop;      // mapped: no more requests
  unsigned long long* hcompl;           // mapped: completion time per request (0 = pending)
  unsigned long long* hdigest;          // mapped: burst digest per request
  const hicr_op_t* tops;
  const unsigned long long* tcstart;
  const unsigned long long* t_opbase;
  const unsigned long long* t_nops;
  const unsigned long long* t_cbase;
  const unsigned long long* t_total;
  const unsigned long long* msizes;
  const unsigned long long* moffs;
  const unsigned long long* t_mbase;
  const unsigned long long* t_nmsg;
  const unsigned long long* gstart;   // group starts (message index within the template), ng + 1 per template
  const unsigned long long* t_gbase;  // template's first entry in gstart
  const unsigned long long* t_ngrp;
  const unsigned long long* t_whole;  // burst template reserves all its messages at once (1) or by groups
  const uint8_t* staging;
  DevTables dt;
  const MpscView* chans;
  unsigned int n_ch;
  unsigned int chunk;
  unsigned int op_cost;
  unsigned long long timeout_ns;
  unsigned long long n_req;   // requests in this run
  unsigned int n_mt, n_bt;    // memcpy / burst templates
  unsigned long long arena_lo, arena_hi;
  unsigned int* wstate;       // per warp: where it is (diagnostics)
  // capture of consumed burst messages (tests and sampled checks): message m
  // of burst request r goes to cap + cap_off[r] + mcap[t_mbase[tmpl] + m]
  // unless cap_off[r] is ~0
  uint8_t* cap;
  const unsigned long long* cap_off;
  const unsigned long long* mcap;  // per template message: offset within the burst's captured bytes
};

// Warp states recorded in SrvArgs::wstate (diagnostics of a stuck run).
enum : unsigned {
  WS_CLAIM = 1, WS_COPY = 2, WS_RESERVE = 3, WS_PUSH = 4, WS_WORKER_DONE = 5,
  WS_C_AVAIL = 10, WS_C_READY = 11, WS_C_DIGEST = 12, WS_C_ACCOUNT = 13, WS_C_DONE = 14,
  WS_DISPATCH = 20, WS_DISPATCH_DONE = 21
};
__device__ __forceinline__ void ws_set(const SrvArgs& a, unsigned st) {
  if ((threadIdx.x & 31u) == 0) {
    const unsigned w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    *(volatile unsigned*)&a.wstate[w] = st;
  }
}

__device__ __forceinline__ unsigned long long ld_acq_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_rlx_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool srv_abort(const SrvArgs& a, unsigned long long deadline) {
  if (*(volatile unsigned long long*)&a.ctl->abort.v) return true;
  if (gtime() > deadline) {
    atomicExch(&a.ctl->abort.v, 1ull);
    return true;
  }
  return false;
}

// Request entries are written by the dispatcher while the kernel runs, so
// every read of one goes to L2 (ld.global.cg): an SM's L1 may still hold the
// line from before the entry was written.
struct ReqView {
  unsigned long long U, id, dst;
  unsigned int N, need, kind, tmpl, unit;
};
__device__ __forceinline__ ReqView load_req(const SrvReq* e) {
  ReqView r;
  r.U = __ldcg(&e->U);
  r.id = __ldcg(&e->id);
  r.dst = __ldcg(&e->dst);
  r.N = __ldcg(&e->N);
  r.need = __ldcg(&e->need);
  r.kind = __ldcg(&e->kind);
  r.tmpl = __ldcg(&e->tmpl);
  r.unit = __ldcg(&e->unit);
  return r;
}

// The request that finishes writes its completion into host memory.
__device__ __forceinline__ void srv_complete(const SrvArgs& a, SrvReq* e) {
  __threadfence();
  const unsigned long long id = __ldcg(&e->id);
  a.hdigest[id] = atomicAdd(&e->digest, 0ull);
  __threadfence_system();
  st_rel_sys(&a.hcompl[id], gtime() | 1ull);
}

__device__ void srv_dispatcher(const SrvArgs& a, unsigned long long deadline) {
  ws_set(a, WS_DISPATCH);
  unsigned long long r = 0, U = 0;
  const unsigned long long workers = (unsigned long long)(gridDim.x - 1 - a.n_ch) * (SRV_THREADS / 32);
  unsigned long long msgs[SRV_MAX_CH];
  for (unsigned c = 0; c < a.n_ch; ++c) msgs[c] = 0;
  unsigned sleep_ns = 64;
  for (;;) {
    const unsigned long long door = ld_acq_sys(a.hdoor);
    bool progressed = false;
    while (r < door) {
      SrvReq* e = a.req + r;
      const unsigned long long w0 = ld_rlx_sys(reinterpret_cast<const unsigned long long*>(a.hdesc + r));
      const unsigned long long dst = ld_rlx_sys(reinterpret_cast<const unsigned long long*>(a.hdesc + r) + 1);
      const unsigned kind = (unsigned)w0, t = (unsigned)(w0 >> 32);
      // A memcpy request's work unit: enough units to occupy the worker
      // warps that no published unit waits for, each between SRV_MIN_UNIT
      // and chunk_bytes of cost. One warp copies a unit, so on an idle engine
      // a request spreads over many warps and finishes in about one small
      // unit's copy; with every warp busy the units are chunk_bytes and the
      // claims as few as they can be.
      unsigned long long unit = a.chunk, N, need;
      if (kind == 0) {
        const unsigned long long total = a.t_total[t];
        const unsigned long long backlog = U - min(U, ld_rlx(&a.ctl->claim.v));
        const unsigned long long idle = workers > backlog ? workers - backlog : 0;
        const unsigned long long want = max(1ull, idle);
        unit = min((unsigned long long)a.chunk, max(SRV_MIN_UNIT, (total + want - 1) / want));
        N = need = (total + unit - 1) / unit;
      } else {
        N = a.t_ngrp[t];
        need = a.t_nmsg[t];
      }
      e->U = U;
      e->id = r;
      e->dst = dst;
      e->done = 0;
      e->digest = 0;
      e->gres = 0;
      e->claimed = 0;
      e->N = (unsigned)N;
      e->need = (unsigned)need;
      e->kind = kind;
      e->tmpl = t;
      e->unit = (unsigned)unit;
      if (kind == 1) msgs[r % a.n_ch] += need;
      if (need == 0) srv_complete(a, e);
      __threadfence();
      st_rel(&a.ctl->req_pub.v, r + 1);
      st_rel(&a.ctl->units_pub.v, U + N);
      U += N;
      ++r;
      progressed = true;
    }
    if (progressed) {
      sleep_ns = 64;
      continue;
    }
    if (ld_acq_sys(a.hstop) && ld_acq_sys(a.hdoor) == r) {
      for (unsigned c = 0; c < a.n_ch; ++c) a.ctl->final_msgs[c] = msgs[c];
      a.ctl->final_units.v = U;
      __threadfence();
      st_rel(&a.ctl->stop.v, 1ull);
      ws_set(a, WS_DISPATCH_DONE);
      return;
    }
    if (srv_abort(a, deadline)) {
      ws_set(a, WS_DISPATCH_DONE);
      return;
    }
    __nanosleep(sleep_ns);
    sleep_ns = min(sleep_ns * 2, 1024u);
  }
}

__device__ void srv_copy_chunk(const SrvArgs& a, SrvReq* e, const ReqView& rv, unsigned long long k, unsigned lane) {
  const unsigned t = rv.tmpl;
  const hicr_op_t* ops = a.tops + a.t_opbase[t];
  const unsigned long long nops = a.t_nops[t];
  const unsigned long long* cstart = a.tcstart + a.t_cbase[t];
  const unsigned long long chunk = rv.unit, total = a.t_total[t];
  const unsigned long long lo = k * chunk, hi = min(lo + chunk, total);
  const unsigned long long dst = rv.dst;
  for (unsigned long long i = find_op(cstart, nops, lo, lane); i < nops; ++i) {
    const unsigned long long cs = cstart[i];
    if (cs >= hi) break;
    const hicr_op_t op = ops[i];
    const unsigned long long bs = cs + a.op_cost, be = bs + op.n;
    const unsigned long long b0 = lo > bs ? lo - bs : 0ull;
    const unsigned long long cap = hi < be ? hi : be;
    const unsigned long long b1 = cap > bs ? cap - bs : 0ull;
    if (b1 > b0) {
      uint8_t* d = reinterpret_cast<uint8_t*>(dst) + op.dst_off + b0;
      const uint8_t* s = reinterpret_cast<const uint8_t*>(a.dt.slot_base[op.src]) + op.src_off + b0;
      warp_copy(d, s, b1 - b0, lane);
    }
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    const unsigned long long prev = atomicAdd(&e->done, 1ull);
    if (prev + 1 == rv.need) srv_complete(a, e);
  }
}

// Push group k of a burst (producer = request index). A burst that takes at
// most half the ring and half the message slots is reserved whole: group 0's
// lane 0 places all its messages (the channel's placement rule, from the
// current reserve word) and takes their tickets and ring bytes with one
// compare-and-swap; every group then replays the placement from that word to
// find its messages' positions, so the groups copy side by side. A larger
// burst reserves group by group: group k waits until group k-1 has reserved,
// reserves its own messages and passes the turn on. Then the warp copies the
// group's messages and publishes their metadata.
__device__ bool srv_push_group(const SrvArgs& a, SrvReq* e, const ReqView& rv, unsigned long long k, unsigned lane,
                               unsigned long long deadline) {
  const unsigned long long id = rv.id;
  const unsigned t = rv.tmpl;
  const MpscView v = a.chans[id % a.n_ch];
  const unsigned long long mbase = a.t_mbase[t];
  const unsigned long long* gs = a.gstart + a.t_gbase[t];
  const unsigned long long m0 = gs[k], m1 = gs[k + 1];
  const int cnt = (int)(m1 - m0);  // 1 .. SRV_GROUP_MSGS
  unsigned long long r[SRV_GROUP_MSGS], st[SRV_GROUP_MSGS];
  for (int i = 0; i < cnt; ++i) r[i] = round16(a.msizes[mbase + m0 + i]);
  unsigned long long W = 0;
  int stop = 0;
  ws_set(a, WS_RESERVE);
  if (a.t_whole[t]) {
    if (lane == 0) {
      const unsigned long long nmsg = a.t_nmsg[t];
      if (k == 0) {
        // place the whole burst and reserve it
        unsigned long long freed = ld_acq(&v.st->freed.v), mt = ld_acq(&v.st->msg_tail.v);
        unsigned sleep_ns = 32;
        for (;;) {
          W = ld_rlx(&v.st->reserve.v);
          unsigned long long b = W & MASK40;
          for (unsigned long long i = 0; i < nmsg; ++i) {
            const unsigned long long ri = round16(a.msizes[mbase + i]), pos = b & (v.R - 1);
            if (pos + ri > v.R) b = (b + (v.R - pos)) & MASK40;
            b = (b + ri) & MASK40;
          }
          const unsigned long long t0 = W >> 40;
          bool room = ((b - freed) & MASK40) <= v.R && (((t0 + nmsg) - mt) & MASK24) <= v.M;
          if (!room) {
            freed = ld_acq(&v.st->freed.v);
            mt = ld_acq(&v.st->msg_tail.v);
            room = ((b - freed) & MASK40) <= v.R && (((t0 + nmsg) - mt) & MASK24) <= v.M;
          }
          if (room && atomicCAS(&v.st->reserve.v, W, (((t0 + nmsg) & MASK24) << 40) | b) == W) break;
          if (srv_abort(a, deadline)) {
            stop = 1;
            break;
          }
          if (!room) {
            __nanosleep(sleep_ns);
            sleep_ns = min(sleep_ns * 2, 4096u);
          }
        }
        if (!stop) {
          e->wbase = W;
          st_rel(&e->gres, 1ull);
        }
      } else {
        unsigned sleep_ns = 32;
        while (ld_acq(&e->gres) == 0) {  // group 0 has not reserved yet
          if (srv_abort(a, deadline)) {
            stop = 1;
            break;
          }
          __nanosleep(sleep_ns);
          sleep_ns = min(sleep_ns * 2, 256u);
        }
        if (!stop) W = __ldcg(&e->wbase);
      }
      if (!stop) {
        // this group's positions: the placement replayed from the burst's word
        unsigned long long b = W & MASK40;
        for (unsigned long long i = 0; i < m1; ++i) {
          const unsigned long long ri = round16(a.msizes[mbase + i]), pos = b & (v.R - 1);
          if (pos + ri > v.R) b = (b + (v.R - pos)) & MASK40;
          if (i >= m0) st[i - m0] = b;
          b = (b + ri) & MASK40;
        }
        // the group's first ticket, in the form the copy below expects
        W = (((W >> 40) + m0) & MASK24) << 40;
      }
    }
  } else if (lane == 0) {
    unsigned sleep_ns = 32;
    while (ld_acq(&e->gres) != k) {  // the previous group's turn
      if (srv_abort(a, deadline)) {
        stop = 1;
        break;
      }
      __nanosleep(sleep_ns);
      sleep_ns = min(sleep_ns * 2, 256u);
    }
    unsigned long long freed = 0, mt = 0;
    bool fresh = false;
    sleep_ns = 32;
    while (!stop) {
      W = ld_rlx(&v.st->reserve.v);
      const unsigned long long end = mpsc_place(W, r, cnt, v.R, st);
      const unsigned long long t0 = W >> 40;
      if (!fresh) {
        freed = ld_acq(&v.st->freed.v);
        mt = ld_acq(&v.st->msg_tail.v);
        fresh = true;
      }
      bool room = ((end - freed) & MASK40) <= v.R && (((t0 + cnt) - mt) & MASK24) <= v.M;
      if (!room) {
        freed = ld_acq(&v.st->freed.v);
        mt = ld_acq(&v.st->msg_tail.v);
        room = ((end - freed) & MASK40) <= v.R && (((t0 + cnt) - mt) & MASK24) <= v.M;
      }
      if (room && atomicCAS(&v.st->reserve.v, W, (((t0 + cnt) & MASK24) << 40) | end) == W) break;
      if (srv_abort(a, deadline)) {
        stop = 1;
        break;
      }
      if (!room) {
        __nanosleep(sleep_ns);
        sleep_ns = min(sleep_ns * 2, 4096u);
      }
    }
    if (!stop) st_rel(&e->gres, k + 1);
  }
  if (__shfl_sync(FULLM, stop, 0)) return false;
  ws_set(a, WS_PUSH);
  W = __shfl_sync(FULLM, W, 0);
  const unsigned long long t0 = W >> 40;
  for (int i = 0; i < cnt; ++i) {
    const unsigned long long si = __shfl_sync(FULLM, st[i], 0);
    ring_copy(v.ring + (si & (v.R - 1)), a.staging + a.moffs[mbase + m0 + i], a.msizes[mbase + m0 + i], lane);
  }
  __threadfence();
  __syncwarp();
  for (int i = 0; i < cnt; ++i) {
    const unsigned long long si = __shfl_sync(FULLM, st[i], 0);
    if (lane == (unsigned)i) {
      const unsigned long long tk = t0 + i;
      MpscMeta* m = v.meta + (tk & (v.M - 1));
      m->start = si;
      m->size = (unsigned int)a.msizes[mbase + m0 + i];
      m->producer = (unsigned int)id;
      m->seq = (unsigned int)(m0 + i);
      m->flags = 0;
      st_rel(&m->ready, (tk & MASK24) + 1);
    }
  }
  return true;
}

// Claim one unit for the warp. Lane 0 reads the window [lo, hi) of published
// requests that may still have unclaimed units, moves lo past exhausted
// requests, and draws a round-robin start; the warp then scans the window from
// there, 32 requests per step (one lane each), and claims from the request
// with the fewest unclaimed units (ties: scan order), trying the next fewest
// when another warp took the last one. Returns 1 with (r, k) = (request, unit index),
// 0 when nothing is claimable right now, 2 when the run is over (every
// request published and claimed) or aborted. All lanes return the same value.
__device__ int srv_claim(const SrvArgs& a, unsigned lane, unsigned long long deadline, unsigned long long& r,
                         unsigned long long& k) {
  unsigned long long lo = 0, hi = 0, start = 0;
  int stop = 0;
  if (lane == 0) {
    if (srv_abort(a, deadline)) {
      stop = 2;
    } else {
      const bool stopping = ld_acq(&a.ctl->stop.v) != 0;  // before req_pub: then hi is final
      hi = ld_acq(&a.ctl->req_pub.v);
      lo = ld_rlx(&a.ctl->lo.v);  // only bounds the scan: a stale (smaller) value is safe
      // lo is read after hi, so other warps may have moved it past this hi
      if (lo > hi) lo = hi;
      for (int step = 0; step < 32 && lo < hi; ++step) {  // move lo past exhausted requests
        const SrvReq* e = a.req + lo;
        if (ld_rlx(&e->claimed) < __ldcg(&e->N)) break;
        atomicCAS(&a.ctl->lo.v, lo, lo + 1);
        lo = ld_rlx(&a.ctl->lo.v);
        if (lo > hi) lo = hi;
      }
      if (hi > lo + SRV_PS_WINDOW) hi = lo + SRV_PS_WINDOW;  // share among the oldest requests only
      if (lo < hi) start = atomicAdd(&a.ctl->rr.v, 1ull) % (hi - lo);
      else if (stopping) stop = 2;
    }
  }
  stop = __shfl_sync(FULLM, stop, 0);
  if (stop) return 2;
  lo = __shfl_sync(FULLM, lo, 0);
  hi = __shfl_sync(FULLM, hi, 0);
  start = __shfl_sync(FULLM, start, 0);
  const unsigned long long w = hi - lo;
  for (unsigned long long base = 0; base < w; base += 32) {
    const unsigned long long off = base + lane;
    unsigned long long cand = 0;
    bool open = false;
    unsigned left = 0xffffffffu;  // unclaimed units (capped), for the shortest-remaining choice
    if (off < w) {
      cand = lo + (start + off) % w;
      const unsigned long long c = ld_rlx(&a.req[cand].claimed), n = __ldcg(&a.req[cand].N);
      open = c < n;
      if (open) left = (unsigned)min(n - c, 0xfffffffeull);
    }
    unsigned m = __ballot_sync(FULLM, open);
    while (m) {
      // the open request with the fewest unclaimed units (ties: scan order)
      const unsigned best = __reduce_min_sync(FULLM, (m >> lane) & 1u ? left : 0xffffffffu);
      const unsigned L = __ffs(__ballot_sync(FULLM, ((m >> lane) & 1u) && left == best)) - 1;
      m &= ~(1u << L);
      const unsigned long long rc = __shfl_sync(FULLM, cand, L);
      unsigned long long kk = 0;
      int got = 0;
      if (lane == 0) {
        kk = atomicAdd(&a.req[rc].claimed, 1ull);
        got = kk < __ldcg(&a.req[rc].N);
        if (got) atomicAdd(&a.ctl->claim.v, 1ull);
      }
      if (__shfl_sync(FULLM, got, 0)) {
        r = rc;
        k = __shfl_sync(FULLM, kk, 0);
        return 1;
      }
    }
  }
  return 0;
}

__device__ void srv_worker(const SrvArgs& a, unsigned long long deadline) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned sleep_ns = 32;
  for (;;) {
    ws_set(a, WS_CLAIM);
    unsigned long long r = 0, k = 0;
    const int got = srv_claim(a, lane, deadline, r, k);
    if (got == 2) {
      ws_set(a, WS_WORKER_DONE);
      return;
    }
    if (got == 0) {
      if (lane == 0) __nanosleep(sleep_ns);
      __syncwarp();
      sleep_ns = min(sleep_ns * 2, 512u);
      continue;
    }
    sleep_ns = 32;
    ws_set(a, WS_COPY);
    const ReqView rv = load_req(a.req + r);  // published entry: the same for every lane
    SrvReq* e = a.req + r;
    // self-check: a request outside this run or with an unknown template is
    // reported (ctl->bad) and stops the engine instead of being executed
    const bool ok = r < a.n_req && rv.id == r && k < rv.N &&
                    ((rv.kind == 0 && rv.tmpl < a.n_mt && rv.dst >= a.arena_lo && rv.dst < a.arena_hi) ||
                     (rv.kind == 1 && rv.tmpl < a.n_bt));
    if (!ok) {
      if (lane == 0) {
        atomicCAS(&a.ctl->bad.v, 0ull, 1ull + r);
        atomicExch(&a.ctl->abort.v, 1ull);
      }
      ws_set(a, WS_WORKER_DONE);
      return;
    }
    if (rv.kind == 0) {
      srv_copy_chunk(a, e, rv, k, lane);
    } else if (!srv_push_group(a, e, rv, k, lane, deadline)) {
      ws_set(a, WS_WORKER_DONE);
      return;
    }
  }
}

__device__ void srv_consumer(const SrvArgs& a, unsigned c, unsigned long long deadline) {
  // s_stop is written only by thread 0 before the first barrier of a round;
  // phase-A waits that give up write s_abort_a, read after the second
  // barrier and cleared by thread 0 at the start of the next round (after the
  // round's last barrier), so no thread can see a flag meant for a later
  // check and leave while others wait at a barrier.
  __shared__ int s_stop, s_abort_a;
  __shared__ unsigned long long s_avail;
  __shared__ unsigned long long s_start[SRV_WIN], s_ppre[SRV_WIN + 1], s_dig[SRV_WIN];
  __shared__ unsigned int s_size[SRV_WIN], s_prod[SRV_WIN], s_seq[SRV_WIN];
  const MpscView v = a.chans[c];
  const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const unsigned long long win_max = min((unsigned long long)SRV_WIN, (unsigned long long)(v.M / 2 ? v.M / 2 : 1));
  __shared__ unsigned long long s_t0;
  if (tid == 0) s_t0 = ld_acq(&v.st->msg_tail.v);
  __syncthreads();
  unsigned long long t = s_t0, consumed = 0;
  for (;;) {
    ws_set(a, WS_C_AVAIL);
    if (tid == 0) {
      int stop = 0;
      unsigned long long avail = 0;
      unsigned sleep_ns = 64;
      for (;;) {
        const unsigned long long W = ld_acq(&v.st->reserve.v);
        avail = ((W >> 40) - t) & MASK24;
        if (avail) break;
        if (ld_acq(&a.ctl->stop.v) && consumed >= *(volatile unsigned long long*)&a.ctl->final_msgs[c]) {
          stop = 2;  // done
          break;
        }
        if (srv_abort(a, deadline)) {
          stop = 1;
          break;
        }
        __nanosleep(sleep_ns);
        sleep_ns = min(sleep_ns * 2, 1024u);
      }
      s_avail = min(avail, win_max);
      s_stop = stop;
      s_abort_a = 0;
    }
    __syncthreads();
    if (s_stop) {
      ws_set(a, WS_C_DONE);
      return;
    }
    const unsigned navail = (unsigned)s_avail;
    ws_set(a, WS_C_READY);
    for (unsigned j = warp; j < navail; j += nwarp) {
      const unsigned long long tk = t + j;
      MpscMeta* m = v.meta + (tk & (v.M - 1));
      if (lane == 0) {
        int stop = 0;
        while (ld_acq(&m->ready) != (tk & MASK24) + 1) {
          if (srv_abort(a, deadline)) {
            stop = 1;
            break;
          }
          __nanosleep(32);
        }
        if (stop) {
          s_abort_a = 1;
        } else {
          s_start[j] = __ldcg(&m->start);
          s_size[j] = __ldcg(&m->size);
          s_prod[j] = __ldcg(&m->producer);
          s_seq[j] = __ldcg(&m->seq);
          s_dig[j] = 0;
        }
      }
    }
    __syncthreads();
    if (s_abort_a) {
      ws_set(a, WS_C_DONE);
      return;
    }
    ws_set(a, WS_C_DIGEST);
    if (warp == 0) {
      const unsigned long long p0 =
          lane < navail ? (((unsigned long long)s_size[lane] + 15) / 16 + SRV_PIECE - 1) / SRV_PIECE : 0;
      const unsigned long long p1 =
          lane + 32 < navail ? (((unsigned long long)s_size[lane + 32] + 15) / 16 + SRV_PIECE - 1) / SRV_PIECE : 0;
      unsigned long long x0 = p0, x1 = p1;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y0 = __shfl_up_sync(FULLM, x0, o), y1 = __shfl_up_sync(FULLM, x1, o);
        if (lane >= (unsigned)o) {
          x0 += y0;
          x1 += y1;
        }
      }
      const unsigned long long tot0 = __shfl_sync(FULLM, x0, 31);
      s_ppre[lane] = x0 - p0;
      s_ppre[lane + 32] = tot0 + x1 - p1;
      if (lane == 31) s_ppre[64] = tot0 + x1;
    }
    __syncthreads();
    const unsigned long long npieces = s_ppre[navail];
    for (unsigned long long pc = warp; pc < npieces; pc += nwarp) {
      unsigned lo = 0, hi = navail;
      while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (s_ppre[mid] <= pc) lo = mid;
        else hi = mid;
      }
      const unsigned j = lo;
      const unsigned long long n = s_size[j];
      const unsigned long long q0 = (pc - s_ppre[j]) * SRV_PIECE;
      const uint4* base = reinterpret_cast<const uint4*>(v.ring + (s_start[j] & (v.R - 1)));
      unsigned long long d = piece_digest<SRV_PIECE / 32>(base, q0, n, lane);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULLM, d, o);
      if (lane == 0) atomicAdd(&s_dig[j], d);
    }
    // self-check of the channel's order per producer: message j must be its
    // request's next one (messages consumed in earlier windows, all of them
    // by this consumer, plus earlier messages of the request in this window)
    for (unsigned j = tid; j < navail; j += blockDim.x) {
      if (s_prod[j] < a.n_req) {
        unsigned k = 0;
        for (unsigned i = 0; i < j; ++i) k += (s_prod[i] == s_prod[j]);
        if (s_seq[j] != __ldcg(&a.req[s_prod[j]].done) + k) {
          atomicCAS(&a.ctl->bad.v, 0ull, 1ull + s_prod[j]);
          atomicExch(&a.ctl->abort.v, 1ull);
        }
      }
    }
    // capture: warp w copies messages w, w + nwarp, ... of the window out of
    // the ring before the window is freed (after the barrier below)
    if (a.cap) {
      for (unsigned j = warp; j < navail; j += nwarp) {
        if (s_prod[j] >= a.n_req) continue;  // the self-check reports it
        const unsigned long long co = __ldcg(&a.cap_off[s_prod[j]]);
        if (co == ~0ull) continue;
        const unsigned tm = __ldcg(&a.req[s_prod[j]].tmpl);
        if (tm >= a.n_bt || s_seq[j] >= a.t_nmsg[tm]) continue;
        const unsigned long long mi = a.t_mbase[tm] + s_seq[j];
        capture_copy(a.cap + co + a.mcap[mi], v.ring + (s_start[j] & (v.R - 1)),
                     min((unsigned long long)s_size[j], a.msizes[mi]), lane);
      }
    }
    __syncthreads();
    ws_set(a, WS_C_ACCOUNT);
    // per-request accounting: message digest weighted by its index in the burst
    for (unsigned j = tid; j < navail; j += blockDim.x) {
      if (s_prod[j] >= a.n_req) {  // self-check, as in the workers
        atomicCAS(&a.ctl->bad.v, 0ull, 1ull + s_prod[j]);
        atomicExch(&a.ctl->abort.v, 1ull);
        continue;
      }
      SrvReq* e = a.req + s_prod[j];
      atomicAdd(&e->digest, s_dig[j] * (2ull * s_seq[j] + 1ull));
      __threadfence();
      const unsigned long long prev = atomicAdd(&e->done, 1ull);
      if (prev + 1 == __ldcg(&e->need)) srv_complete(a, e);
    }
    if (tid == 0) {
      st_rel(&v.st->freed.v, (s_start[navail - 1] + round16(s_size[navail - 1])) & MASK40);
      st_rel(&v.st->msg_tail.v, t + navail);
    }
    t += navail;
    consumed += navail;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SRV_THREADS) k_serve(SrvArgs a) {
  __shared__ unsigned long long s_deadline;
  if (threadIdx.x == 0) s_deadline = gtime() + a.timeout_ns;
  __syncthreads();
  const unsigned long long deadline = s_deadline;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) srv_dispatcher(a, deadline);
  } else if (blockIdx.x <= a.n_ch) {
    srv_consumer(a, blockIdx.x - 1, deadline);
  } else {
    srv_worker(a, deadline);
  }
  atomicAdd(&a.ctl->exited.v, 1ull);  // diagnostics: threads that reached the end
}

// Verify mode: digest of every op's destination bytes, weighted by the op's
// index in its template, summed per request. One warp per (request, op).
struct VerifyItem {
  unsigned long long addr, n, req, k;
};
__global__ void k_serve_verify(const VerifyItem* items, unsigned long long count, unsigned long long* out) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long i = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += warps) {
    const VerifyItem it = items[i];
    const uint8_t* p = reinterpret_cast<const uint8_t*>(it.addr);
    const unsigned long long nw = (it.n + 7) / 8;
    unsigned long long d = 0;
    for (unsigned long long j = lane; j < nw; j += 32) {
      unsigned long long w = 0;
      for (int b = 0; b < 8; ++b)
        if (8 * j + b < it.n) w |= (unsigned long long)p[8 * j + b] << (8 * b);
      d += w * (2ull * j + 1ull);
    }
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULLM, d, o);
    if (lane == 0) atomicAdd(out + it.req, d * (2ull * it.k + 1ull));
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct Arena {
  // first-fit over free ranges (offset -> size), 256-byte granules
  std::map<uint64_t, uint64_t> free_;
  uint64_t size = 0, used = 0, high = 0;
  void reset(uint64_t n) {
    free_.clear();
    free_[0] = n;
    size = n;
    used = high = 0;
  }
  bool alloc(uint64_t n, uint64_t* off) {
    n = std::max<uint64_t>(256, (n + 255) & ~255ull);
    if (size - used < n) return false;  // no walk while the arena is full
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const uint64_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used += n;
        high = std::max(high, used);
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    n = std::max<uint64_t>(256, (n + 255) & ~255ull);
    used -= n;
    auto next = free_.lower_bound(off);
    uint64_t a = off, b = off + n;
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == a) {
        a = prev->first;
        free_.erase(prev);
      }
    }
    next = free_.lower_bound(b);
    if (next != free_.end() && next->first == b) {
      b += next->second;
      free_.erase(next);
    }
    free_[a] = b - a;
  }
};

struct Server {
  hicr_serve_config_t cfg{};
  bool live = false;
  hicr_slot_t arena_slot = 0;
  uint8_t* arena = nullptr;
  uint8_t* rings = nullptr;           // n_ch rings, states and metadata (one allocation)
  std::vector<MpscView> views;
  // templates (host copies; uploaded lazily)
  std::vector<hicr_op_t> tops;
  std::vector<unsigned long long> tcstart, t_opbase, t_nops, t_cbase, t_total, t_region;
  std::vector<unsigned long long> msizes, moffs, t_mbase, t_nmsg, gstart, t_gbase, t_ngrp, t_whole;
  hicr_slot_t staging = 0;
  bool have_staging = false;
  bool uploaded = false;
  void* dev_tmpl = nullptr;  // one allocation for all template arrays
  SrvArgs base{};
  SrvCtl* ctl = nullptr;
  MpscView* d_views = nullptr;
  std::vector<unsigned long long> t_bytes, m_bytes;  // payload bytes per template
  std::vector<unsigned long long> mcap;              // per template message: exclusive prefix of sizes
  std::vector<uint8_t> kept;  // last run: memcpy requests whose region was not reused
};

static Server* srv_get(Instance* in, hicr_serve_t s);

}  // namespace hicr

// the instance keeps its servers in a side table keyed by instance pointer
#include <unordered_map>
namespace hicr {
static std::unordered_map<Instance*, std::vector<Server*>> g_servers;
static Server* srv_get(Instance* in, hicr_serve_t s) {
  auto it = g_servers.find(in);
  if (it == g_servers.end() || s == 0 || s > it->second.size()) return nullptr;
  Server* v = it->second[s - 1];
  return (v && v->live) ? v : nullptr;
}

// Called by hicr_finalize: release every engine the caller did not destroy.
// The arena is an owned slot and is freed with the instance's slots.
void destroy_servers(Instance* in) {
  auto it = g_servers.find(in);
  if (it == g_servers.end()) return;
  for (Server* sv : it->second) {
    if (!sv) continue;
    if (sv->rings) cudaFree(sv->rings);
    if (sv->dev_tmpl) cudaFree(sv->dev_tmpl);
    delete sv;
  }
  g_servers.erase(it);
}

template <class T>
static char* put(char* p, const std::vector<T>& v, const T** dst) {
  const size_t n = v.size() * sizeof(T);
  *dst = (const T*)p;
  return p + ((n + 255) & ~(size_t)255);
}

static hicr_status srv_upload(Instance* in, Server* sv) {
  if (sv->uploaded) return HICR_OK;
  if (sv->t_nops.empty()) sv->t_nops.push_back(0), sv->t_opbase.push_back(0), sv->t_cbase.push_back(0),
      sv->t_total.push_back(0), sv->t_region.push_back(0), sv->tcstart.push_back(0);
  if (sv->t_nmsg.empty()) sv->t_nmsg.push_back(0), sv->t_mbase.push_back(0), sv->t_gbase.push_back(0),
      sv->t_ngrp.push_back(0), sv->t_whole.push_back(0);
  if (sv->gstart.empty()) sv->gstart.push_back(0);
  if (sv->tops.empty()) sv->tops.push_back(hicr_op_t{0, 0, 0, 0, 0});
  if (sv->msizes.empty()) sv->msizes.push_back(0), sv->moffs.push_back(0), sv->mcap.push_back(0);
  std::vector<const void*> dummy;
  auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const size_t bytes = al(sv->tops.size() * sizeof(hicr_op_t)) +
                       8 * (al(sv->tcstart.size() * 8) + al(sv->t_opbase.size() * 8) + al(sv->t_nops.size() * 8) +
                            al(sv->t_cbase.size() * 8) + al(sv->t_total.size() * 8) +
                            al(sv->msizes.size() * 8) + al(sv->moffs.size() * 8) + al(sv->t_mbase.size() * 8) +
                            al(sv->t_nmsg.size() * 8) + al(sv->gstart.size() * 8) + al(sv->t_gbase.size() * 8) +
                            al(sv->t_ngrp.size() * 8) + al(sv->t_whole.size() * 8) + al(sv->mcap.size() * 8)) / 8;
  char* d = nullptr;
  HICR_CUDA(in, cudaMalloc(&d, bytes + 4096));
  sv->dev_tmpl = d;
  char* p = d;
  SrvArgs& a = sv->base;
  auto up = [&](const void* src, size_t n) -> hicr_status {
    HICR_CUDA(in, cudaMemcpy(p, src, n, cudaMemcpyHostToDevice));
    p += al(n);
    return HICR_OK;
  };
  a.tops = (const hicr_op_t*)p;
  if (up(sv->tops.data(), sv->tops.size() * sizeof(hicr_op_t))) return HICR_ERR_DEVICE;
#define UP(field, vec)                                   \
  a.field = (const unsigned long long*)p;                \
  if (up(vec.data(), vec.size() * 8)) return HICR_ERR_DEVICE;
  UP(tcstart, sv->tcstart);
  UP(t_opbase, sv->t_opbase);
  UP(t_nops, sv->t_nops);
  UP(t_cbase, sv->t_cbase);
  UP(t_total, sv->t_total);
  UP(msizes, sv->msizes);
  UP(moffs, sv->moffs);
  UP(t_mbase, sv->t_mbase);
  UP(t_nmsg, sv->t_nmsg);
  UP(gstart, sv->gstart);
  UP(t_gbase, sv->t_gbase);
  UP(t_ngrp, sv->t_ngrp);
  UP(t_whole, sv->t_whole);
  UP(mcap, sv->mcap);
#undef UP
  sv->uploaded = true;
  return HICR_OK;
}

}  // namespace hicr

using namespace hicr;

static Instance* I(hicr_instance_t h) { return h ? &h->impl : nullptr; }

static bool pow2u(unsigned long long x) { return x && !(x & (x - 1)); }

extern "C" {

hicr_status hicr_serve_create(hicr_instance_t h, const hicr_serve_config_t* cfg, hicr_serve_t* out) {
  Instance* in = I(h);
  if (!in || !cfg || !out || in->capturing) return HICR_ERR_INVALID;
  if (cfg->n_channels == 0 || cfg->n_channels > SRV_MAX_CH || !pow2u(cfg->ring_bytes) || cfg->ring_bytes < 64 ||
      cfg->ring_bytes > (1ull << 39) || !pow2u(cfg->max_msgs) || cfg->max_msgs > (1u << 23) ||
      cfg->chunk_bytes < 1024 || cfg->chunk_bytes % 1024 || cfg->op_cost_bytes == 0)
    return HICR_ERR_INVALID;
  const uint64_t ring_total = (uint64_t)cfg->n_channels * cfg->ring_bytes;
  if (cfg->budget_bytes <= ring_total) return HICR_ERR_INVALID;
  Server* sv = new Server();
  sv->cfg = *cfg;
  const uint64_t arena_bytes = cfg->budget_bytes - ring_total;
  hicr_status st = hicr_mem_alloc(h, HICR_SPACE_HBM, arena_bytes, 0, &sv->arena_slot);
  if (st != HICR_OK) {
    delete sv;
    return st;
  }
  void* ap = nullptr;
  hicr_slot_info(h, sv->arena_slot, &ap, nullptr, nullptr, nullptr);
  sv->arena = (uint8_t*)ap;
  // rings + channel states + metadata + control block + request ring
  const size_t n = cfg->n_channels;
  const size_t st_b = (sizeof(MpscState) + 255) & ~(size_t)255;
  const size_t meta_b = ((sizeof(MpscMeta) * (size_t)cfg->max_msgs) + 255) & ~(size_t)255;
  const size_t ctl_b = (sizeof(SrvCtl) + 255) & ~(size_t)255;
  const size_t views_b = (sizeof(MpscView) * n + 255) & ~(size_t)255;
  const size_t total = ring_total + n * (st_b + meta_b) + ctl_b + views_b;
  char* p = nullptr;
  cudaError_t e = cudaMalloc(&p, total);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    hicr_mem_free(h, sv->arena_slot);
    delete sv;
    return e == cudaErrorMemoryAllocation ? HICR_ERR_NOMEM : HICR_ERR_DEVICE;
  }
  sv->rings = (uint8_t*)p;
  char* q = p + ring_total;
  for (size_t c = 0; c < n; ++c) {
    MpscView v;
    v.ring = (uint8_t*)p + c * cfg->ring_bytes;
    v.st = (MpscState*)q;
    q += st_b;
    v.meta = (MpscMeta*)q;
    q += meta_b;
    v.R = cfg->ring_bytes;
    v.M = cfg->max_msgs;
    sv->views.push_back(v);
  }
  const size_t zero_from = ring_total;
  sv->ctl = (SrvCtl*)q;
  q += ctl_b;
  sv->d_views = (MpscView*)q;
  HICR_CUDA(in, cudaMemset(p + zero_from, 0, total - zero_from));
  HICR_CUDA(in, cudaMemcpy(sv->d_views, sv->views.data(), sizeof(MpscView) * n, cudaMemcpyHostToDevice));
  sv->live = true;
  auto& vec = g_servers[in];
  vec.push_back(sv);
  *out = (hicr_serve_t)vec.size();
  return HICR_OK;
}

hicr_status hicr_serve_destroy(hicr_instance_t h, hicr_serve_t s) {
  Instance* in = I(h);
  if (!in) return HICR_ERR_INVALID;
  Server* sv = srv_get(in, s);
  if (!sv) return HICR_ERR_INVALID;
  HICR_CUDA(in, cudaDeviceSynchronize());
  hicr_mem_free(h, sv->arena_slot);
  cudaFree(sv->rings);
  if (sv->dev_tmpl) cudaFree(sv->dev_tmpl);
  sv->live = false;
  g_servers[in][s - 1] = nullptr;
  delete sv;
  return HICR_OK;
}

hicr_status hicr_serve_add_memcpy_template(hicr_instance_t h, hicr_serve_t s, const hicr_op_t* ops, uint64_t count,
                                           uint64_t region_bytes, uint32_t* tmpl) {
  Instance* in = I(h);
  if (!in || !tmpl || (count && !ops)) return HICR_ERR_INVALID;
  Server* sv = srv_get(in, s);
  if (!sv || sv->uploaded) return HICR_ERR_INVALID;
  const uint64_t region = (region_bytes + 255) & ~255ull;
  if (region > sv->cfg.budget_bytes - (uint64_t)sv->cfg.n_channels * sv->cfg.ring_bytes) return HICR_ERR_NOMEM;
  for (uint64_t i = 0; i < count; ++i) {
    const hicr_op_t& o = ops[i];
    void* sp = nullptr;
    uint64_t ssize = 0;
    uint32_t sspace = 0;
    if (hicr_slot_info(h, o.src, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
    if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
    if (o.src_off > ssize || o.n > ssize - o.src_off) return HICR_ERR_BOUNDS;
    if (o.dst_off > region_bytes || o.n > region_bytes - o.dst_off) return HICR_ERR_BOUNDS;
  }
  const uint32_t t = (uint32_t)sv->t_nops.size();
  sv->t_opbase.push_back(sv->tops.size());
  sv->t_nops.push_back(count);
  sv->t_cbase.push_back(sv->tcstart.size());
  unsigned long long c = 0;
  for (uint64_t i = 0; i < count; ++i) {
    sv->tops.push_back(ops[i]);
    sv->tcstart.push_back(c);
    c += ops[i].n + sv->cfg.op_cost_bytes;
  }
  sv->tcstart.push_back(c);
  sv->t_total.push_back(c);
  sv->t_region.push_back(region_bytes);
  unsigned long long tb = 0;
  for (uint64_t i = 0; i < count; ++i) tb += ops[i].n;
  sv->t_bytes.push_back(tb);
  *tmpl = t;
  return HICR_OK;
}

hicr_status hicr_serve_add_burst_template(hicr_instance_t h, hicr_serve_t s, const uint64_t* sizes,
                                          const uint64_t* staging_off, uint64_t count, hicr_slot_t staging,
                                          uint32_t* tmpl) {
  Instance* in = I(h);
  if (!in || !tmpl || (count && (!sizes || !staging_off))) return HICR_ERR_INVALID;
  Server* sv = srv_get(in, s);
  if (!sv || sv->uploaded) return HICR_ERR_INVALID;
  void* sp = nullptr;
  uint64_t ssize = 0;
  uint32_t sspace = 0;
  if (hicr_slot_info(h, staging, &sp, &ssize, &sspace, nullptr) != HICR_OK) return HICR_ERR_INVALID;
  if (sspace != HICR_SPACE_HBM) return HICR_ERR_UNSUPPORTED;
  if (sv->have_staging && staging != sv->staging) return HICR_ERR_INVALID;  // one staging slot per engine
  for (uint64_t i = 0; i < count; ++i) {
    if (staging_off[i] > ssize || sizes[i] > ssize - staging_off[i]) return HICR_ERR_BOUNDS;
    if (round16(sizes[i]) > sv->cfg.ring_bytes / 2) return HICR_ERR_TOO_LARGE;
  }
  sv->staging = staging;
  sv->have_staging = true;
  sv->base.staging = (const uint8_t*)sp;
  const uint32_t t = (uint32_t)sv->t_nmsg.size();
  sv->t_mbase.push_back(sv->msizes.size());
  sv->t_nmsg.push_back(count);
  unsigned long long mb = 0;
  for (uint64_t i = 0; i < count; ++i) {
    sv->msizes.push_back(sizes[i]);
    sv->moffs.push_back(staging_off[i]);
    sv->mcap.push_back(mb);
    mb += sizes[i];
  }
  sv->m_bytes.push_back(mb);
  // message groups (work units): consecutive messages, at most SRV_GROUP_MSGS
  // of them and at most SRV_GROUP_BYTES rounded bytes unless a single message
  // is larger; every group is at most half a ring (each message is)
  sv->t_gbase.push_back(sv->gstart.size());
  uint64_t ng = 0, gb = 0, gm = 0;
  for (uint64_t i = 0; i < count; ++i) {
    const uint64_t r = round16(sizes[i]);
    if (gm == 0 || gm == SRV_GROUP_MSGS || gb + r > SRV_GROUP_BYTES || gb + r > sv->cfg.ring_bytes / 2) {
      sv->gstart.push_back(i);
      ++ng;
      gb = 0;
      gm = 0;
    }
    gb += r;
    ++gm;
  }
  sv->gstart.push_back(count);
  sv->t_ngrp.push_back(ng);
  // reserved whole when the burst takes at most half the ring and half the
  // message slots (so that it fits an emptied channel)
  uint64_t rb = 0;
  for (uint64_t i = 0; i < count; ++i) rb += round16(sizes[i]);
  sv->t_whole.push_back(rb <= sv->cfg.ring_bytes / 2 && count <= sv->cfg.max_msgs / 2 ? 1 : 0);
  *tmpl = t;
  return HICR_OK;
}

}  // extern "C"

namespace hicr {

static hicr_status serve_run(hicr_instance_t h, hicr_serve_t s, const hicr_serve_request_t* reqs, uint64_t n,
                             uint32_t mode, uint64_t timeout_ns, const uint8_t* keep, void* d_capture,
                             const uint64_t* d_cap_off, hicr_serve_result_t* results, hicr_serve_stats_t* stats) {
  hicr::NvtxRange nvtx_range("hicr_serve_run");
  Instance* in = I(h);
  if (!in || (n && !reqs) || mode > 1 || in->capturing || (d_capture && !d_cap_off)) return HICR_ERR_INVALID;
  Server* sv = srv_get(in, s);
  if (!sv) return HICR_ERR_INVALID;
  for (uint64_t i = 0; i < n; ++i) {
    const hicr_serve_request_t& r = reqs[i];
    if (r.kind > 1) return HICR_ERR_INVALID;
    if (r.kind == 0 && r.tmpl >= sv->t_nops.size()) return HICR_ERR_INVALID;
    if (r.kind == 1 && r.tmpl >= sv->t_nmsg.size()) return HICR_ERR_INVALID;
    if (i && r.arrival_ns < reqs[i - 1].arrival_ns) return HICR_ERR_INVALID;
    if (r.kind == 1 && !sv->have_staging) return HICR_ERR_INVALID;
  }
  hicr_status st = hicr_flush(h);
  if (st != HICR_OK) return st;
  // a cooperative grid sized for the whole device: a latency-mode server ends first
  if ((st = lat_stop(in)) != HICR_OK) return st;
  HICR_CUDA(in, cudaStreamSynchronize(in->comm()));
  if ((st = srv_upload(in, sv)) != HICR_OK) return st;

  // mapped host memory: descriptors, doorbell, stop, completion, digests
  const size_t hbytes = sizeof(SrvHostDesc) * (n + 1) + 256 + 16 * (n + 1);
  char* hp = nullptr;
  HICR_CUDA(in, cudaHostAlloc((void**)&hp, hbytes, cudaHostAllocMapped));
  memset(hp, 0, hbytes);
  char* dp = nullptr;
  cudaError_t ce = cudaHostGetDevicePointer((void**)&dp, hp, 0);
  if (ce != cudaSuccess) {
    cudaFreeHost(hp);
    return cuda_fail(in, ce, "cudaHostGetDevicePointer");
  }
  SrvHostDesc* hdesc = (SrvHostDesc*)hp;
  const size_t o_door = sizeof(SrvHostDesc) * (n + 1);
  std::atomic<unsigned long long>* door = (std::atomic<unsigned long long>*)(hp + o_door);
  std::atomic<unsigned long long>* hstop = (std::atomic<unsigned long long>*)(hp + o_door + 128);
  std::atomic<unsigned long long>* compl_ = (std::atomic<unsigned long long>*)(hp + o_door + 256);
  unsigned long long* digest = (unsigned long long*)(hp + o_door + 256 + 8 * (n + 1));

  // fresh control block and per-request state for this run; channels keep
  // their counters
  SrvReq* dreq = nullptr;
  ce = cudaMalloc(&dreq, sizeof(SrvReq) * (n + 1));
  if (ce != cudaSuccess) {
    cudaFreeHost(hp);
    return cuda_fail(in, ce, "cudaMalloc(requests)");
  }
  // on the communication stream, so that the engine launched there sees them
  HICR_CUDA(in, cudaMemsetAsync(dreq, 0, sizeof(SrvReq) * (n + 1), in->comm()));
  HICR_CUDA(in, cudaMemsetAsync(sv->ctl, 0, sizeof(SrvCtl), in->comm()));
  SrvArgs a = sv->base;
  a.ctl = sv->ctl;
  a.req = dreq;
  a.hdesc = (const SrvHostDesc*)dp;
  a.hdoor = (const unsigned long long*)(dp + o_door);
  a.hstop = (const unsigned long long*)(dp + o_door + 128);
  a.hcompl = (unsigned long long*)(dp + o_door + 256);
  a.hdigest = (unsigned long long*)(dp + o_door + 256 + 8 * (n + 1));
  a.dt = in->dt;
  a.chans = sv->d_views;
  a.n_ch = sv->cfg.n_channels;
  a.chunk = sv->cfg.chunk_bytes;
  a.op_cost = sv->cfg.op_cost_bytes;
  a.timeout_ns = timeout_ns;
  a.n_req = n;
  a.n_mt = (unsigned)sv->t_nops.size();
  a.n_bt = (unsigned)sv->t_nmsg.size();
  a.arena_lo = (unsigned long long)sv->arena;
  a.arena_hi = (unsigned long long)sv->arena + (sv->cfg.budget_bytes - (uint64_t)sv->cfg.n_channels * sv->cfg.ring_bytes);
  a.cap = (uint8_t*)d_capture;
  a.cap_off = (const unsigned long long*)d_cap_off;
  sv->kept.assign(n, sv->cfg.verify ? 1 : 0);
  if (keep)
    for (uint64_t r = 0; r < n; ++r) sv->kept[r] |= keep[r] ? 1 : 0;
  int per_sm = 0;
  HICR_CUDA(in, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_serve, SRV_THREADS, 0));
  const unsigned grid = (unsigned)(in->sm_count * std::max(1, per_sm));
  const size_t n_warps = (size_t)grid * (SRV_THREADS / 32);
  unsigned int* wstate = nullptr;
  HICR_CUDA(in, cudaMalloc(&wstate, 4 * n_warps));
  HICR_CUDA(in, cudaMemsetAsync(wstate, 0, 4 * n_warps, in->comm()));
  a.wstate = wstate;
  if (grid < a.n_ch + 2) {
    cudaFreeHost(hp);
    cudaFree(dreq);
    cudaFree(wstate);
    return HICR_ERR_INVALID;
  }
  void* args[] = {&a};
  cudaStream_t cs = in->comm();
  ce = cudaLaunchCooperativeKernel((const void*)k_serve, dim3(grid), dim3(SRV_THREADS), args, 0, cs);
  if (ce != cudaSuccess) {
    cudaFreeHost(hp);
    cudaFree(dreq);
    cudaFree(wstate);
    return cuda_fail(in, ce, "cudaLaunchCooperativeKernel(k_serve)");
  }

  Arena arena;
  arena.reset(sv->cfg.budget_bytes - (uint64_t)sv->cfg.n_channels * sv->cfg.ring_bytes);
  std::vector<uint64_t> region_off(n, 0), region_len(n, 0), admit_t(n, 0);
  std::vector<uint64_t> inflight;
  inflight.reserve(4096);
  // requests [next_admit, next_arrival) have arrived and wait, in order, for admission
  uint64_t next_arrival = 0, next_admit = 0, completed = 0, max_inflight = 0, bytes = 0, burst_bytes = 0;
  // Fault the results array in now: a fresh (lazily mapped) array would
  // otherwise take its page faults inside the run, and a fault that makes the
  // kernel zero or compact a huge page stops this thread for milliseconds.
  if (results) memset(results, 0, sizeof(hicr_serve_result_t) * n);
  const uint64_t t0 = now_ns();
  uint64_t last_done = t0;
  uint64_t prev_pass = 0, max_gap = 0, max_gap_at = 0;  // longest interval between two passes of this loop
  hicr_status result = HICR_OK;
  for (;;) {
    const uint64_t now = now_ns() - t0;
    if (now - prev_pass > max_gap) {
      max_gap = now - prev_pass;
      max_gap_at = now;
    }
    prev_pass = now;
    if (now > timeout_ns) {
      result = HICR_ERR_TIMEOUT;
      break;
    }
    // arrivals
    if (mode == 0) {
      while (next_arrival < n && reqs[next_arrival].arrival_ns <= now) ++next_arrival;
    } else if (inflight.empty() && next_arrival < n && next_admit == next_arrival) {
      ++next_arrival;  // alone: the next request once the previous completed
    }
    // FIFO admission under the arena budget
    bool published = false;
    while (next_admit < next_arrival) {
      const uint64_t r = next_admit;
      const hicr_serve_request_t& q = reqs[r];
      uint64_t off = 0;
      if (q.kind == 0) {
        const uint64_t need = sv->t_region[q.tmpl];
        if (!arena.alloc(need, &off)) break;
        region_len[r] = need;
        region_off[r] = off;
      }
      hdesc[r].kind = q.kind;
      hdesc[r].tmpl = q.tmpl;
      hdesc[r].dst = (unsigned long long)(sv->arena + off);
      admit_t[r] = now_ns() - t0;
      inflight.push_back(r);
      max_inflight = std::max<uint64_t>(max_inflight, inflight.size());
      ++next_admit;
      published = true;
    }
    if (published) door->store(next_admit, std::memory_order_release);
    // completions
    for (size_t i = 0; i < inflight.size();) {
      const uint64_t r = inflight[i];
      if (compl_[r].load(std::memory_order_acquire) != 0) {
        const uint64_t tnow = now_ns();
        if (results) {
          results[r].latency_ns = (tnow - t0) - std::min<uint64_t>(tnow - t0, mode == 0 ? reqs[r].arrival_ns : admit_t[r]);
          results[r].admit_ns = mode == 0 ? admit_t[r] - std::min(admit_t[r], reqs[r].arrival_ns) : 0;
          results[r].digest = digest[r];
          results[r].dst_offset = region_off[r];
          results[r].device_done_ns = compl_[r].load(std::memory_order_relaxed) & ~1ull;
        }
        if (reqs[r].kind == 0) {
          bytes += sv->t_bytes[reqs[r].tmpl];
          if (!sv->kept[r]) arena.release(region_off[r], region_len[r]);
        } else {
          bytes += sv->m_bytes[reqs[r].tmpl];
          burst_bytes += sv->m_bytes[reqs[r].tmpl];
        }
        ++completed;
        last_done = tnow;
        inflight[i] = inflight.back();
        inflight.pop_back();
      } else {
        ++i;
      }
    }
    if (completed == n) break;
    // Idle until the next arrival: yield rather than sleep. A timed sleep on
    // Linux wakes up to a timer-slack late (tens of microseconds, sometimes
    // milliseconds), and that delay went straight into the next request's
    // admission time.
    if (next_admit == next_arrival && mode == 0 && next_arrival < n && inflight.empty())
      std::this_thread::yield();
  }
  hstop->store(1, std::memory_order_release);
  // Wait for the engine with a bound: its own deadline ends every device
  // wait, so it should stop by then; if it has not 10 s later, report and
  // return without freeing what it may still touch.
  const uint64_t wait_until = now_ns() + (timeout_ns > now_ns() - t0 ? timeout_ns - (now_ns() - t0) : 0) +
                              10ull * 1000000000ull;
  for (;;) {
    ce = cudaStreamQuery(cs);
    if (ce != cudaErrorNotReady) break;
    if (now_ns() > wait_until) break;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  // device-side progress counters and warp states (readable while the
  // kernel runs, on a side stream)
  unsigned long long dv[7] = {0, 0, 0, 0, 0, 0, 0};
  std::vector<SrvReq> stuck_req;
  std::vector<unsigned int> ws(n_warps, 0);
  const bool overdue = ce == cudaErrorNotReady;
  {
    cudaStream_t ps = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) == cudaSuccess) {
      cudaMemcpyAsync(ws.data(), wstate, 4 * n_warps, cudaMemcpyDeviceToHost, ps);
      if (overdue) {
        // ask every bounded wait to give up now
        static const unsigned long long one = 1;
        cudaMemcpyAsync(&sv->ctl->abort.v, &one, 8, cudaMemcpyHostToDevice, ps);
      }
      cudaMemcpyAsync(&dv[0], &sv->ctl->units_pub.v, 8, cudaMemcpyDeviceToHost, ps);
      cudaMemcpyAsync(&dv[1], &sv->ctl->claim.v, 8, cudaMemcpyDeviceToHost, ps);
      cudaMemcpyAsync(&dv[2], &sv->ctl->req_pub.v, 8, cudaMemcpyDeviceToHost, ps);
      cudaMemcpyAsync(&dv[3], &sv->ctl->stop.v, 8, cudaMemcpyDeviceToHost, ps);
      cudaMemcpyAsync(&dv[4], &sv->ctl->abort.v, 8, cudaMemcpyDeviceToHost, ps);
      cudaMemcpyAsync(&dv[5], &sv->ctl->bad.v, 8, cudaMemcpyDeviceToHost, ps);
      cudaMemcpyAsync(&dv[6], &sv->ctl->exited.v, 8, cudaMemcpyDeviceToHost, ps);
      if (result != HICR_OK || overdue) {
        stuck_req.resize(std::min<size_t>(inflight.size(), 8));
        for (size_t i = 0; i < stuck_req.size(); ++i)
          cudaMemcpyAsync(&stuck_req[i], dreq + inflight[i], sizeof(SrvReq), cudaMemcpyDeviceToHost, ps);
      }
      cudaStreamSynchronize(ps);
      cudaStreamDestroy(ps);
    }
    (void)cudaGetLastError();
  }
  if (stats) {
    stats->max_poll_gap_ns = max_gap;
    stats->max_poll_gap_at_ns = max_gap_at;
    stats->admitted = next_admit;
    stats->dev_units = dv[0];
    stats->dev_claimed = dv[1];
    stats->dev_requests = dv[2];
    stats->dev_flags = (dv[3] ? 1ull : 0ull) | (dv[4] ? 2ull : 0ull) | (dv[5] ? 4ull : 0ull);
  }
  if (overdue || result != HICR_OK) {
    std::map<unsigned, unsigned> hist;
    for (unsigned w : ws) hist[w]++;
    std::string msg = overdue ? "engine kernel overdue; warp states:" : "engine timed out; warp states:";
    for (auto& kv : hist) msg += " " + std::to_string(kv.first) + "x" + std::to_string(kv.second);
    msg += "; units_pub " + std::to_string(dv[0]) + " claimed " + std::to_string(dv[1]) + " req_pub " +
           std::to_string(dv[2]) + " admitted " + std::to_string(next_admit) + " completed " + std::to_string(completed) +
           " of " + std::to_string(n) + " flags stop/abort/bad " + std::to_string(dv[3]) + "/" + std::to_string(dv[4]) +
           "/" + std::to_string(dv[5]) + " threads exited " + std::to_string(dv[6]) + " of " +
           std::to_string(n_warps * 32) + "; pending:";
    for (size_t i = 0; i < stuck_req.size(); ++i)
      msg += " [r" + std::to_string(inflight[i]) + " kind " + std::to_string(stuck_req[i].kind) + " done " +
             std::to_string(stuck_req[i].done) + "/" + std::to_string(stuck_req[i].need) + " units " +
             std::to_string(stuck_req[i].U) + "+" + std::to_string(stuck_req[i].N) + "]";
    log_error(in, msg);
    fprintf(stderr, "hicr_serve_run: %s\n", msg.c_str());
    fflush(stderr);
  }
  if (overdue) {
    const uint64_t until = now_ns() + 10ull * 1000000000ull;
    while ((ce = cudaStreamQuery(cs)) == cudaErrorNotReady && now_ns() < until)
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    if (ce == cudaErrorNotReady) {
      if (stats) {
        stats->completed = completed;
        stats->status = HICR_ERR_TIMEOUT;
      }
      return HICR_ERR_TIMEOUT;
    }
  }
  cudaFree(wstate);
  cudaFree(dreq);
  if (ce != cudaSuccess) {
    cudaFreeHost(hp);
    return cuda_fail(in, ce, "k_serve");
  }
  const unsigned long long bad = dv[5];
  if (bad) {
    log_error(in, "serving engine self-check failed at request " + std::to_string(bad - 1));
    result = HICR_ERR_DEVICE;
  }
  if (stats) {
    stats->completed = completed;
    stats->bytes_moved = bytes;
    stats->burst_bytes = burst_bytes;
    stats->wall_ns = last_done - t0 - (n && mode == 0 ? std::min<uint64_t>(last_done - t0, reqs[0].arrival_ns) : 0);
    stats->max_inflight = max_inflight;
    stats->max_region_bytes = arena.high;
    stats->status = result;
  }
  cudaFreeHost(hp);
  HICR_CUDA(in, cudaGetLastError());
  return result;
}

}  // namespace hicr

extern "C" {

hicr_status hicr_serve_run(hicr_instance_t h, hicr_serve_t s, const hicr_serve_request_t* reqs, uint64_t n,
                           uint32_t mode, uint64_t timeout_ns, hicr_serve_result_t* results,
                           hicr_serve_stats_t* stats) {
  return serve_run(h, s, reqs, n, mode, timeout_ns, nullptr, nullptr, nullptr, results, stats);
}

hicr_status hicr_serve_run_ex(hicr_instance_t h, hicr_serve_t s, const hicr_serve_request_t* reqs, uint64_t n,
                              uint32_t mode, uint64_t timeout_ns, const uint8_t* keep, void* d_capture,
                              const uint64_t* d_cap_off, hicr_serve_result_t* results, hicr_serve_stats_t* stats) {
  return serve_run(h, s, reqs, n, mode, timeout_ns, keep, d_capture, d_cap_off, results, stats);
}

hicr_status hicr_serve_arena(hicr_instance_t h, hicr_serve_t s, hicr_slot_t* out) {
  Instance* in = I(h);
  if (!in || !out) return HICR_ERR_INVALID;
  Server* sv = srv_get(in, s);
  if (!sv) return HICR_ERR_INVALID;
  *out = sv->arena_slot;
  return HICR_OK;
}

hicr_status hicr_serve_run_plain(hicr_instance_t h, hicr_serve_t s, const hicr_serve_request_t* reqs, uint64_t n,
                                 uint64_t horizon_ns, uint64_t timeout_ns, hicr_serve_result_t* results,
                                 hicr_serve_stats_t* stats) {
  Instance* in = I(h);
  if (!in || (n && !reqs) || in->capturing) return HICR_ERR_INVALID;
  Server* sv = srv_get(in, s);
  if (!sv) return HICR_ERR_INVALID;
  uint64_t m = 0;
  while (m < n && reqs[m].arrival_ns <= horizon_ns) ++m;
  for (uint64_t i = 0; i < m; ++i) {
    if (reqs[i].kind == 0 && reqs[i].tmpl >= sv->t_nops.size()) return HICR_ERR_INVALID;
    if (reqs[i].kind == 1 && (reqs[i].tmpl >= sv->t_nmsg.size() || !sv->have_staging)) return HICR_ERR_INVALID;
  }
  cudaStream_t cs = in->comm();
  HICR_CUDA(in, cudaStreamSynchronize(cs));
  const size_t EV = 8192;
  std::vector<cudaEvent_t> ev(EV);
  for (auto& e : ev) HICR_CUDA(in, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  Arena arena;
  arena.reset(sv->cfg.budget_bytes - (uint64_t)sv->cfg.n_channels * sv->cfg.ring_bytes);
  std::vector<uint64_t> region_off(m, 0), region_len(m, 0);
  std::vector<uint64_t> ring_pos(sv->cfg.n_channels, 0);
  uint64_t next = 0, head = 0, completed = 0, bytes = 0, burst_bytes = 0, max_inflight = 0;  // in-flight = [head, next)
  if (results) memset(results, 0, sizeof(hicr_serve_result_t) * m);  // faulted in before the clock starts
  const uint64_t t0 = now_ns();
  uint64_t last_done = t0;
  uint64_t prev_pass = 0, max_gap = 0, max_gap_at = 0;
  hicr_status result = HICR_OK;
  const uint8_t* staging = sv->base.staging;
  while (completed < m) {
    const uint64_t now = now_ns() - t0;
    if (now - prev_pass > max_gap) {
      max_gap = now - prev_pass;
      max_gap_at = now;
    }
    prev_pass = now;
    if (now > timeout_ns) {
      result = HICR_ERR_TIMEOUT;
      break;
    }
    while (next < m && reqs[next].arrival_ns <= now && next - head < EV) {
      const hicr_serve_request_t& q = reqs[next];
      const unsigned t = q.tmpl;
      if (q.kind == 0) {
        uint64_t off = 0;
        if (!arena.alloc(sv->t_region[t], &off)) break;
        region_off[next] = off;
        region_len[next] = sv->t_region[t];
        for (uint64_t k = 0; k < sv->t_nops[t]; ++k) {
          const hicr_op_t& o = sv->tops[sv->t_opbase[t] + k];
          if (o.n == 0) continue;
          HICR_CUDA(in, cudaMemcpyAsync(sv->arena + off + o.dst_off, (const void*)(in->slots[o.src].base + o.src_off),
                                        o.n, cudaMemcpyDeviceToDevice, cs));
        }
      } else {
        const unsigned c = (unsigned)(next % sv->cfg.n_channels);
        for (uint64_t k = 0; k < sv->t_nmsg[t]; ++k) {
          const uint64_t sz = sv->msizes[sv->t_mbase[t] + k], r16 = round16(sz);
          if (ring_pos[c] + r16 > sv->cfg.ring_bytes) ring_pos[c] = 0;
          HICR_CUDA(in, cudaMemcpyAsync(sv->views[c].ring + ring_pos[c], staging + sv->moffs[sv->t_mbase[t] + k], sz,
                                        cudaMemcpyDeviceToDevice, cs));
          ring_pos[c] += r16;
        }
      }
      HICR_CUDA(in, cudaEventRecord(ev[next % EV], cs));
      ++next;
      max_inflight = std::max(max_inflight, next - head);
    }
    while (head < next) {
      cudaError_t e = cudaEventQuery(ev[head % EV]);
      if (e == cudaErrorNotReady) break;
      HICR_CUDA(in, e);
      const uint64_t tnow = now_ns();
      const hicr_serve_request_t& q = reqs[head];
      if (results) {
        results[head].latency_ns = (tnow - t0) - std::min<uint64_t>(tnow - t0, q.arrival_ns);
        results[head].admit_ns = 0;
        results[head].digest = 0;
        results[head].dst_offset = region_off[head];
        results[head].device_done_ns = 0;
      }
      if (q.kind == 0) {
        bytes += sv->t_bytes[q.tmpl];
        arena.release(region_off[head], region_len[head]);
      } else {
        bytes += sv->m_bytes[q.tmpl];
        burst_bytes += sv->m_bytes[q.tmpl];
      }
      ++completed;
      ++head;
      last_done = tnow;
    }
  }
  {
    const uint64_t until = now_ns() + 60ull * 1000000000ull;
    while (cudaStreamQuery(cs) == cudaErrorNotReady && now_ns() < until)
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    (void)cudaGetLastError();
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (stats) {
    stats->completed = completed;
    stats->bytes_moved = bytes;
    stats->burst_bytes = burst_bytes;
    stats->wall_ns = last_done - t0 - (m ? std::min<uint64_t>(last_done - t0, reqs[0].arrival_ns) : 0);
    stats->max_inflight = max_inflight;
    stats->max_region_bytes = arena.high;
    stats->max_poll_gap_ns = max_gap;
    stats->max_poll_gap_at_ns = max_gap_at;
    stats->status = result;
  }
  return result;
}

hicr_status hicr_serve_digests(hicr_instance_t h, hicr_serve_t s, const hicr_serve_request_t* reqs, uint64_t n,
                               hicr_serve_result_t* results) {
  Instance* in = I(h);
  if (!in || (n && (!reqs || !results))) return HICR_ERR_INVALID;
  Server* sv = srv_get(in, s);
  if (!sv || sv->kept.size() != n) return HICR_ERR_INVALID;
  bool any = false;
  for (uint64_t r = 0; r < n; ++r) any = any || (reqs[r].kind == 0 && sv->kept[r]);
  if (!any && !sv->cfg.verify) return HICR_ERR_INVALID;
  std::vector<VerifyItem> items;
  for (uint64_t r = 0; r < n; ++r) {
    if (reqs[r].kind != 0 || !sv->kept[r]) continue;
    const unsigned t = reqs[r].tmpl;
    if (t >= sv->t_nops.size()) return HICR_ERR_INVALID;
    for (uint64_t k = 0; k < sv->t_nops[t]; ++k) {
      const hicr_op_t& o = sv->tops[sv->t_opbase[t] + k];
      items.push_back({(unsigned long long)(sv->arena + results[r].dst_offset + o.dst_off), o.n, r, k});
    }
  }
  VerifyItem* d_items = nullptr;
  unsigned long long* d_out = nullptr;
  HICR_CUDA(in, cudaMalloc(&d_items, sizeof(VerifyItem) * std::max<size_t>(1, items.size())));
  cudaError_t e = cudaMalloc(&d_out, 8 * std::max<uint64_t>(1, n));
  if (e != cudaSuccess) {
    cudaFree(d_items);
    return cuda_fail(in, e, "cudaMalloc");
  }
  cudaStream_t cs = in->comm();
  std::vector<unsigned long long> out(n, 0);
  e = cudaMemcpyAsync(d_items, items.data(), sizeof(VerifyItem) * items.size(), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, 8 * std::max<uint64_t>(1, n), cs);
  if (e == cudaSuccess && !items.empty()) {
    k_serve_verify<<<in->sm_count * 8, 256, 0, cs>>>(d_items, items.size(), d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), d_out, 8 * n, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  cudaFree(d_items);
  cudaFree(d_out);
  if (e != cudaSuccess) return cuda_fail(in, e, "serve digests");
  for (uint64_t r = 0; r < n; ++r)
    if (reqs[r].kind == 0 && sv->kept[r]) results[r].digest = out[r];
  return HICR_OK;
}

}  // extern "C"
