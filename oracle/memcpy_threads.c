/*
 * CPU baseline for batched memcpy on all host cores -- TEST AND CPU-BASELINE
 * INFRASTRUCTURE ONLY (never part of the library's product path).
 *
 * What it computes: the local-to-local memcpy of the HiCR communication
 * manager (paper Sec. 3.1.4; Sec. 4.2 notes that such copies are typically a
 * plain memcpy), applied to a table of already validated, hazard-free ops,
 * one fence epoch after another. Within an epoch the ops are unordered
 * (their destinations overlap nothing the epoch reads or writes), so the
 * epoch's bytes, taken in table order as one stream, are cut into `threads`
 * equal byte ranges and each thread copies its range with memcpy. Threads
 * are joined at the end of every epoch (the fence).
 *
 * It is the "CPU on all cores" line beside the single-threaded oracle; its
 * results are compared with the oracle's in the CPU tests.
 */
#include <pthread.h>
#include <stdint.h>
#include <string.h>

typedef struct {
  uint32_t dst, src;
  uint64_t dst_off, src_off, n;
} mt_op_t; /* the 32-byte op record */

typedef struct {
  uint8_t* const* slots;
  const mt_op_t* ops;
  const uint64_t* prefix; /* prefix[i] = bytes of ops [a, a+i) of the epoch */
  uint64_t a, count;      /* the epoch: ops [a, a + count) */
  uint64_t lo, hi;        /* this thread's byte range of the epoch stream */
} mt_job_t;

static void* mt_run(void* arg) {
  const mt_job_t* j = (const mt_job_t*)arg;
  if (j->lo >= j->hi) return NULL;
  /* first op whose bytes end after lo */
  uint64_t l = 0, r = j->count;
  while (l < r) {
    const uint64_t m = (l + r) / 2;
    if (j->prefix[m + 1] <= j->lo) l = m + 1;
    else r = m;
  }
  for (uint64_t i = l; i < j->count && j->prefix[i] < j->hi; ++i) {
    const mt_op_t* o = j->ops + j->a + i;
    const uint64_t b0 = j->prefix[i] > j->lo ? j->prefix[i] : j->lo;
    const uint64_t b1 = j->prefix[i + 1] < j->hi ? j->prefix[i + 1] : j->hi;
    if (b1 <= b0) continue;
    const uint64_t k = b0 - j->prefix[i];
    memcpy(j->slots[o->dst] + o->dst_off + k, j->slots[o->src] + o->src_off + k, b1 - b0);
  }
  return NULL;
}

/* Apply ops epoch by epoch: epoch e is ops [epoch_start[e], epoch_start[e+1]).
 * `prefix_scratch` holds at least (largest epoch + 1) entries. Returns 0, or
 * -1 when a thread could not be started (the epoch is then finished on the
 * calling thread). */
int mt_memcpy_epochs(uint8_t* const* slots, const mt_op_t* ops, const uint64_t* epoch_start, int n_epochs,
                     int threads, uint64_t* prefix_scratch) {
  enum { MAXT = 512 };
  pthread_t tid[MAXT];
  mt_job_t job[MAXT];
  int rc = 0;
  if (threads < 1) threads = 1;
  if (threads > MAXT) threads = MAXT;
  for (int e = 0; e < n_epochs; ++e) {
    const uint64_t a = epoch_start[e], count = epoch_start[e + 1] - a;
    prefix_scratch[0] = 0;
    for (uint64_t i = 0; i < count; ++i) prefix_scratch[i + 1] = prefix_scratch[i] + ops[a + i].n;
    const uint64_t total = prefix_scratch[count];
    int started = 0;
    for (int t = 0; t < threads; ++t) {
      job[t].slots = slots;
      job[t].ops = ops;
      job[t].prefix = prefix_scratch;
      job[t].a = a;
      job[t].count = count;
      job[t].lo = total * (uint64_t)t / (uint64_t)threads;
      job[t].hi = total * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    for (int t = 1; t < threads; ++t) {
      if (pthread_create(&tid[t], NULL, mt_run, &job[t]) != 0) break;
      ++started;
    }
    mt_run(&job[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    if (started < threads - 1) {
      rc = -1;
      for (int t = started + 1; t < threads; ++t) mt_run(&job[t]);
    }
  }
  return rc;
}
