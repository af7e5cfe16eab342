/*
 * hicr_latency -- host-observed latency of small synchronous operations,
 * timed from C through the library's C ABI (no interpreter on the path).
 *
 *   hicr_latency [device] [reps]
 *
 * Each case runs `reps` times after reps / 10 untimed warm-up rounds and
 * prints one JSON object with p50 / p90 / p99 / max in microseconds:
 *   memcpy16_fence  hicr_memcpy of 16 bytes, then hicr_fence on its tag;
 *   fence_idle      hicr_fence with nothing outstanding;
 *   exec_await      hicr_exec_launch of the built-in digest unit over 16
 *                   bytes (1 CTA), then hicr_exec_await;
 *   spsc_push_pop   hicr_channel_push of one 64-byte token, then
 *                   hicr_channel_pop of it;
 *   dobj_get_fence  hicr_dobj_get of a 16-byte Data Object, then hicr_fence;
 *   memcpy16_fence_latency_mode, dobj_get_fence_latency_mode,
 *   spsc_push_pop_latency_mode
 *                   the same three with hicr_set_latency_mode on (a persistent
 *                   server kernel takes the small copies and the channel
 *                   calls; no launch per call).
 * Exit status 0 on success, 1 on any library error (its name is printed).
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "../include/hicr.h"
#include "../include/hicr_channels.h"
#include "../include/hicr_dataobject.h"

static uint64_t now_ns(void) {
  struct timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return (uint64_t)t.tv_sec * 1000000000ull + (uint64_t)t.tv_nsec;
}

static int cmp_u64(const void* a, const void* b) {
  const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : x > y;
}

#define CHECK(call)                                                              \
  do {                                                                           \
    hicr_status s_ = (call);                                                     \
    if (s_ != HICR_OK) {                                                         \
      fprintf(stderr, "hicr_latency: %s failed: %s\n", #call, hicr_status_str(s_)); \
      exit(1);                                                                   \
    }                                                                            \
  } while (0)

static void report(const char* name, uint64_t* t, int n, int last) {
  qsort(t, (size_t)n, sizeof(uint64_t), cmp_u64);
  printf("  \"%s\": {\"p50_us\": %.3f, \"p90_us\": %.3f, \"p99_us\": %.3f, \"max_us\": %.3f}%s\n", name,
         t[n / 2] / 1e3, t[(n * 9) / 10] / 1e3, t[(n * 99) / 100] / 1e3, t[n - 1] / 1e3, last ? "" : ",");
}

int main(int argc, char** argv) {
  const int dev = argc > 1 ? atoi(argv[1]) : 0;
  const int reps = argc > 2 ? atoi(argv[2]) : 2000;
  if (reps < 10) return 1;
  const int warm = reps / 10;
  uint64_t* t = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)reps);
  hicr_instance_t inst;
  CHECK(hicr_init(dev, &inst));
  hicr_slot_t a, b;
  CHECK(hicr_mem_alloc(inst, HICR_SPACE_HBM, 1 << 20, 0, &a));
  CHECK(hicr_mem_alloc(inst, HICR_SPACE_HBM, 1 << 20, 0, &b));
  const uint64_t fence_to = 10000000000ull;
  printf("{\n");

  for (int i = -warm; i < reps; ++i) {
    const uint64_t t0 = now_ns();
    CHECK(hicr_memcpy(inst, b, 64 * (uint64_t)(i & 1023), a, 16 * (uint64_t)(i & 4095), 16));
    CHECK(hicr_fence(inst, 0, fence_to));
    if (i >= 0) t[i] = now_ns() - t0;
  }
  report("memcpy16_fence", t, reps, 0);

  for (int i = -warm; i < reps; ++i) {
    const uint64_t t0 = now_ns();
    CHECK(hicr_fence(inst, 0, fence_to));
    if (i >= 0) t[i] = now_ns() - t0;
  }
  report("fence_idle", t, reps, 0);

  {
    hicr_exec_unit_t u;
    CHECK(hicr_exec_unit_builtin("digest_words", &u));
    u.grid[0] = 1;
    u.block[0] = 32;
    void* pa = NULL;
    CHECK(hicr_slot_info(inst, a, &pa, NULL, NULL, NULL));
    void* pb = NULL;
    CHECK(hicr_slot_info(inst, b, &pb, NULL, NULL, NULL));
    const uint8_t* p = (const uint8_t*)pa;
    uint64_t n = 16;
    uint64_t* out = (uint64_t*)pb;
    void* args[] = {&p, &n, &out};
    hicr_pu_t pu;
    CHECK(hicr_pu_create(inst, NULL, &pu));
    for (int i = -warm; i < reps; ++i) {
      const uint64_t t0 = now_ns();
      hicr_exec_t e;
      CHECK(hicr_exec_launch(inst, pu, &u, args, &e));
      CHECK(hicr_exec_await(inst, e, fence_to));
      if (i >= 0) t[i] = now_ns() - t0;
    }
    report("exec_await", t, reps, 0);
    CHECK(hicr_pu_destroy(inst, pu));
  }

  {
    hicr_channel_t ch;
    CHECK(hicr_spsc_create(inst, 64, 1024, &ch));
    for (int i = -warm; i < reps; ++i) {
      const uint64_t t0 = now_ns();
      CHECK(hicr_channel_push(inst, ch, 0, a, 64 * (uint64_t)(i & 1023), 1));
      CHECK(hicr_channel_pop(inst, ch, 1));
      if (i >= 0) t[i] = now_ns() - t0;
    }
    report("spsc_push_pop", t, reps, 0);
    CHECK(hicr_channel_destroy(inst, ch));
  }

  {
    uint64_t id;
    CHECK(hicr_dobj_publish(inst, a, 4096, 16, &id));
    hicr_dobj_handle_t hd;
    CHECK(hicr_dobj_get_handle(inst, id, &hd));
    for (int i = -warm; i < reps; ++i) {
      const uint64_t t0 = now_ns();
      CHECK(hicr_dobj_get(inst, &hd, b, 16 * (uint64_t)(i & 4095)));
      CHECK(hicr_fence(inst, 0, fence_to));
      if (i >= 0) t[i] = now_ns() - t0;
    }
    report("dobj_get_fence", t, reps, 0);

    CHECK(hicr_set_latency_mode(inst, 2000));
    for (int i = -warm; i < reps; ++i) {
      const uint64_t t0 = now_ns();
      CHECK(hicr_memcpy(inst, b, 64 * (uint64_t)(i & 1023), a, 16 * (uint64_t)(i & 4095), 16));
      CHECK(hicr_fence(inst, 0, fence_to));
      if (i >= 0) t[i] = now_ns() - t0;
    }
    report("memcpy16_fence_latency_mode", t, reps, 0);
    for (int i = -warm; i < reps; ++i) {
      const uint64_t t0 = now_ns();
      CHECK(hicr_dobj_get(inst, &hd, b, 16 * (uint64_t)(i & 4095)));
      CHECK(hicr_fence(inst, 0, fence_to));
      if (i >= 0) t[i] = now_ns() - t0;
    }
    report("dobj_get_fence_latency_mode", t, reps, 0);
    hicr_channel_t ch;
    CHECK(hicr_spsc_create(inst, 64, 1024, &ch));
    for (int i = -warm; i < reps; ++i) {
      const uint64_t t0 = now_ns();
      CHECK(hicr_channel_push(inst, ch, 0, a, 64 * (uint64_t)(i & 1023), 1));
      CHECK(hicr_channel_pop(inst, ch, 1));
      if (i >= 0) t[i] = now_ns() - t0;
    }
    report("spsc_push_pop_latency_mode", t, reps, 1);
    CHECK(hicr_channel_destroy(inst, ch));
    CHECK(hicr_set_latency_mode(inst, 0));
    CHECK(hicr_dobj_release(inst, id));
  }
  printf("}\n");
  CHECK(hicr_mem_free(inst, a));
  CHECK(hicr_mem_free(inst, b));
  CHECK(hicr_finalize(inst));
  free(t);
  return 0;
}
