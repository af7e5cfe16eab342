// Exercises HostPool (paper_2509_01425_gb300/csrc/host_pool.h) without a GPU:
// jobs back to back (workers spinning), jobs after the spin window (workers
// asleep on the condition variable), every part run exactly once, results
// visible to the caller after run(), and destruction with sleeping workers.
// Prints "ok" and exits 0, or prints the failure and exits 1.
#include <stdio.h>

#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "host_pool.h"

int main() {
  for (int threads : {1, 2, 3, 8}) {
    hicr::HostPool pool(threads);
    if (pool.size() != threads) {
      printf("size %d != %d\n", pool.size(), threads);
      return 1;
    }
    const uint64_t n = 100003;
    std::vector<uint32_t> hits(n);
    for (int job = 0; job < 200; ++job) {
      if (job == 100 || job == 150)  // let the workers fall asleep
        std::this_thread::sleep_for(std::chrono::nanoseconds(hicr::HostPool::kSpinNs + 20000000));
      std::atomic<int> calls{0};
      pool.run([&](int t, int nt) {
        calls.fetch_add(1);
        const uint64_t a = n * t / nt, b = n * (t + 1) / nt;
        for (uint64_t i = a; i < b; ++i) hits[i] += 1;  // plain writes, read by the caller after run()
      });
      if (calls.load() != threads) {
        printf("threads %d job %d: %d parts ran\n", threads, job, calls.load());
        return 1;
      }
      for (uint64_t i = 0; i < n; ++i) {
        if (hits[i] != (uint32_t)(job + 1)) {
          printf("threads %d job %d: index %llu hit %u times\n", threads, job, (unsigned long long)i, hits[i]);
          return 1;
        }
      }
    }
    std::this_thread::sleep_for(std::chrono::nanoseconds(hicr::HostPool::kSpinNs + 20000000));
  }  // destroyed with its workers asleep
  {
    hicr::HostPool pool(4);  // destroyed with its workers spinning
    pool.run([](int, int) {});
  }
  printf("ok\n");
  return 0;
}
