// A small pool of host worker threads for the host side of large batches
// (validating and staging op tables). A job runs on every worker and on the
// calling thread, each taking the part of the range its index selects, and
// run() returns when all parts are done.
//
// Between jobs a worker spins (yielding) for up to kSpinNs before it blocks
// on a condition variable: batches issued back to back, one fence apart,
// then find the workers awake. A worker that had to be woken from the
// condition variable costs tens of microseconds, which is what an OpenMP team
// put to sleep during a fence wait cost per batch.
#pragma once

#include <stdint.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace hicr {

class HostPool {
 public:
  static constexpr uint64_t kSpinNs = 5000000;  // 5 ms

  explicit HostPool(int threads) : n_(threads < 1 ? 1 : threads) {
    for (int i = 1; i < n_; ++i) th_.emplace_back([this, i] { work(i); });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_.store(true, std::memory_order_release);
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  HostPool(const HostPool&) = delete;
  HostPool& operator=(const HostPool&) = delete;

  int size() const { return n_; }

  // f(t, n) for t = 0 .. n-1 (t = 0 on the calling thread); one job at a time.
  void run(const std::function<void(int, int)>& f) {
    job_ = &f;
    pending_.store(n_ - 1, std::memory_order_relaxed);
    {
      std::lock_guard<std::mutex> lk(m_);
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    f(0, n_);
    while (pending_.load(std::memory_order_acquire) != 0) std::this_thread::yield();
    job_ = nullptr;
  }

 private:
  static uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
  }

  void work(int id) {
    uint64_t seen = 0;
    for (;;) {
      const uint64_t t0 = now_ns();
      while (gen_.load(std::memory_order_acquire) == seen && !stop_.load(std::memory_order_acquire)) {
        if (now_ns() - t0 > kSpinNs) {
          std::unique_lock<std::mutex> lk(m_);
          cv_.wait(lk, [&] {
            return gen_.load(std::memory_order_acquire) != seen || stop_.load(std::memory_order_acquire);
          });
          break;
        }
        std::this_thread::yield();
      }
      if (stop_.load(std::memory_order_acquire)) return;
      seen = gen_.load(std::memory_order_acquire);
      (*job_)(id, n_);
      pending_.fetch_sub(1, std::memory_order_acq_rel);
    }
  }

  const int n_;
  std::vector<std::thread> th_;
  std::mutex m_;
  std::condition_variable cv_;
  std::atomic<uint64_t> gen_{0};
  std::atomic<int> pending_{0};
  std::atomic<bool> stop_{false};
  const std::function<void(int, int)>* job_ = nullptr;
};

}  // namespace hicr
