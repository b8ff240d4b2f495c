// A small persistent worker pool for the host side of the steps: the
// tessellation (a0) tiles of one simulation, or the independent
// simulations of a batch, run on all host cores.  parallel_for hands out
// task indices dynamically (an atomic counter), so tasks of very different
// sizes balance.  A build issues a dozen short parallel passes, so the
// workers poll for the next batch of tasks for a short while before they
// sleep, and the caller polls for their completion: waking sleeping
// threads through a condition variable costs tens of microseconds a pass.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace rich {

class ThreadPool {
public:
    explicit ThreadPool(int nthreads)
    {
        if (nthreads < 1) nthreads = 1;
        for (int t = 1; t < nthreads; t++) workers_.emplace_back([this] { loop(); });
    }

    ~ThreadPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_.store(true, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        for (auto &w : workers_) w.join();
    }

    int size() const { return (int)workers_.size() + 1; }

    // Run fn(i) for i in [0, n) on the pool and the calling thread; returns
    // when every task has finished.  Every worker takes part in every call
    // (it may find no task left), and the next call starts only after all
    // of them have left this one.
    void parallel_for(int64_t n, const std::function<void(int64_t)> &fn)
    {
        if (n <= 0) return;
        if (workers_.empty() || n == 1) {
            for (int64_t i = 0; i < n; i++) fn(i);
            return;
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            fn_ = &fn;
            n_ = n;
            next_.store(0, std::memory_order_relaxed);
            active_.store((int)workers_.size(), std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        run_tasks();
        while (active_.load(std::memory_order_acquire) != 0) std::this_thread::yield();
        fn_ = nullptr;
    }

private:
    // polls of the generation before a worker sleeps (tens of microseconds)
    static constexpr int kSpin = 1 << 14;

    void run_tasks()
    {
        for (;;) {
            int64_t i = next_.fetch_add(1);
            if (i >= n_) break;
            (*fn_)(i);
        }
    }

    void loop()
    {
        uint64_t seen = 0;
        for (;;) {
            bool woke = false;
            for (int i = 0; i < kSpin && !woke; i++) woke = gen_.load(std::memory_order_acquire) != seen;
            if (!woke) {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
            }
            seen = gen_.load(std::memory_order_acquire);
            if (stop_.load(std::memory_order_relaxed)) return;
            run_tasks();
            active_.fetch_sub(1, std::memory_order_acq_rel);
        }
    }

    std::vector<std::thread> workers_;
    std::mutex mu_;
    std::condition_variable cv_;
    const std::function<void(int64_t)> *fn_ = nullptr;
    int64_t n_ = 0;
    std::atomic<int64_t> next_{0};
    std::atomic<int> active_{0};
    std::atomic<uint64_t> gen_{0};
    std::atomic<bool> stop_{false};
};

}  // namespace rich
