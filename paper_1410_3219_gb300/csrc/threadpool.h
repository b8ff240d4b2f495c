// A small persistent worker pool for the host side of batched steps: the
// tessellation (a0) of independent simulations runs on all host cores while
// the device sweeps.  parallel_for hands out task indices dynamically (an
// atomic counter), so instances of very different sizes balance.
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
            stop_ = true;
            gen_++;
        }
        cv_.notify_all();
        for (auto &w : workers_) w.join();
    }

    int size() const { return (int)workers_.size() + 1; }

    // Run fn(i) for i in [0, n) on the pool and the calling thread; returns
    // when every task has finished.
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
            next_.store(0);
            active_ = (int)workers_.size();
            gen_++;
        }
        cv_.notify_all();
        run_tasks();
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [this] { return active_ == 0; });
        fn_ = nullptr;
    }

private:
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
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                if (stop_) return;
            }
            run_tasks();
            {
                std::lock_guard<std::mutex> lk(mu_);
                if (--active_ == 0) done_cv_.notify_one();
            }
        }
    }

    std::vector<std::thread> workers_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int64_t)> *fn_ = nullptr;
    int64_t n_ = 0;
    std::atomic<int64_t> next_{0};
    int active_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

}  // namespace rich
