// A small persistent worker pool for the host side of the steps: the
// tessellation (a0) tiles of one simulation, or the independent
// simulations of a batch, run on all host cores.  parallel_for hands out
// task indices dynamically (an atomic counter), so tasks of very different
// sizes balance.  A build issues a dozen short parallel passes, so the
// workers poll for new tasks for a short while before they sleep, and the
// caller polls for the completion of its own tasks: waking sleeping threads
// through a condition variable costs tens of microseconds a pass.
//
// Several threads may call parallel_for at once (the server's lanes share
// one pool): each call is a group of tasks, the workers take tasks from the
// group of the highest priority with tasks left (the calling thread's, set
// by set_priority; the oldest first among equals), a group's caller works
// only on its own group, and a call returns when its group is done.  So a
// long task of one caller (a whole simulation tessellated on one thread)
// holds one worker, not the pool, while another caller's tiles run on the
// rest.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <memory>
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
            posted_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        for (auto &w : workers_) w.join();
    }

    int size() const { return (int)workers_.size() + 1; }

    // Priority of the groups the calling thread posts from now on (0 by
    // default; higher first).
    static void set_priority(int p) { caller_priority() = p; }

    // Run fn(i) for i in [0, n) on the pool and the calling thread; returns
    // when every task of this call has finished.
    void parallel_for(int64_t n, const std::function<void(int64_t)> &fn)
    {
        if (n <= 0) return;
        if (workers_.empty() || n == 1) {
            for (int64_t i = 0; i < n; i++) fn(i);
            return;
        }
        auto g = std::make_shared<Group>();
        g->fn = &fn;
        g->n = n;
        g->priority = caller_priority();
        {
            std::lock_guard<std::mutex> lk(mu_);
            groups_.push_back(g);
            posted_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        run_group(*g);
        // the other tasks of the group may still run on workers
        while (g->done.load(std::memory_order_acquire) != n) std::this_thread::yield();
        std::lock_guard<std::mutex> lk(mu_);
        for (size_t k = 0; k < groups_.size(); k++)
            if (groups_[k] == g) {
                groups_.erase(groups_.begin() + k);
                break;
            }
    }

private:
    struct Group {
        const std::function<void(int64_t)> *fn = nullptr;
        int64_t n = 0;
        int priority = 0;
        std::atomic<int64_t> next{0}, done{0};
    };

    static int &caller_priority()
    {
        thread_local int p = 0;
        return p;
    }

    // polls for new tasks before a worker sleeps (tens of microseconds)
    static constexpr int kSpin = 1 << 14;

    static bool run_one(Group &g)
    {
        const int64_t i = g.next.fetch_add(1, std::memory_order_relaxed);
        if (i >= g.n) return false;
        (*g.fn)(i);
        g.done.fetch_add(1, std::memory_order_acq_rel);
        return true;
    }

    static void run_group(Group &g)
    {
        while (run_one(g)) {
        }
    }

    // the group of the highest priority with a task left (the oldest among
    // equals), or null
    std::shared_ptr<Group> pick()
    {
        std::lock_guard<std::mutex> lk(mu_);
        std::shared_ptr<Group> best;
        for (auto &g : groups_)
            if (g->next.load(std::memory_order_relaxed) < g->n && (!best || g->priority > best->priority)) best = g;
        return best;
    }

    void loop()
    {
        uint64_t seen = 0;
        for (;;) {
            if (stop_.load(std::memory_order_relaxed)) return;
            std::shared_ptr<Group> g = pick();
            if (g) {
                run_one(*g);
                continue;
            }
            bool woke = false;
            for (int i = 0; i < kSpin && !woke; i++) woke = posted_.load(std::memory_order_acquire) != seen;
            if (!woke) {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return posted_.load(std::memory_order_acquire) != seen; });
            }
            seen = posted_.load(std::memory_order_acquire);
        }
    }

    std::vector<std::thread> workers_;
    std::mutex mu_;  // the list of groups; the sleep of idle workers
    std::condition_variable cv_;
    std::vector<std::shared_ptr<Group>> groups_;
    std::atomic<uint64_t> posted_{0};  // bumped when a group is posted (and at shutdown)
    std::atomic<bool> stop_{false};
};

}  // namespace rich
