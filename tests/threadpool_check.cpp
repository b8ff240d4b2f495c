// Stress check of the host worker pool (csrc/threadpool.h): several threads
// call parallel_for at once with different priorities, tasks of very
// different lengths, nested calls from inside tasks, and single-task calls;
// every task of every call must run exactly once, and each call must return
// only after all of its tasks have finished.  Prints "ok" or the failure.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <thread>
#include <vector>

#include "../paper_1410_3219_gb300/csrc/threadpool.h"

int main()
{
    rich::ThreadPool pool(6);
    std::atomic<int> failures{0};
    auto caller = [&](int id) {
        rich::ThreadPool::set_priority(id % 3);
        for (int round = 0; round < 60; round++) {
            const int64_t n = 1 + (id * 37 + round * 11) % 97;
            std::vector<std::atomic<int>> hits(n);
            for (auto &h : hits) h.store(0);
            std::atomic<int64_t> finished{0};
            pool.parallel_for(n, [&](int64_t i) {
                if ((i + round) % 13 == 0) std::this_thread::sleep_for(std::chrono::microseconds(200));
                if (i == 3 && round % 5 == 0) {
                    // a nested call from inside a task
                    std::atomic<int> inner{0};
                    pool.parallel_for(17, [&](int64_t) { inner.fetch_add(1); });
                    if (inner.load() != 17) failures.fetch_add(1);
                }
                hits[i].fetch_add(1);
                finished.fetch_add(1);
            });
            if (finished.load() != n) failures.fetch_add(1);
            for (auto &h : hits)
                if (h.load() != 1) failures.fetch_add(1);
        }
    };
    std::vector<std::thread> callers;
    for (int id = 0; id < 4; id++) callers.emplace_back(caller, id);
    for (auto &t : callers) t.join();
    if (failures.load()) {
        std::printf("failures %d\n", failures.load());
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
