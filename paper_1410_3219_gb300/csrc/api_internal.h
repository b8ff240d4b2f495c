// Helpers shared by the C ABI implementations (single simulation and batch):
// per-thread error text, CUDA error mapping, growable device buffers.
#pragma once

#include <chrono>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rich.h"

namespace rich {

int set_error(int code, const std::string &msg);

#define RICH_CUDA_TRY(expr)                                                                       \
    do {                                                                                          \
        cudaError_t err_ = (expr);                                                                \
        if (err_ != cudaSuccess)                                                                  \
            return ::rich::set_error(err_ == cudaErrorMemoryAllocation ? RICH_ENOMEM : RICH_ECUDA, \
                                     std::string(#expr) + ": " + cudaGetErrorString(err_));       \
    } while (0)

// Device allocation that only grows (25% headroom), freed with the owner.
struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf()
    {
        if (p) cudaFree(p);
    }
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes + bytes / 4 + 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Page-locked host memory: copies to and from it run at the link's speed
// and can run beside kernels (grown like DBuf; freed with the handle).
struct HBuf {
    void *p = nullptr;
    size_t cap = 0;
    HBuf() = default;
    HBuf(const HBuf &) = delete;
    HBuf &operator=(const HBuf &) = delete;
    ~HBuf()
    {
        if (p) cudaFreeHost(p);
    }
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= cap && p) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMallocHost(&p, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

template <class T> cudaError_t upload(DBuf &b, const std::vector<T> &v, cudaStream_t st)
{
    cudaError_t e = b.ensure(sizeof(T) * (v.size() + 1));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
}

// NVTX range for the host phases of a step (tessellation, uploads, sweep
// launch, synchronisation), visible to profilers that record NVTX; the calls
// do nothing when no profiler is attached.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

inline double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool valid_config(const rich_config *c);

class ThreadPool;
// rich_batch_create whose host work runs on a pool shared with other
// batches (nullptr: its own pool of host_threads threads)
int batch_create(int32_t precision, int64_t max_cells, int32_t host_threads, ThreadPool *shared, rich_batch **out);
bool point_inside(const rich_config *c, double x, double y);

// dst[f * n + perm[k]] = src[f][k] for the six fields (null sources skipped)
cudaError_t launch_unpermute(int32_t n, const int32_t *perm, const double *const src[6], double *dst,
                             cudaStream_t st);

}  // namespace rich
