// Courant time step over caller-owned device arrays, without allocating.
//
// Some callers cannot allocate GPU memory at the point where they need a
// time step: code running inside a memory pool or arena that owns the whole
// device, and code that must not synchronise the device (cudaMalloc/cudaFree
// can).  This entry point gives them the time step of the sweep without any
// allocation: its scratch (one partial minimum per thread block and a
// completion counter) lives in a file-scope __device__ array that every
// process loading the library holds on every GPU it uses, until exit.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (in host code the array's name is only a
// host-side stand-in); make that first call before any stream capture.
// Calls share the array: calls that overlap on the GPU (different streams,
// or different host threads) race and must not be issued.
#include <cfloat>
#include <cmath>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/rich.h"
#include "api_internal.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = RICH_NOALLOC_MAX_CELLS / kBlock;

// scratch: per-block minima of the cell time step as bit patterns (the
// integer order of non-negative doubles is their numeric order; kBad marks
// a block that met a cell whose time step is not a finite non-negative
// number), then the number of blocks that have finished
static __device__ __align__(256) unsigned long long g_courant_scratch[kMaxBlocks + 1];

constexpr unsigned long long kBad = ~0ull;

// The cell time step's bits as the sweep's own reduction orders them: a
// non-negative double's bits; -0.0, negative values and NaNs (negative as an
// integer, or above the bits of +inf) are flagged instead of being skipped.
__device__ __forceinline__ unsigned long long step_key(double v, bool &bad)
{
    const long long k = __double_as_longlong(v);
    if (k < 0 || k > 0x7ff0000000000000ll) {
        bad = true;
        return kBad;
    }
    return (unsigned long long)k;
}

__device__ __forceinline__ unsigned long long key_min(unsigned long long a, unsigned long long b)
{
    return a < b ? a : b;
}

__global__ void k_courant_noalloc(int32_t n, double gamma, double cfl, int32_t motion_static,
                                  const double *__restrict__ area, const double *__restrict__ rho,
                                  const double *__restrict__ vx, const double *__restrict__ vy,
                                  const double *__restrict__ p, const double *__restrict__ wx,
                                  const double *__restrict__ wy, unsigned long long *scratch, double *dt_out)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    // kMax: the bits of +inf, above every finite non-negative time step
    const unsigned long long kMax = 0x7ff0000000000000ull;
    unsigned long long k = kMax;
    bool bad = false;
    if (i < n) {
        const double cs = sqrt(gamma * p[i] / rho[i]);
        const double R = sqrt(area[i] * (1.0 / M_PI));
        const double ux = motion_static ? vx[i] : vx[i] - wx[i];
        const double uy = motion_static ? vy[i] : vy[i] - wy[i];
        k = step_key(R / (cs + sqrt(ux * ux + uy * uy)), bad);
    }
    bad = __any_sync(0xffffffffu, bad);
    for (int o = 16; o > 0; o >>= 1) k = key_min(k, __shfl_down_sync(0xffffffffu, k, o));
    __shared__ unsigned long long red[kBlock / 32];
    __shared__ int bad_block;
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) bad_block = 0;
    __syncthreads();
    if (lane == 0) {
        red[wid] = k;
        if (bad) bad_block = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = red[0];
        for (int q = 1; q < kBlock / 32; q++) m = key_min(m, red[q]);
        scratch[blockIdx.x] = bad_block ? kBad : m;
        __threadfence();
        unsigned long long done = atomicAdd(&scratch[kMaxBlocks], 1ull);
        last = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block to finish reduces the per-block minima
    __threadfence();
    unsigned long long m = kMax;
    bool any_bad = false;
    for (int32_t b = threadIdx.x; b < (int32_t)gridDim.x; b += blockDim.x) {
        const unsigned long long v = ((volatile unsigned long long *)scratch)[b];
        if (v == kBad) any_bad = true;
        else m = key_min(m, v);
    }
    any_bad = __any_sync(0xffffffffu, any_bad);
    for (int o = 16; o > 0; o >>= 1) m = key_min(m, __shfl_down_sync(0xffffffffu, m, o));
    __syncthreads();
    if (threadIdx.x == 0) bad_block = 0;
    __syncthreads();
    if (lane == 0) {
        red[wid] = m;
        if (any_bad) bad_block = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long r = red[0];
        for (int q = 1; q < kBlock / 32; q++) r = key_min(r, red[q]);
        *dt_out = bad_block ? __longlong_as_double(0x7ff8000000000000ll) : cfl * __longlong_as_double((long long)r);
    }
}

std::mutex g_setup_mutex;
unsigned long long *g_scratch_addr[64] = {};

}  // namespace

extern "C" int rich_courant_dt_noalloc(const rich_config *cfg, int64_t n, const double *area, const double *rho,
                                       const double *vx, const double *vy, const double *p, const double *wx,
                                       const double *wy, double *dt_out, void *stream)
{
    if (!rich::valid_config(cfg)) return rich::set_error(RICH_EINVAL, "invalid configuration");
    if (!area || !rho || !vx || !vy || !p || !dt_out) return rich::set_error(RICH_EINVAL, "NULL array");
    if (cfg->motion != RICH_MESH_EULERIAN && (!wx || !wy))
        return rich::set_error(RICH_EINVAL, "wx, wy are needed with a moving mesh");
    if (n < 1 || n > RICH_NOALLOC_MAX_CELLS)
        return rich::set_error(RICH_EINVAL, "n must be in [1, RICH_NOALLOC_MAX_CELLS]: the fixed scratch holds one "
                                            "partial minimum per 256 cells");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return rich::set_error(RICH_ECUDA, "no device");
    unsigned long long *scratch;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_courant_scratch) != cudaSuccess || !ptr)
                return rich::set_error(RICH_ECUDA, "cudaGetSymbolAddress failed for the scratch array");
            g_scratch_addr[dev] = static_cast<unsigned long long *>(ptr);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = (int)((n + kBlock - 1) / kBlock);
    // the completion counter must start at zero on every call
    if (cudaMemsetAsync(scratch + kMaxBlocks, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return rich::set_error(RICH_ECUDA, "cudaMemsetAsync failed");
    k_courant_noalloc<<<blocks, kBlock, 0, st>>>((int32_t)n, cfg->gamma, cfg->cfl,
                                                 cfg->motion == RICH_MESH_EULERIAN ? 1 : 0, area, rho, vx, vy, p,
                                                 wx, wy, scratch, dt_out);
    return cudaGetLastError() == cudaSuccess ? RICH_OK : rich::set_error(RICH_ECUDA, "launch failed");
}
