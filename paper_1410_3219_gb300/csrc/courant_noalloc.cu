// Courant time step over caller-owned device arrays, without allocating.
//
// Some callers cannot allocate GPU memory at the point where they need a
// time step: code running inside a memory pool or arena that owns the whole
// device, code that must not synchronise the device (cudaMalloc/cudaFree
// can), and code that is later replayed from a recorded sequence of
// launches. This entry point gives them the time step of the sweep without
// any allocation: its scratch (one partial minimum per thread block and a
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

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = RICH_NOALLOC_MAX_CELLS / kBlock;

// scratch: per-block minima of the cell time step (as bit patterns of
// non-negative doubles, whose integer order is their numeric order), then
// the number of blocks that have finished
static __device__ __align__(256) unsigned long long g_courant_scratch[kMaxBlocks + 1];

__global__ void k_courant_noalloc(int32_t n, double gamma, double cfl, int32_t motion_static,
                                  const double *__restrict__ area, const double *__restrict__ rho,
                                  const double *__restrict__ vx, const double *__restrict__ vy,
                                  const double *__restrict__ p, const double *__restrict__ wx,
                                  const double *__restrict__ wy, unsigned long long *scratch, double *dt_out)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = DBL_MAX;
    if (i < n) {
        const double cs = sqrt(gamma * p[i] / rho[i]);
        const double R = sqrt(area[i] * (1.0 / M_PI));
        const double ux = motion_static ? vx[i] : vx[i] - wx[i];
        const double uy = motion_static ? vy[i] : vy[i] - wy[i];
        v = R / (cs + sqrt(ux * ux + uy * uy));
    }
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    __shared__ double red[kBlock / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int k = 1; k < kBlock / 32; k++) m = fmin(m, red[k]);
        scratch[blockIdx.x] = (unsigned long long)__double_as_longlong(m);
        __threadfence();
        unsigned long long done = atomicAdd(&scratch[kMaxBlocks], 1ull);
        last = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block to finish reduces the per-block minima
    __threadfence();
    double m = DBL_MAX;
    for (int32_t b = threadIdx.x; b < (int32_t)gridDim.x; b += blockDim.x)
        m = fmin(m, __longlong_as_double((long long)((volatile unsigned long long *)scratch)[b]));
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) red[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = red[0];
        for (int k = 1; k < kBlock / 32; k++) r = fmin(r, red[k]);
        *dt_out = cfl * r;
    }
}

std::mutex g_setup_mutex;
unsigned long long *g_scratch_addr[64] = {};

}  // namespace

extern "C" int rich_courant_dt_noalloc(const rich_config *cfg, int64_t n, const double *area, const double *rho,
                                       const double *vx, const double *vy, const double *p, const double *wx,
                                       const double *wy, double *dt_out, void *stream)
{
    if (!cfg || !area || !rho || !vx || !vy || !p || !dt_out) return RICH_EINVAL;
    if (cfg->motion != RICH_MESH_EULERIAN && (!wx || !wy)) return RICH_EINVAL;
    if (n < 1 || n > RICH_NOALLOC_MAX_CELLS) return RICH_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RICH_ECUDA;
    unsigned long long *scratch;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_courant_scratch) != cudaSuccess || !ptr) return RICH_ECUDA;
            g_scratch_addr[dev] = static_cast<unsigned long long *>(ptr);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = (int)((n + kBlock - 1) / kBlock);
    // the completion counter must start at zero on every call
    if (cudaMemsetAsync(scratch + kMaxBlocks, 0, sizeof(unsigned long long), st) != cudaSuccess) return RICH_ECUDA;
    k_courant_noalloc<<<blocks, kBlock, 0, st>>>((int32_t)n, cfg->gamma, cfg->cfl,
                                                 cfg->motion == RICH_MESH_EULERIAN ? 1 : 0, area, rho, vx, vy, p,
                                                 wx, wy, scratch, dt_out);
    return cudaGetLastError() == cudaSuccess ? RICH_OK : RICH_ECUDA;
}
