// Reordering of per-cell device arrays into the caller's order, so that a
// read of the state is a device gather and plain copies (no per-cell host
// work).
#include <cstdint>

#include <cuda_runtime.h>

namespace rich {
namespace {

// dst[f * n + perm[k]] = src_f[k] for the fields f < nf (null sources are
// skipped): perm[k] is the caller's index of internal cell k
__global__ void k_unpermute(int32_t n, const int32_t *__restrict__ perm, const double *s0, const double *s1,
                            const double *s2, const double *s3, const double *s4, const double *s5, double *dst)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t u = perm[k];
    const double *src[6] = {s0, s1, s2, s3, s4, s5};
#pragma unroll
    for (int f = 0; f < 6; f++)
        if (src[f]) dst[(int64_t)f * n + u] = src[f][k];
}

}  // namespace

cudaError_t launch_unpermute(int32_t n, const int32_t *perm, const double *const src[6], double *dst,
                             cudaStream_t st)
{
    if (n > 0)
        k_unpermute<<<(n + 255) / 256, 256, 0, st>>>(n, perm, src[0], src[1], src[2], src[3], src[4], src[5], dst);
    return cudaGetLastError();
}

}  // namespace rich
