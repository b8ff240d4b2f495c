// Accuracy of the sweep's FP64 reciprocal and square root (fp64ops.cuh)
// against the IEEE-rounded 1/x and sqrt on the same GPU, and of its
// integer-pipe FP64 <-> FP32 conversions against the hardware's.  Prints one
// line "recip <max ulp> <mismatches in the fallback domain> sqrt <max ulp>
// <mismatches at zero> d2f <mismatches> f2d <mismatches>" and exits 0.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include <cuda_runtime.h>

#include "../paper_1410_3219_gb300/csrc/fp64ops.cuh"

__global__ void k_conv(const double *x, const unsigned *fb, int *bad, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = rich::d2f_rn(x[i]), b = __double2float_rn(x[i]);
    if (__float_as_uint(a) != __float_as_uint(b)) atomicAdd(bad, 1);
    const float f = __uint_as_float(fb[i]);
    const double c = rich::f2d(f), d = (double)f;
    if (__double_as_longlong(c) != __double_as_longlong(d)) atomicAdd(bad + 1, 1);
}

__global__ void k_ops(const double *x, double *r_fast, double *r_ieee, double *s_fast, double *s_ieee, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    r_fast[i] = rich::recip(v);
    r_ieee[i] = 1.0 / v;
    const double a = fabs(v);
    s_fast[i] = rich::sqrt_nonneg(a);
    s_ieee[i] = sqrt(a);
}

static double ulps(double a, double b)
{
    if (a == b) return 0.0;
    if (!std::isfinite(a) || !std::isfinite(b)) return INFINITY;
    const double u = std::fabs(std::nextafter(b, INFINITY) - b);
    return std::fabs(a - b) / u;
}

int main(int argc, char **argv)
{
    const int n = argc > 1 ? atoi(argv[1]) : (1 << 22);
    std::mt19937_64 g(20141012);
    std::uniform_real_distribution<double> mant(1.0, 2.0);
    std::uniform_int_distribution<int> ex(-1021, 1019), sgn(0, 1);
    std::vector<double> x(n);
    for (int i = 0; i < n; i++) x[i] = (sgn(g) ? -1.0 : 1.0) * std::ldexp(mant(g), ex(g));
    // the fallback domain and the ends of the fast one
    const double special[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 1e-310, -4e-320, DBL_MAX, -DBL_MAX,
                              std::ldexp(1.0, -1021), std::ldexp(1.0, -1022), std::ldexp(1.999, 1019),
                              std::ldexp(1.0, 1020), std::ldexp(1.0, 1021), 1.0, 3.0, 0.1};
    const int ns = (int)(sizeof(special) / sizeof(special[0]));
    for (int i = 0; i < ns && i < n; i++) x[i] = special[i];
    double *d[5];
    for (auto &p : d)
        if (cudaMalloc(&p, sizeof(double) * n) != cudaSuccess) return 2;
    cudaMemcpy(d[0], x.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    k_ops<<<(n + 255) / 256, 256>>>(d[0], d[1], d[2], d[3], d[4], n);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    std::vector<double> rf(n), ri(n), sf(n), si(n);
    cudaMemcpy(rf.data(), d[1], sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(ri.data(), d[2], sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(sf.data(), d[3], sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(si.data(), d[4], sizeof(double) * n, cudaMemcpyDeviceToHost);
    double r_max = 0.0, s_max = 0.0;
    long r_bad = 0, s_bad = 0;
    for (int i = 0; i < n; i++) {
        const int e = std::isfinite(x[i]) && x[i] != 0.0 ? std::ilogb(x[i]) : 99999;
        const bool fast = e >= -1021 && e <= 1019;
        if (fast) {
            r_max = std::fmax(r_max, ulps(rf[i], ri[i]));
        } else if (!(rf[i] == ri[i] || (std::isnan(rf[i]) && std::isnan(ri[i])))) {
            r_bad++;  // outside the refined range the IEEE division is taken
        }
        const double a = std::fabs(x[i]);
        if (std::isfinite(a) && a > 0.0) s_max = std::fmax(s_max, ulps(sf[i], si[i]));
        else if (a == 0.0 && sf[i] != 0.0) s_bad++;
    }
    // conversions: doubles of every exponent that matters to FP32 (normal,
    // subnormal, overflow and the rounding boundaries), and random FP32 bit
    // patterns (subnormals, inf and NaN included)
    std::vector<double> xc(n);
    std::vector<unsigned> fb(n);
    std::uniform_int_distribution<unsigned long long> bits64;
    std::uniform_int_distribution<unsigned> bits32;
    std::uniform_int_distribution<int> exf(-160, 140);
    for (int i = 0; i < n; i++) {
        double v = std::ldexp(mant(g), exf(g)) * (sgn(g) ? -1.0 : 1.0);
        if (i % 4 == 1) {
            // exact ties and their neighbours: 24 significant bits plus one
            unsigned long long b;
            std::memcpy(&b, &v, 8);
            b = (b & ~0x1fffffffull) | 0x10000000ull;
            b += (long long)(i % 3) - 1;
            std::memcpy(&v, &b, 8);
        }
        if (i % 4 == 2) {
            unsigned long long b = bits64(g);
            std::memcpy(&v, &b, 8);
        }
        xc[i] = v;
        fb[i] = bits32(g);
    }
    const double cs[] = {0.0, -0.0, FLT_MAX, -FLT_MAX, 3.4028235677973366e38, 3.4028235677973362e38, 1e39, FLT_MIN,
                         FLT_MIN * 0.5, 1e-46, INFINITY, -INFINITY, NAN, 1.0, 0.1};
    for (int i = 0; i < (int)(sizeof(cs) / sizeof(cs[0])) && i < n; i++) xc[i] = cs[i];
    int *dbad;
    unsigned *dfb;
    cudaMalloc(&dbad, 2 * sizeof(int));
    cudaMalloc(&dfb, sizeof(unsigned) * n);
    cudaMemset(dbad, 0, 2 * sizeof(int));
    cudaMemcpy(d[0], xc.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dfb, fb.data(), sizeof(unsigned) * n, cudaMemcpyHostToDevice);
    k_conv<<<(n + 255) / 256, 256>>>(d[0], dfb, dbad, n);
    if (cudaDeviceSynchronize() != cudaSuccess) return 4;
    int hbad[2];
    cudaMemcpy(hbad, dbad, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dbad);
    cudaFree(dfb);
    printf("recip %.3f %ld sqrt %.3f %ld d2f %d f2d %d\n", r_max, r_bad, s_max, s_bad, hbad[0], hbad[1]);
    for (auto &p : d) cudaFree(p);
    return 0;
}
