// Sweep kernels: steps a1-a9 of one extrapolated-fluxes time step of the
// moving Voronoi mesh scheme (paper Section 2), templated on the
// reconstruction precision R (double: all FP64; float: split precision).
//
// FP64 throughput on GB300 is ~1.2 TFLOP/s (2 FP64 lanes per clock per SM),
// so every FP64 quantity is computed once and kept in HBM for the next
// kernel (Voronoi vertices per triangle, edge geometry per edge, one HLLC
// flux per edge), divisions and square roots are not repeated, and the
// fluxes are gathered per cell in a fixed order (deterministic, no atomics).
// In the split instantiation only the geometry (positions, vertices, areas,
// centres of mass, coordinate differences) and the conserved variables with
// their flux accumulation are FP64; everything else runs on the FP32 pipe.
#include <cfloat>
#include <cmath>

#include "fp64ops.cuh"
#include "sweep.cuh"

namespace rich {
namespace {

constexpr int kBlock = 256;
// threads per block of the point motion (a light, memory-bound pass)
constexpr int kAdvanceBlock = 256;

// A per-simulation constant in the reconstruction precision (the FP32 copy
// rounded by the host: no conversion per thread)
template <class R> __device__ __forceinline__ R inst_value(double d, float f);
template <> __device__ __forceinline__ double inst_value<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float inst_value<float>(double, float f) { return f; }

template <class R> __device__ __forceinline__ double px_of(const SweepParams<R> &p, int32_t q)
{
    return q < p.n ? p.x[q] : p.gx[q - p.n];
}
template <class R> __device__ __forceinline__ double py_of(const SweepParams<R> &p, int32_t q)
{
    return q < p.n ? p.y[q] : p.gy[q - p.n];
}

template <class R> __device__ __forceinline__ int32_t inst_of(const SweepParams<R> &p, int32_t i)
{
    return p.cell_inst ? p.cell_inst[i] : 0;
}

// cell handled by thread k of a per-cell stage
template <class R> __device__ __forceinline__ int32_t cell_at(const SweepParams<R> &p, int32_t k)
{
    return p.cell_order ? __ldg(p.cell_order + k) : k;
}

// real cell behind point q and its mirror flags
template <class R> __device__ __forceinline__ int32_t src_of(const SweepParams<R> &p, int32_t q, int32_t &xf)
{
    if (q < p.n) { xf = 0; return q; }
    xf = p.ghost_xf[q - p.n];
    return p.ghost_src[q - p.n];
}

// v with its sign flipped where the mask has the sign bit (a mirror image's
// component), on the integer pipe instead of a multiply by -1 or 1
__device__ __forceinline__ double flip(double v, unsigned long long m)
{
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)m);
}
__device__ __forceinline__ float flip(float v, unsigned long long m)
{
    return __int_as_float(__float_as_int(v) ^ (int)(unsigned)(m >> 32));
}


template <class R> __device__ __forceinline__ Vec4<R> load_W(const SweepParams<R> &p, int32_t q)
{
    int32_t xf;
    int32_t k = src_of(p, q, xf);
    Vec4<R> W = p.W[k];
    W.y = flip(W.y, (xf & 1) ? 0x8000000000000000ull : 0ull);
    W.z = flip(W.z, (xf & 2) ? 0x8000000000000000ull : 0ull);
    return W;
}

// FP64 max/min on the integer pipe: the bits of a double, with the magnitude
// bits flipped for negative values, order like the doubles themselves
// (GB300 issues FP64 instructions, comparisons included, at 1/64 of the
// FP32 rate; 64-bit integer compares run on the integer pipe).
__device__ __forceinline__ long long dkey(double v)
{
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
// dkey with -0.0 taken as +0.0 (the only key of -1), so that the integer
// order matches the comparisons of doubles exactly
__device__ __forceinline__ long long dkey0(double v)
{
    const long long k = dkey(v);
    return k == -1 ? 0 : k;
}
__device__ __forceinline__ double dunkey(long long k)
{
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

template <class R> struct Extremes;
template <> struct Extremes<double> {
    long long hi, lo;
    __device__ __forceinline__ void init(double v) { hi = lo = dkey(v); }
    __device__ __forceinline__ void add(double v)
    {
        const long long k = dkey(v);
        hi = k > hi ? k : hi;
        lo = k < lo ? k : lo;
    }
    __device__ __forceinline__ double max() const { return dunkey(hi); }
    __device__ __forceinline__ double min() const { return dunkey(lo); }
    // max() > 0 and min() < 0 on the keys (the key of -0.0 is -1)
    __device__ __forceinline__ bool max_positive() const { return hi > 0; }
    __device__ __forceinline__ bool min_negative() const { return lo < -1; }
};
template <> struct Extremes<float> {
    float hi, lo;
    __device__ __forceinline__ void init(float v) { hi = lo = v; }
    __device__ __forceinline__ void add(float v)
    {
        hi = fmaxf(hi, v);
        lo = fminf(lo, v);
    }
    __device__ __forceinline__ float max() const { return hi; }
    __device__ __forceinline__ float min() const { return lo; }
    __device__ __forceinline__ bool max_positive() const { return hi > 0.0f; }
    __device__ __forceinline__ bool min_negative() const { return lo < 0.0f; }
};

// a < b for non-negative values (bit patterns of non-negative doubles order
// like the values)
__device__ __forceinline__ bool nonneg_less(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
// a < b for any non-NaN values, through order-preserving integer keys (-0.0
// and +0.0 equal), and the sign tests x >= 0 and x <= 0 likewise
__device__ __forceinline__ long long okey(double v) { return dkey0(v); }
__device__ __forceinline__ bool key_less(double a, double b) { return okey(a) < okey(b); }
__device__ __forceinline__ bool key_nonneg(double a) { return okey(a) >= 0; }
__device__ __forceinline__ bool key_nonpos(double a) { return okey(a) <= 0; }
// FP32 compares are cheap on their own pipe and give the same answers
__device__ __forceinline__ bool key_less(float a, float b) { return a < b; }
__device__ __forceinline__ bool key_nonneg(float a) { return a >= 0.0f; }
__device__ __forceinline__ bool key_nonpos(float a) { return a <= 0.0f; }
__device__ __forceinline__ bool nonneg_less(float a, float b) { return a < b; }

// Smallest non-negative cell time step of each simulation: a warp whose
// cells all belong to one simulation reduces first and issues one atomic;
// a mixed warp issues one atomic per lane.
// The minimum is taken on the bits: non-negative doubles order like their
// bit patterns, and a negative value, -0.0 or a negative NaN (negative as
// an integer) is mapped past every candidate, as are +inf and positive NaNs
// (above DBL_MAX's bits).
__device__ __forceinline__ void warp_min_to(double v, int32_t inst, unsigned long long *dst)
{
    const long long kmax = __double_as_longlong(DBL_MAX);
    long long k = __double_as_longlong(v);
    if (k < 0) k = kmax;
    const int32_t first = __shfl_sync(0xffffffffu, inst, 0);
    if (__all_sync(0xffffffffu, inst == first)) {
        for (int o = 16; o > 0; o >>= 1) {
            const long long q = __shfl_down_sync(0xffffffffu, k, o);
            k = q < k ? q : k;
        }
        if ((threadIdx.x & 31) == 0 && k < kmax) atomicMin(dst + first, (unsigned long long)k);
    } else if (k < kmax) {
        atomicMin(dst + inst, (unsigned long long)k);
    }
}

// ---------------------------------------------------------------------------
// a1: circumcentre of every triangle touching a real cell (Voronoi vertices), FP64
template <class R> __device__ __forceinline__ void stage_circumcentre(const SweepParams<R> &p, int32_t t)
{
    int32_t a = p.tri[3 * t], b = p.tri[3 * t + 1], c = p.tri[3 * t + 2];
    double ax = px_of(p, a), ay = py_of(p, a);
    double bx = px_of(p, b) - ax, by = py_of(p, b) - ay;
    double cx = px_of(p, c) - ax, cy = py_of(p, c) - ay;
    double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    double inv = 0.5 * recip(bx * cy - by * cx);
    p.ccx[t] = ax + (cy * b2 - by * c2) * inv;
    p.ccy[t] = ay + (bx * c2 - cx * b2) * inv;
}

// (the first n_inst threads also clear the simulations' time-step minima,
// which the geometry stage's cells then lower)
template <class R> __global__ void k_circumcentre(SweepParams<R> p)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < p.n_inst) p.dtmin_bits[t] = 0x7f7f7f7f7f7f7f7full;
    if (t < p.T) stage_circumcentre(p, t);
}

// a1: per-edge geometry relative to the edge's left generator.  The
// coordinate differences are taken in FP64; the rest in R.
template <class R> __device__ __forceinline__ void stage_edge_geometry(const SweepParams<R> &p, int32_t e)
{
    int32_t l = p.edge_l[e], r = p.edge_r[e];
    double xl = p.x[l], yl = p.y[l];
    const int32_t ta = p.edge_ta[e], tb = p.edge_tb[e];
    const double cax = p.ccx[ta], cay = p.ccy[ta];
    R ax = to_R<R>(cax - xl), ay = to_R<R>(cay - yl);
    R dx = to_R<R>(px_of(p, r) - xl), dy = to_R<R>(py_of(p, r) - yl);
    // the edge vector as the FP64 difference of its two vertices: a
    // zero-length edge stays ~0 instead of inheriting the rounding of two
    // separately rounded endpoints (six FP64 subtractions per edge)
    R ex = to_R<R>(p.ccx[tb] - cax), ey = to_R<R>(p.ccy[tb] - cay);
    R mx = ax + R(0.5) * ex, my = ay + R(0.5) * ey;
    // 1/|r_ij| with one reciprocal square root (a divide and a square root
    // each cost several FP64 issue slots on this part)
    const R rinv = rsqrt(dx * dx + dy * dy);
    const R nx = dx * rinv, ny = dy * rinv;
    // The Voronoi edge runs along the unit tangent t = (-n_y, n_x) (from
    // circumcentre ta to tb, counter-clockwise about the left cell), so its
    // length is e.t: the vertices' rounding across the edge changes |e| only
    // in second order, and a zero-length edge (co-circular generators) stays
    // ~0; a round-off-negative length is taken as zero.  Two operations
    // instead of the square root of e.e.
    const R Lt = ey * nx - ex * ny;
    const R L = key_nonneg(Lt) ? Lt : R(0);
    const R mrx = mx - dx, mry = my - dy;
    p.eL[e] = L;
    p.emlx[e] = mx;
    p.emly[e] = my;
    p.emrx[e] = mrx;
    p.emry[e] = mry;
    p.enx[e] = nx;
    p.eny[e] = ny;
    const R qx = (mx - R(0.5) * dx) * rinv, qy = (my - R(0.5) * dy) * rinv;
    p.eqx[e] = qx;
    p.eqy[e] = qy;
    // P = L (q + n/2) = (L/|r|) m_l and M = L (n/2 - q) = -(L/|r|) m_r, with
    // m_l, m_r the edge midpoint relative to the left and right generators
    const R k = L * rinv;
    p.ePM[e] = Vec4<R>{k * mx, k * my, -(k * mrx), -(k * mry)};
}


// a1 + a2: area and centre of mass (shoelace about the generator, FP64),
// then the primitive variables; in a sweep also a5 (mesh velocity) and a6:
// returns the cell's Courant time step R_i / (c_s + |v - w|) (DBL_MAX
// outside a sweep).  With init_W the conserved variables are set.
template <class R>
__device__ __forceinline__ double stage_cell_geometry(const SweepParams<R> &p, const double *__restrict__ init_W,
                                                      int32_t i, int32_t &my_inst)
{
    const int32_t lo = p.cell_ptr[i], hi = p.cell_ptr[i + 1];
    const double xi = p.x[i], yi = p.y[i];
    // Shoelace over the ring v_0 .. v_{m-1} (v_{-1} = v_{m-1}), with
    // c_s = v_{s-1} x v_s: 2A = sum c_s and 6A s = sum (v_{s-1} + v_s) c_s
    // = sum v_s (c_s + c_{s+1}), so each vertex enters once with the sum of
    // its two crosses (v_{m-1} last, when c_{m-1} + c_0 is known).
    int32_t tl = p.slot_tri[hi - 1];
    const double zx = p.ccx[tl] - xi, zy = p.ccy[tl] - yi;
    double ax = zx, ay = zy, c0, cp;
    double A2 = 0.0, sx = 0.0, sy = 0.0;
    {
        const int32_t t = p.slot_tri[lo];
        const double bx = p.ccx[t] - xi, by = p.ccy[t] - yi;
        const double cr = ax * by - ay * bx;
        A2 += cr;
        c0 = cp = cr;
        ax = bx;
        ay = by;
    }
    // two slots per pass: the next vertex's loads issue before this one's sums
#pragma unroll 2
    for (int32_t s = lo + 1; s < hi; s++) {
        const int32_t t = p.slot_tri[s];
        const double bx = p.ccx[t] - xi, by = p.ccy[t] - yi;
        const double cr = ax * by - ay * bx;
        A2 += cr;
        const double wv = cp + cr;
        sx += ax * wv;
        sy += ay * wv;
        cp = cr;
        ax = bx;
        ay = by;
    }
    {
        const double wv = cp + c0;
        sx += zx * wv;
        sy += zy * wv;
    }
    const double A = 0.5 * A2;
    // one division serves both the centre of mass and 1/A
    const double rA2 = recip(A2);
    const double inv3 = rA2 * (1.0 / 3.0);
    const double ox = sx * inv3, oy = sy * inv3;
    p.A[i] = A;
    p.o[i] = Vec2<R>{to_R<R>(ox), to_R<R>(oy)};
    // Section 6 trigger: the generator is more than eta R_i from its centre of
    // mass, d^2 > eta^2 A / pi (both sides non-negative, so no square roots).
    // Rounded cells settle at that distance, so the decision is taken in
    // FP64 in every precision.
    my_inst = inst_of(p, i);
    const InstParams &ip = p.inst[my_inst];
    const bool rounding = nonneg_less((ip.eta * ip.eta) * (A * (1.0 / M_PI)), ox * ox + oy * oy);
    p.rounding[i] = rounding ? 1 : 0;
    const int32_t n = p.n;
    const double gamma = ip.gamma;
    const double gm1 = gamma - 1.0;
    if (init_W) {
        if (!ip.init) return DBL_MAX;
        double rho = init_W[i], vx = init_W[n + i], vy = init_W[2 * n + i], pr = init_W[3 * n + i];
        double m = rho * A;
        p.Un[i] = m;
        p.Un[n + i] = m * vx;
        p.Un[2 * n + i] = m * vy;
        p.Un[3 * n + i] = (pr / gm1 + 0.5 * rho * (vx * vx + vy * vy)) * A;
        return DBL_MAX;
    }
    double m = p.U[i], Px = p.U[n + i], Py = p.U[2 * n + i], E = p.U[3 * n + i];
    Vec4<R> W;
    if (sizeof(R) == sizeof(double)) {
        double invA = 2.0 * rA2, invm = recip(m);
        double rho = m * invA, vx = Px * invm, vy = Py * invm;
        double pr = gm1 * (E - 0.5 * (Px * vx + Py * vy)) * invA;
        W = Vec4<R>{to_R<R>(rho), to_R<R>(vx), to_R<R>(vy), to_R<R>(pr)};
    } else {
        // the thermal energy cancels kinetic against total energy: FP64; the
        // FP64 pressure also feeds the shock switch's pressure-ratio test
        double eth = E - 0.5 * (Px * Px + Py * Py) * recip(m);
        double pr = gm1 * eth * (2.0 * rA2);
        p.p64[i] = pr;
        R Af = to_R<R>(A), mf = to_R<R>(m);
        W = Vec4<R>{mf / Af, to_R<R>(Px) / mf, to_R<R>(Py) / mf, to_R<R>(pr)};
    }
    p.W[i] = W;
    // c_s = sqrt(gamma p / rho) = gamma p / sqrt(gamma p rho): one reciprocal square root
    const R gp = inst_value<R>(ip.gamma, ip.gamma_f) * W.w;
    const R cs = gp * rsqrt(gp * W.x);
    p.cs[i] = cs;
    if (!p.motion) return DBL_MAX;
    // Section 6: mesh-generating point velocity, the fluid velocity plus,
    // where the trigger is on, chi c_s towards the centre of mass
    R wx = 0, wy = 0;
    if (ip.motion == 0) {
        wx = W.y;
        wy = W.z;
        if (rounding) {
            const R oxr = to_R<R>(ox), oyr = to_R<R>(oy);
            R f = inst_value<R>(ip.chi, ip.chi_f) * cs * rsqrt(oxr * oxr + oyr * oyr);
            wx += f * oxr;
            wy += f * oyr;
        }
    }
    p.w[i] = Vec2<R>{wx, wy};
    // Courant step R_i / (c_s + |v - w|), R_i = sqrt(A/pi) = (A/pi) rsqrt(A/pi)
    const R Api = to_R<R>(A) * (R(1) / R(M_PI));
    const R Rad = Api * rsqrt(Api);
    const R rx = W.y - wx, ry = W.z - wy;
    const R speed = cs + sqrt_nonneg(rx * rx + ry * ry);
    return to_d(Rad * recip(speed));
}

// a1 + a2 in one launch: the first edge_blocks blocks compute the edge
// geometry, the others the cell geometry and primitives.  The two depend
// only on the circumcentres, and sharing the SMs lets the edge part's
// loads and FP32 work (split precision) run beside the cell part's FP64
// shoelace instead of after it.
template <class R>
__global__ void k_geometry(SweepParams<R> p, const double *__restrict__ init_W, int32_t edge_blocks)
{
    if ((int32_t)blockIdx.x < edge_blocks) {
        int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
        if (e < p.E) stage_edge_geometry(p, e);
    } else {
        int32_t k = (blockIdx.x - edge_blocks) * blockDim.x + threadIdx.x;
        double dt_cell = DBL_MAX;
        int32_t my_inst = 0;
        if (k < p.n) dt_cell = stage_cell_geometry(p, init_W, cell_at(p, k), my_inst);
        // (init_W and motion are the same for the whole grid)
        if (!init_W && p.motion) warp_min_to(dt_cell, my_inst, p.dtmin_bits);
    }
}

// What the gradient stage reads per ring slot s of a cell: the edge length
// L, the cell's Eq. 1 weights for the neighbour (A = P, or -M for the
// edge's right cell) and for itself (B), the edge midpoint relative to the
// cell's generator, and the neighbour's primitives (mirrored for an image)
// with its FP64 pressure, here read from the sweep's arrays.
template <class R> struct GlobalSlots {
    const SweepParams<R> &p;
    __device__ __forceinline__ R L(int32_t s) const { return p.eL[p.slot_edge[s] >> 1]; }
    __device__ __forceinline__ void weights(int32_t s, R &Ax, R &Ay, R &Bx, R &By) const
    {
        const int32_t es = p.slot_edge[s];
        const Vec4<R> pm = p.ePM[es >> 1];
        // the right cell of an edge takes -M, -P (sign flips on the integer pipe)
        const unsigned long long ms = (es & 1) ? 0x8000000000000000ull : 0ull;
        Ax = flip((es & 1) ? pm.z : pm.x, ms);
        Ay = flip((es & 1) ? pm.w : pm.y, ms);
        Bx = flip((es & 1) ? pm.x : pm.z, ms);
        By = flip((es & 1) ? pm.y : pm.w, ms);
    }
    __device__ __forceinline__ void midpoint(int32_t s, R &mx, R &my) const
    {
        const int32_t es = p.slot_edge[s];
        const int32_t e = es >> 1;
        mx = (es & 1) ? p.emrx[e] : p.emlx[e];
        my = (es & 1) ? p.emry[e] : p.emly[e];
    }
    __device__ __forceinline__ Vec4<R> W(int32_t s) const { return load_W(p, p.slot_nb[s]); }
    __device__ __forceinline__ double p64(int32_t s, R pj) const
    {
        if (sizeof(R) == sizeof(double)) return (double)pj;
        int32_t xf;
        return p.p64[src_of(p, p.slot_nb[s], xf)];
    }
};

// a3-a4: Green-Gauss gradient (Eq. 1), limiter with the shock switch
// (Eqs. 3-8), and the cell terms of the half-step prediction, for cell i
// whose ring slots are [lo, hi) of the accessor `sl`.
template <class R, class Slots>
__device__ __forceinline__ void stage_cell_gradient(const SweepParams<R> &p, int32_t i, int32_t lo, int32_t hi,
                                                    const Slots &sl)
{
    {
        const InstParams &ip = p.inst[inst_of(p, i)];
        const Vec4<R> W4 = p.W[i];
        const R Wi[4] = {W4.x, W4.y, W4.z, W4.w};
        R acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        R Bx = 0, By = 0;
        Extremes<R> ext[4];
#pragma unroll
        for (int v = 0; v < 4; v++) ext[v].init(Wi[v]);
        bool shock = false;
        const R A = to_R<R>(p.A[i]);
        const double dp = ip.delta_p;
        const double pi64 = sizeof(R) == sizeof(double) ? (double)Wi[3] : p.p64[i];
        // R_i = sqrt(A/pi) and 1/A from one reciprocal square root:
        // rR = 1/R_i, so 1/A = rR^2 / pi and R_i = (A/pi) rR
        const R Api = A * (R(1) / R(M_PI));
        const R rR = rsqrt(Api);
        const R Rad = Api * rR;
        // Eqs. 3-8 look at the cells sharing an edge longer than 1e-9 sqrt(A)
        // = 1e-9 sqrt(pi) R_i: shorter edges are point contacts whose
        // presence depends on round-off
        const R Lmin = R(1.7724538509055160273e-9) * Rad;
        for (int32_t s = lo; s < hi; s++) {
            const R L = sl.L(s);
            // Eq. 1: g_i A_i = sum_j phi_j P_ij + phi_i sum_j M_ij
            R Ax, Ay, bx, by;
            sl.weights(s, Ax, Ay, bx, by);
            Bx += bx;
            By += by;
            const Vec4<R> Wv = sl.W(s);
            const R Wj[4] = {Wv.x, Wv.y, Wv.z, Wv.w};
#pragma unroll
            for (int v = 0; v < 4; v++) {
                acc[2 * v] += Wj[v] * Ax;
                acc[2 * v + 1] += Wj[v] * Ay;
            }
            if (nonneg_less(Lmin, L)) {
#pragma unroll
                for (int v = 0; v < 4; v++) ext[v].add(Wj[v]);
                const double pj64 = sl.p64(s, Wj[3]);
                const bool jl = nonneg_less(pj64, pi64);
                const double pmin = jl ? pj64 : pi64, pmax = jl ? pi64 : pj64;
                if (nonneg_less(pmin, dp * pmax)) shock = true;
            }
        }
#pragma unroll
        for (int v = 0; v < 4; v++) {
            acc[2 * v] += Wi[v] * Bx;
            acc[2 * v + 1] += Wi[v] * By;
        }
        R fmx[4], fmn[4];
#pragma unroll
        for (int v = 0; v < 4; v++) {
            fmx[v] = ext[v].max();
            fmn[v] = ext[v].min();
        }
        const R invA = rR * rR * (R(1) / R(M_PI));
        R g[8];
#pragma unroll
        for (int c = 0; c < 8; c++) g[c] = acc[c] * invA;
        const R cs = p.cs[i];
        // Eq. 7: -div v > delta_v c_s / R_i, as (delta_v c_s) < -(div v) R_i
        if (key_less(inst_value<R>(ip.delta_v, ip.delta_v_f) * cs, flip((g[2] + g[5]) * Rad, 0x8000000000000000ull)))
            shock = true;
        const bool use_tess = ip.limiter == 2 || (ip.limiter == 0 && shock);
        const Vec2<R> oi = p.o[i];
        const R ox = oi.x, oy = oi.y;
        // alpha = min(1, min_j psi_ij) without a division per edge.
        // AREPO (Eqs. 4-5): psi_ij = (phi_max - phi_i)/dphi for dphi > 0, so the
        // minimum over those edges sits at the largest dphi (likewise for
        // dphi < 0); one division per sign and variable.
        // TESS (Eq. 6): psi_ij = max(theta (phi_j - phi_i)/dphi, 0); the
        // smallest ratio is found by cross-multiplication, divided once.
        // alpha_v = an[v] / ad[v] (1/1 where the variable is not limited)
        R an[4] = {1, 1, 1, 1}, ad[4] = {1, 1, 1, 1};
        bool lim[4] = {false, false, false, false};
        if (!use_tess) {
            Extremes<R> dex[4];
#pragma unroll
            for (int v = 0; v < 4; v++) dex[v].init(R(0));
            for (int32_t s = lo; s < hi; s++) {
                if (!nonneg_less(Lmin, sl.L(s))) continue;
                R mx, my;
                sl.midpoint(s, mx, my);
                const R offx = mx - ox, offy = my - oy;
#pragma unroll
                for (int v = 0; v < 4; v++) dex[v].add(g[2 * v] * offx + g[2 * v + 1] * offy);
            }
#pragma unroll
            for (int v = 0; v < 4; v++) {
                // alpha = min(1, (phi_max - phi_i)/dphi_max, (phi_i - phi_min)/|dphi_min|):
                // a ratio below one needs its numerator to be the smaller, and
                // the smaller of two such ratios is found by cross-multiplication
                // (all terms non-negative)
                const R n1 = fmx[v] - Wi[v], d1 = dex[v].max();
                const R n2 = Wi[v] - fmn[v], d2 = -dex[v].min();
                const bool c1 = dex[v].max_positive() && nonneg_less(n1, d1);
                const bool c2 = dex[v].min_negative() && nonneg_less(n2, d2);
                if (c1 || c2) {
                    const bool use1 = c1 && (!c2 || nonneg_less(n1 * d2, n2 * d1));
                    an[v] = use1 ? n1 : n2;
                    ad[v] = use1 ? d1 : d2;
                    lim[v] = true;
                }
            }
        } else {
            R bn[4] = {0, 0, 0, 0}, bd[4] = {0, 0, 0, 0};  // smallest |N|/|D| so far (bd == 0: none)
            bool zero[4] = {false, false, false, false};
            for (int32_t s = lo; s < hi; s++) {
                if (!nonneg_less(Lmin, sl.L(s))) continue;
                R mx, my;
                sl.midpoint(s, mx, my);
                const R offx = mx - ox, offy = my - oy;
                const Vec4<R> Wv = sl.W(s);
                const R Wj[4] = {Wv.x, Wv.y, Wv.z, Wv.w};
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    R dphi = g[2 * v] * offx + g[2 * v + 1] * offy;
                    if (dphi == R(0)) continue;
                    R num = Wj[v] - Wi[v];
                    if (!(num * dphi > R(0))) { zero[v] = true; continue; }
                    R a_n = fabs(num), a_d = fabs(dphi);
                    if (bd[v] == R(0) || a_n * bd[v] < bn[v] * a_d) { bn[v] = a_n; bd[v] = a_d; }
                }
            }
#pragma unroll
            for (int v = 0; v < 4; v++) {
                // alpha = 0, or min(1, theta bn / bd)
                const R tn = inst_value<R>(ip.theta, ip.theta_f) * bn[v];
                if (zero[v]) { an[v] = R(0); lim[v] = true; }
                else if (bd[v] > R(0) && tn < bd[v]) { an[v] = tn; ad[v] = bd[v]; lim[v] = true; }
            }
        }
        // the cell's five quotients (alpha of each variable, 1/rho for the
        // prediction terms), each through one refined reciprocal
        R alpha[4];
#pragma unroll
        for (int v = 0; v < 4; v++) alpha[v] = lim[v] ? an[v] * recip(ad[v]) : R(1);
        const R irho = recip(Wi[0]);
        R lg[8];
#pragma unroll
        for (int c = 0; c < 8; c++) lg[c] = alpha[c >> 1] * g[c];
        p.gl[2 * i] = Vec4<R>{lg[0], lg[1], lg[2], lg[3]};
        p.gl[2 * i + 1] = Vec4<R>{lg[4], lg[5], lg[6], lg[7]};
        {
            // cell-only terms of the half-step prediction (used by every edge
            // of the cell): rho div v, grad p / rho, gamma p div v
            const R ldiv = lg[2] + lg[5];
            p.psrc[i] = Vec4<R>{Wi[0] * ldiv, lg[6] * irho, lg[7] * irho, inst_value<R>(ip.gamma, ip.gamma_f) * Wi[3] * ldiv};
        }
        if (p.diagnostics) {
            p.g[2 * i] = Vec4<R>{g[0], g[1], g[2], g[3]};
            p.g[2 * i + 1] = Vec4<R>{g[4], g[5], g[6], g[7]};
            p.alpha[i] = Vec4<R>{alpha[0], alpha[1], alpha[2], alpha[3]};
            p.tess[i] = use_tess ? 1 : 0;
        }
    }
}

// launched in blocks of 128 threads; six blocks per SM cap the FP64 build at
// 80 registers (from 94, with a few spilled to L1), 24 warps instead of 20;
// nine hold the FP32 build's 56 registers, 36 warps, which hide more of its
// gather latency than 28 did (0.102 -> 0.093 ms at 1M cells, when the cap
// took it from 72 registers, before the mesh velocity and the time step
// moved to the geometry stage; ten blocks spilled and lost it again).
// The FP64 build visits cells in the degree-sorted order (FP64 issue is per
// warp instruction, so a warp should loop near the mean degree); the FP32
// build, bound by its gathers, visits them in the Hilbert order itself, so
// that the rings of a warp's cells are adjacent in the slot arrays and their
// neighbours share cache lines.
template <class R> __global__ void __launch_bounds__(128, sizeof(R) == 4 ? 9 : 6) k_cell_gradient(SweepParams<R> p)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < p.n) {
        const int32_t i = sizeof(R) == sizeof(double) ? cell_at(p, k) : k;
        stage_cell_gradient(p, i, p.cell_ptr[i], p.cell_ptr[i + 1], GlobalSlots<R>{p});
    }
}

template <class R> __device__ __forceinline__ double step_dt(const SweepParams<R> &p, int32_t inst)
{
    const InstParams &ip = p.inst[inst];
    // the second sweep of the time-centred scheme keeps the first one's dt
    if (ip.phase == 2) return __ldcg(p.dt_out + inst);
    // read through L2: in the persistent sweep the minimum was reset and then
    // reduced with atomics earlier in the same launch, and a line of it may
    // still sit stale in this SM's L1
    double dt = ip.cfl * __longlong_as_double((long long)__ldcg(p.dtmin_bits + inst));
    return nonneg_less(ip.remaining, dt) ? ip.remaining : dt;
}

// The step's dt in the stages after the point motion, which records it
// (the same bits as step_dt, without its FP64 multiply per thread)
template <class R> __device__ __forceinline__ double recorded_dt(const SweepParams<R> &p, int32_t inst)
{
    return __ldcg(p.dt_out + inst);
}

// half-step prediction of one side's edge state in the frame moving with wf:
// Eq. 2 extrapolation minus hdt times the primitive Euler right-hand side,
// whose cell-only terms (rho div v, grad p / rho, gamma p div v) come in src.
// The velocity comes out relative to the edge (v - wf), ready for the
// rotation into the edge frame.
template <class R>
__device__ __forceinline__ void predict(R hdt, const R W[4], const R g[8], const R src[4], R offx, R offy, R wfx,
                                        R wfy, R out[4])
{
    // phi + g.off - hdt (u.g + src) = phi + g.(off - hdt u) - hdt src, u = v - wf:
    // the advective part of the prediction moves the extrapolation point
    const R ux = W[1] - wfx, uy = W[2] - wfy;
    const R ax = offx - hdt * ux, ay = offy - hdt * uy;
    const R base[4] = {W[0], ux, uy, W[3]};
#pragma unroll
    for (int c = 0; c < 4; c++) out[c] = base[c] + g[2 * c] * ax + g[2 * c + 1] * ay - hdt * src[c];
}

// HLLC (Toro) in the edge frame, states (rho, u_n, u_t, p)
template <class R> __device__ __forceinline__ void hllc(R gam, R igm1, const R L[4], const R Rs[4], R F[4])
{
    const R rL = L[0], uL = L[1], tL = L[2], pL = L[3];
    const R rR = Rs[0], uR = Rs[1], tR = Rs[2], pR = Rs[3];
    // c = sqrt(gamma p / rho) = gamma p / sqrt(gamma p rho): one reciprocal
    // square root instead of a divide and a square root
    const R gpL = gam * pL, gpR = gam * pR;
    const R cL = gpL * rsqrt(gpL * rL), cR = gpR * rsqrt(gpR * rR);
    // Davis speeds, min / max chosen through integer keys
    const R aL = uL - cL, aR = uR - cR, bL = uL + cL, bR = uR + cR;
    const R SL = key_less(aR, aL) ? aR : aL;
    const R SR = key_less(bL, bR) ? bR : bL;
    // The flux is that of one side K plus, between the outer waves,
    // S_K (U*_K - U_K).  K is picked by selects rather than branches, so a
    // warp whose edges take different sides evaluates one star state, not two.
    const bool supL = key_nonneg(SL), supR = !supL && key_nonpos(SR);
    const bool sub = !(supL || supR);
    // m_K = rho_K (S_K - u_K): m_L < 0 < m_R, so the contact speed
    // S* = num / den has den = m_L - m_R < 0 and S* >= 0 exactly when num <= 0
    const R mL = rL * (SL - uL), mR = rR * (SR - uR);
    const R num = pR - pL + uL * mL - uR * mR, den = mL - mR;
    const bool useL = supL || (sub && key_nonpos(num));
    const R rK = useL ? rL : rR, uK = useL ? uL : uR, tK = useL ? tL : tR, pK = useL ? pL : pR;
    // only side K's total energy enters the flux
    const R EK = pK * igm1 + R(0.5) * rK * (uK * uK + tK * tK);
    const R ruK = rK * uK;
    F[0] = ruK;
    F[1] = ruK * uK + pK;
    F[3] = uK * (EK + pK);
    if (sub) {
        // star state: rho* = m_K/(S_K - S*), E* = ((S_K - u_K) E_K + (S* - u_K)(m_K S* + p_K))/(S_K - S*).
        // With D = S_K den - num, S_K - S* = D / den; one reciprocal
        // r = 1/(den D) gives S* = num D r and 1/(S_K - S*) = den^2 r.
        const R SK = useL ? SL : SR, mK = useL ? mL : mR;
        const R D = SK * den - num;
        const R r = recip(den * D);
        const R Ss = num * D * r;
        const R inv = den * den * r;
        const R f = mK * inv;
        const R Es = ((SK - uK) * EK + (Ss - uK) * (mK * Ss + pK)) * inv;
        F[0] += SK * (f - rK);
        F[1] += SK * (f * Ss - ruK);
        F[3] += SK * (Es - EK);
    }
    // the tangential momentum flux is the mass flux times u_t of side K
    F[2] = F[0] * tK;
}

// a7: one flux per edge in the frame of the moving edge
template <class R> __device__ __forceinline__ void stage_edge_flux(const SweepParams<R> &p, int32_t e)
{
    const int32_t l = p.edge_l[e];
    const int32_t li = inst_of(p, l);
    // edge states advance half a step in time only in the extrapolated scheme
    // (the hardware converts FP64 -> R in this stage: the integer-pipe
    // conversions' extra registers cost it more than the FP64 issue slots
    // they save)
    const R hdt = p.inst[li].phase == 0 ? R(0.5) * (R)recorded_dt(p, li) : R(0);
    int32_t xf;
    const int32_t k = src_of(p, p.edge_r[e], xf);
    // sign masks of a mirror image across an x wall, a y wall, and both
    const unsigned long long mx = (xf & 1) ? 0x8000000000000000ull : 0ull;
    const unsigned long long my = (xf & 2) ? 0x8000000000000000ull : 0ull;
    const unsigned long long mxy = mx ^ my;
    const Vec4<R> Wl4 = p.W[l], Wr4 = p.W[k];
    const R Wl[4] = {Wl4.x, Wl4.y, Wl4.z, Wl4.w};
    const R Wr[4] = {Wr4.x, flip(Wr4.y, mx), flip(Wr4.z, my), Wr4.w};
    const Vec4<R> gl0 = p.gl[2 * l], gl1 = p.gl[2 * l + 1];
    const Vec4<R> gr0 = p.gl[2 * k], gr1 = p.gl[2 * k + 1];
    const R gL[8] = {gl0.x, gl0.y, gl0.z, gl0.w, gl1.x, gl1.y, gl1.z, gl1.w};
    // mirrored source: each derivative takes the flip of its axis, velocity
    // components also the flip of their own axis
    const R gR[8] = {flip(gr0.x, mx), flip(gr0.y, my), gr0.z, flip(gr0.w, mxy),
                     flip(gr1.x, mxy), gr1.y, flip(gr1.z, mx), flip(gr1.w, my)};
    const Vec2<R> wl = p.w[l], wk = p.w[k];
    const Vec2<R> ol = p.o[l], ok = p.o[k];
    const R wlx = wl.x, wly = wl.y;
    const R wrx = flip(wk.x, mx), wry = flip(wk.y, my);
    const R orx = flip(ok.x, mx), ory = flip(ok.y, my);
    const R L = p.eL[e];
    const R nx = p.enx[e], ny = p.eny[e];
    const R qx = p.eqx[e], qy = p.eqy[e];
    // velocity of the perpendicular bisector at the edge midpoint
    const R dwc = (wrx - wlx) * qx + (wry - wly) * qy;
    const R wfx = R(0.5) * (wlx + wrx) - dwc * nx;
    const R wfy = R(0.5) * (wly + wry) - dwc * ny;
    R Sl[4], Sr[4];
    const R gam = inst_value<R>(p.inst[li].gamma, p.inst[li].gamma_f);
    const Vec4<R> sl4 = p.psrc[l], sr4 = p.psrc[k];
    // a mirrored source flips the pressure-gradient term of its axis
    const R srcL[4] = {sl4.x, sl4.y, sl4.z, sl4.w};
    const R srcR[4] = {sr4.x, flip(sr4.y, mx), flip(sr4.z, my), sr4.w};
    predict(hdt, Wl, gL, srcL, p.emlx[e] - ol.x, p.emly[e] - ol.y, wfx, wfy, Sl);
    predict(hdt, Wr, gR, srcR, p.emrx[e] - orx, p.emry[e] - ory, wfx, wfy, Sr);
    const R tx = -ny, ty = nx;
    R WL[4] = {Sl[0], Sl[1] * nx + Sl[2] * ny, Sl[1] * tx + Sl[2] * ty, Sl[3]};
    R WR[4] = {Sr[0], Sr[1] * nx + Sr[2] * ny, Sr[1] * tx + Sr[2] * ty, Sr[3]};
    R Fe[4];
    hllc(gam, inst_value<R>(p.inst[li].igm1, p.inst[li].igm1_f), WL, WR, Fe);
    if (xf && k == l) {
        // a wall: the cell faces its own mirror image.  The mirrored Riemann
        // problem has u* = 0 and the wall does not move normal to itself, so
        // mass, tangential momentum and energy fluxes vanish exactly; only
        // the normal pressure flux remains (round-off would otherwise leak).
        p.F[e] = Vec4<R>{R(0), L * Fe[1] * nx, L * Fe[1] * ny, R(0)};
        return;
    }
    const R Fmx = Fe[1] * nx + Fe[2] * tx, Fmy = Fe[1] * ny + Fe[2] * ty;
    p.F[e] = Vec4<R>{L * Fe[0], L * (Fmx + Fe[0] * wfx), L * (Fmy + Fe[0] * wfy),
                     L * (Fe[3] + Fmx * wfx + Fmy * wfy + R(0.5) * (wfx * wfx + wfy * wfy) * Fe[0])};
}

// launched in blocks of 128 threads; ten blocks per SM cap the FP64 build
// at 48 registers (a few spilled to L1): the FP64 flux times the same as
// with 62 registers; sixteen cap the FP32 build at 32 (4 bytes spilled),
// 64 warps: 0.069 -> 0.063 ms at 1M cells
template <class R> __global__ void __launch_bounds__(128, sizeof(R) == 4 ? 16 : 10) k_edge_flux(SweepParams<R> p)
{
    int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < p.E) stage_edge_flux(p, e);
}

// a9: advance the generating points in FP64, x <- x0 + hdt w, wrapped
// across a periodic box or mirrored back across a rigid wall.  The step's dt
// is final once every cell's Courant candidate is in (after the geometry
// stage); the first cell of each simulation records it.
template <class R> __device__ __forceinline__ void stage_advance(const SweepParams<R> &p, int32_t i)
{
    const int32_t my_inst = inst_of(p, i);
    const InstParams &ip = p.inst[my_inst];
    const double dt = step_dt(p, my_inst);
    if (ip.phase != 2 && (i == 0 || inst_of(p, i - 1) != my_inst)) p.dt_out[my_inst] = dt;
    // the first sweep of the time-centred scheme moves the points half a step
    // (branches rather than selects: each FP64 instruction a warp issues
    // costs 16 clocks of the SM's FP64 pipe, taken or not)
    double hdt = dt;
    if (ip.phase == 1) hdt = 0.5 * dt;
    const Vec2<R> w = p.w[i];
    double xn = p.x0[i] + hdt * to_d(w.x), yn = p.y0[i] + hdt * to_d(w.y);
    // the box tests compare bit patterns on the integer pipe (dkey orders
    // doubles); the few points that crossed an edge of the box take the
    // FP64 corrections in a branch of their own
    const long long kx0 = dkey0(ip.x0), kx1 = dkey0(ip.x1), ky0 = dkey0(ip.y0), ky1 = dkey0(ip.y1);
    long long kx = dkey0(xn), ky = dkey0(yn);
    int32_t st = 0;
    if (ip.boundary == 1) {
        if (kx < kx0 || kx >= kx1 || ky < ky0 || ky >= ky1) {
            const double Lx = ip.x1 - ip.x0, Ly = ip.y1 - ip.y0;
            if (kx < kx0) xn += Lx;
            else if (kx >= kx1) xn -= Lx;
            if (ky < ky0) yn += Ly;
            else if (ky >= ky1) yn -= Ly;
        }
    } else if (kx <= kx0 || kx >= kx1 || ky <= ky0 || ky >= ky1) {
        // a point that crossed a rigid wall comes back as its mirror image
        if (kx <= kx0) xn = (ip.x0 + ip.x0) - xn;
        else if (kx >= kx1) xn = (ip.x1 + ip.x1) - xn;
        if (ky <= ky0) yn = (ip.y0 + ip.y0) - yn;
        else if (ky >= ky1) yn = (ip.y1 + ip.y1) - yn;
        kx = dkey0(xn);
        ky = dkey0(yn);
        if (!(kx > kx0 && kx < kx1 && ky > ky0 && ky < ky1)) st |= ST_LEFT_BOX;
    }
    p.xn[i] = xn;
    p.yn[i] = yn;
    if (st) atomicOr(p.status + my_inst, st);
}

template <class R> __global__ void __launch_bounds__(kAdvanceBlock) k_advance_points(SweepParams<R> p)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p.n) stage_advance(p, i);
}

// a8: conservative update in FP64 (fixed CSR order, no atomics)
template <class R> __device__ __forceinline__ void stage_cell_update(const SweepParams<R> &p, int32_t i)
{
    const int32_t n = p.n;
    const int32_t my_inst = inst_of(p, i);
    const InstParams &ip = p.inst[my_inst];
    const double dt = recorded_dt(p, my_inst);
    // the first sweep of the time-centred scheme moves the state half a step
    double hdt = dt;
    if (ip.phase == 1) hdt = 0.5 * dt;
    const int32_t lo = p.cell_ptr[i], hi = p.cell_ptr[i + 1];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int32_t s = lo; s < hi; s++) {
        int32_t es = p.slot_edge[s];
        const Vec4<R> f = p.F[es >> 1];
        // the right cell takes the flux with the opposite sign: flip the sign
        // bit (integer pipe) rather than branch, so each slot costs one add
        // per component whatever the mix of sides in the warp; a split-
        // precision flux is widened exactly on the integer pipe (to_d), so
        // both cells of the edge add the same FP64 value
        const unsigned long long sg = (unsigned long long)(es & 1) << 63;
        s0 += __longlong_as_double(__double_as_longlong(to_d(f.x)) ^ sg);
        s1 += __longlong_as_double(__double_as_longlong(to_d(f.y)) ^ sg);
        s2 += __longlong_as_double(__double_as_longlong(to_d(f.z)) ^ sg);
        s3 += __longlong_as_double(__double_as_longlong(to_d(f.w)) ^ sg);
    }
    double m = p.U0[i] - hdt * s0;
    double Px = p.U0[n + i] - hdt * s1;
    double Py = p.U0[2 * n + i] - hdt * s2;
    double E = p.U0[3 * n + i] - hdt * s3;
    p.Un[i] = m;
    p.Un[n + i] = Px;
    p.Un[2 * n + i] = Py;
    p.Un[3 * n + i] = E;
    // the checks compare bit patterns on the integer pipe: a double is not
    // finite when its exponent bits are all set, positive when its bits are
    // positive as an integer
    int32_t st = 0;
    {
        const long long bm = __double_as_longlong(m), bx = __double_as_longlong(Px);
        const long long by = __double_as_longlong(Py), be = __double_as_longlong(E);
        const long long ex = 0x7ff0000000000000ll;
        if ((bm & ex) == ex || (bx & ex) == ex || (by & ex) == ex || (be & ex) == ex) st |= ST_NAN;
        else if (!(bm > 0) || !(__double_as_longlong(2.0 * m * E - (Px * Px + Py * Py)) > 0)) st |= ST_NEGATIVE;
    }
    if (st) atomicOr(p.status + my_inst, st);
}

template <class R> __global__ void __launch_bounds__(kBlock) k_cell_update(SweepParams<R> p)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < p.n) stage_cell_update(p, cell_at(p, k));
}

// ---------------------------------------------------------------------------
// Persistent sweep: every stage in one cooperative launch.

constexpr long long kSpinLimit = 1ll << 24;  // ~1-2 s of polling with 64 ns sleeps

// Grid-wide barrier.  Thread 0 of each block reads the generation, arrives,
// and waits for the last block to bump the generation; a wait that exceeds
// `limit` polls sets the timeout flag instead, and the other waiters leave
// when they see it.  Returns false once any block has given up, and the
// caller then leaves the kernel.
__device__ bool grid_sync(GridSync *gs, unsigned int nblocks, long long limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &gs->gen;
        volatile int32_t *vto = &gs->timeout;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&gs->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == g && *vto == 0) {
                if (++it > limit) {
                    atomicExch(&gs->timeout, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int32_t *)&gs->timeout == 0;
}

template <class R>
__global__ void __launch_bounds__(512) k_sweep_persistent(SweepParams<R> p, const DeviceSizes *sz, GridSync *gs)
{
    p.n = sz->n;
    p.ng = sz->ng;
    p.T = sz->T;
    p.E = sz->E;
    p.n_inst = sz->n_inst;
    // blocks the barrier waits for (more than the grid only when a test makes
    // the waits run out) and polls before a wait gives up
    const unsigned int nb = gridDim.x + (unsigned int)gs->extra;
    const long long lim = gs->spin_limit > 0 ? gs->spin_limit : kSpinLimit;
    const int32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t k = tid; k < p.n_inst; k += stride) atomicExch(p.dtmin_bits + k, 0x7f7f7f7f7f7f7f7full);
    for (int32_t t = tid; t < p.T; t += stride) stage_circumcentre(p, t);
    if (!grid_sync(gs, nb, lim)) return;
    for (int32_t e = tid; e < p.E; e += stride) stage_edge_geometry(p, e);
    // (whole warps through the cell loop, for the warp-wide dt minimum)
    for (int32_t base = blockIdx.x * blockDim.x; base < p.n; base += stride) {
        const int32_t k = base + threadIdx.x;
        double v = DBL_MAX;
        int32_t inst = 0;
        if (k < p.n) v = stage_cell_geometry(p, (const double *)nullptr, cell_at(p, k), inst);
        warp_min_to(v, inst, p.dtmin_bits);
    }
    if (!grid_sync(gs, nb, lim)) return;
    for (int32_t i = tid; i < p.n; i += stride) stage_advance(p, i);
    for (int32_t k = tid; k < p.n; k += stride) {
        const int32_t i = cell_at(p, k);
        stage_cell_gradient(p, i, p.cell_ptr[i], p.cell_ptr[i + 1], GlobalSlots<R>{p});
    }
    if (!grid_sync(gs, nb, lim)) return;
    for (int32_t e = tid; e < p.E; e += stride) stage_edge_flux(p, e);
    if (!grid_sync(gs, nb, lim)) return;
    for (int32_t k = tid; k < p.n; k += stride) stage_cell_update(p, cell_at(p, k));
}

__global__ void k_repack(const int32_t *__restrict__ src, int32_t n_new, int32_t n_old,
                         const double *__restrict__ U_old, double *__restrict__ U_new)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_new) return;
    int32_t k = src[i];
    if (k < 0) return;
#pragma unroll
    for (int c = 0; c < 4; c++) U_new[(size_t)c * n_new + i] = U_old[(size_t)c * n_old + k];
}

// owner of the edge between real cell i and point j (1: i, 0: the other
// side, -1: inconsistent), the host builder's rule
__device__ __forceinline__ int edge_owner(int32_t i, int32_t j, int32_t n, int32_t periodic,
                                          const int32_t *ghost_src, const int32_t *ghost_shift)
{
    if (j < n) return j > i ? 1 : (j < i ? 0 : -1);
    if (!periodic) return 1;
    const int32_t src = ghost_src[j - n];
    if (src != i) return src > i ? 1 : 0;
    const int32_t sh = ghost_shift[j - n];
    const int32_t sx = sh % 3 - 1, sy = sh / 3 - 1;
    return (sy < 0 || (sy == 0 && sx < 0)) ? 0 : 1;
}

__global__ void k_build_edges(int32_t n, const int32_t *__restrict__ cell_ptr, const int32_t *__restrict__ slot_nb,
                              const int32_t *__restrict__ slot_tri, const int32_t *__restrict__ ghost_src,
                              const int32_t *__restrict__ ghost_shift, const int32_t *__restrict__ edge_off,
                              int32_t periodic_all, const InstParams *__restrict__ inst,
                              const int32_t *__restrict__ cell_inst, int32_t *slot_edge, int32_t *edge_l,
                              int32_t *edge_r, int32_t *edge_ta, int32_t *edge_tb)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t periodic = cell_inst ? (inst[cell_inst[i]].boundary == 1 ? 1 : 0) : periodic_all;
    const int32_t lo = cell_ptr[i], deg = cell_ptr[i + 1] - lo;
    int32_t e = edge_off[i];
    const int32_t e_end = edge_off[i + 1];
    for (int32_t k = 0; k < deg; k++) {
        const int32_t s = lo + k, j = slot_nb[s];
        if (edge_owner(i, j, n, periodic, ghost_src, ghost_shift) <= 0) continue;
        if (e >= e_end) return;  // more owned slots than the host counted: left unset, caught by the check
        edge_l[e] = i;
        edge_r[e] = j;
        edge_ta[e] = slot_tri[lo + (k + deg - 1) % deg];
        edge_tb[e] = slot_tri[s];
        slot_edge[s] = 2 * e;
        // the same edge seen from the other cell's ring
        int32_t pc = -1, want = -1;
        if (j < n) {
            pc = j;
        } else if (periodic) {
            pc = ghost_src[j - n];
            const int32_t sh = ghost_shift[j - n];
            want = (1 - (sh % 3 - 1)) + 3 * (1 - (sh / 3 - 1));
        }
        if (pc >= 0) {
            const int32_t q1 = cell_ptr[pc + 1];
            for (int32_t q = cell_ptr[pc]; q < q1; q++) {
                const int32_t c2 = slot_nb[q];
                const bool hit = j < n ? c2 == i
                                       : (c2 >= n && ghost_src[c2 - n] == i && ghost_shift[c2 - n] == want && q != s);
                if (hit) {
                    slot_edge[q] = 2 * e + 1;
                    break;
                }
            }
        }
        e++;
    }
}

// a slot left without its edge (or triangle): any negative entry
__global__ void k_check_edges(int32_t S, const int32_t *__restrict__ slot_edge, int32_t *bad)
{
    const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S && slot_edge[s] < 0) *bad = 1;
}

// One thread per real cell: its owned triangles (both other vertices with
// larger ids) numbered in ring order, and for every other slot the number
// its owner gave the triangle, found by walking the owner's ring.
__global__ void k_build_tris(int32_t n, const int32_t *__restrict__ cell_ptr, const int32_t *__restrict__ slot_nb,
                             const int32_t *__restrict__ tri_off, int32_t *tri, int32_t *slot_tri, int32_t *bad)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t lo = cell_ptr[i], deg = cell_ptr[i + 1] - lo;
    int32_t t = tri_off[i];
    const int32_t t_end = tri_off[i + 1];
    for (int32_t k = 0; k < deg; k++) {
        const int32_t a = slot_nb[lo + k], b = slot_nb[lo + (k + 1 == deg ? 0 : k + 1)];
        if (i < a && i < b) {
            if (t >= t_end) {
                *bad = 1;
                return;
            }
            tri[3 * t] = i;
            tri[3 * t + 1] = a;
            tri[3 * t + 2] = b;
            slot_tri[lo + k] = t++;
            continue;
        }
        // the owner o is the smaller of a and b (a real cell, below i); in
        // its ring the triangle (i, a, b) reads (o, p, q): (a, b, i) or
        // (b, i, a)
        const int32_t o = a < b ? a : b;
        if (o < 0 || o >= n) {
            *bad = 1;
            return;
        }
        const int32_t p = o == a ? b : i, q = o == a ? i : a;
        const int32_t olo = cell_ptr[o], odeg = cell_ptr[o + 1] - olo;
        int32_t num = tri_off[o], found = -1;
        for (int32_t kk = 0; kk < odeg; kk++) {
            const int32_t x = slot_nb[olo + kk], y = slot_nb[olo + (kk + 1 == odeg ? 0 : kk + 1)];
            if (x == p && y == q) {
                found = num;
                break;
            }
            num += (o < x && o < y) ? 1 : 0;
        }
        if (found < 0) {
            *bad = 1;
            return;
        }
        slot_tri[lo + k] = found;
    }
    if (t != t_end) *bad = 1;
}

inline int blocks(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }
// Threads per block of each stage.  Small blocks let the block scheduler
// balance the SMs at a fine grain: with 256 threads a per-cell stage over
// 262,144 cells ran 1.1-3.4 waves of 8-warp blocks, and SMs idled for up
// to 17 % of the launch waiting for the last blocks (per-SM active cycles
// from 0.77x to 1.17x of the mean).  Chosen by timing 32, 64, 128 and 256 on
// GB300 (Sedov, 262,144 cells): the gradient and flux stages, whose register
// counts cap an SM at 16-21 warps, run best at 128, the others at 32.
constexpr int kStageBlock[NUM_STAGES] = {32, 32, kAdvanceBlock, 128, 128, 32};
static_assert(kStageBlock[K_CELL_GRADIENT] == 128 && kStageBlock[K_EDGE_FLUX] == 128,
              "the gradient's and flux's launch bounds assume 128 threads");
inline int stage_block(int k) { return kStageBlock[k]; }
inline int nblk(int64_t n, int k) { return (int)((n + stage_block(k) - 1) / stage_block(k)); }

}  // namespace

const char *stage_name(int k)
{
    static const char *names[NUM_STAGES] = {"k_circumcentre", "k_geometry", "k_advance_points", "k_cell_gradient",
                                            "k_edge_flux", "k_cell_update"};
    return k >= 0 && k < NUM_STAGES ? names[k] : "";
}

template <class R> void launch_stage(int k, const SweepParams<R> &p, const double *init_W, cudaStream_t st)
{
    switch (k) {
    case K_CIRCUMCENTRE: {
        const int32_t m = p.T > p.n_inst ? p.T : p.n_inst;
        if (m > 0) k_circumcentre<R><<<nblk(m, K_CIRCUMCENTRE), stage_block(K_CIRCUMCENTRE), 0, st>>>(p);
        break;
    }
    case K_GEOMETRY: {
        const int eb = nblk(p.E, K_GEOMETRY), cb = nblk(p.n, K_GEOMETRY);
        if (eb + cb > 0) k_geometry<R><<<eb + cb, stage_block(K_GEOMETRY), 0, st>>>(p, init_W, eb);
        break;
    }
    case K_ADVANCE:
        if (p.n > 0) k_advance_points<R><<<nblk(p.n, K_ADVANCE), stage_block(K_ADVANCE), 0, st>>>(p);
        break;
    case K_CELL_GRADIENT:
        if (p.n > 0) k_cell_gradient<R><<<nblk(p.n, K_CELL_GRADIENT), stage_block(K_CELL_GRADIENT), 0, st>>>(p);
        break;
    case K_EDGE_FLUX:
        if (p.E > 0) k_edge_flux<R><<<nblk(p.E, K_EDGE_FLUX), stage_block(K_EDGE_FLUX), 0, st>>>(p);
        break;
    case K_CELL_UPDATE:
        if (p.n > 0) k_cell_update<R><<<nblk(p.n, K_CELL_UPDATE), stage_block(K_CELL_UPDATE), 0, st>>>(p);
        break;
    default:
        break;
    }
}

cudaError_t launch_build_tris(int32_t n, int32_t S, const int32_t *cell_ptr, const int32_t *slot_nb,
                              const int32_t *tri_off, int32_t *tri, int32_t *slot_tri, int32_t *bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
    if (e == cudaSuccess && S > 0) e = cudaMemsetAsync(slot_tri, 0xff, sizeof(int32_t) * (size_t)S, st);
    if (e != cudaSuccess) return e;
    if (n > 0) k_build_tris<<<blocks(n), kBlock, 0, st>>>(n, cell_ptr, slot_nb, tri_off, tri, slot_tri, bad);
    if (S > 0) k_check_edges<<<blocks(S), kBlock, 0, st>>>(S, slot_tri, bad);
    return cudaGetLastError();
}

cudaError_t launch_build_edges(int32_t n, int32_t S, const int32_t *cell_ptr, const int32_t *slot_nb,
                               const int32_t *slot_tri, const int32_t *ghost_src, const int32_t *ghost_shift,
                               const int32_t *edge_off, int32_t periodic, const InstParams *inst,
                               const int32_t *cell_inst, int32_t *slot_edge, int32_t *edge_l, int32_t *edge_r,
                               int32_t *edge_ta, int32_t *edge_tb, int32_t *bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
    if (e == cudaSuccess && S > 0) e = cudaMemsetAsync(slot_edge, 0xff, sizeof(int32_t) * (size_t)S, st);
    if (e != cudaSuccess) return e;
    if (n > 0)
        k_build_edges<<<blocks(n), kBlock, 0, st>>>(n, cell_ptr, slot_nb, slot_tri, ghost_src, ghost_shift, edge_off,
                                                     periodic, inst, cell_inst, slot_edge, edge_l, edge_r, edge_ta,
                                                     edge_tb);
    if (S > 0) k_check_edges<<<blocks(S), kBlock, 0, st>>>(S, slot_edge, bad);
    return cudaGetLastError();
}

void launch_repack(const int32_t *src, int32_t n_new, int32_t n_old, const double *U_old, double *U_new,
                   cudaStream_t st)
{
    if (n_new > 0) k_repack<<<blocks(n_new), kBlock, 0, st>>>(src, n_new, n_old, U_old, U_new);
}

template <class R>
cudaError_t launch_persistent(const SweepParams<R> &p, const DeviceSizes *sizes, GridSync *sync, int block, int grid,
                              cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep_persistent<R>, p, sizes, sync);
}

template <class R> int persistent_blocks_per_sm(int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_persistent<R>, block, 0) != cudaSuccess) return 0;
    return nb;
}

template cudaError_t launch_persistent<double>(const SweepParams<double> &, const DeviceSizes *, GridSync *, int, int,
                                               cudaStream_t);
template cudaError_t launch_persistent<float>(const SweepParams<float> &, const DeviceSizes *, GridSync *, int, int,
                                              cudaStream_t);
template int persistent_blocks_per_sm<double>(int);
template int persistent_blocks_per_sm<float>(int);

template void launch_stage<double>(int, const SweepParams<double> &, const double *, cudaStream_t);
template void launch_stage<float>(int, const SweepParams<float> &, const double *, cudaStream_t);

}  // namespace rich
