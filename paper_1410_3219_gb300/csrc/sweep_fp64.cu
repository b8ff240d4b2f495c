// FP64 sweep kernels: steps a1-a9 of one extrapolated-fluxes time step of
// the moving Voronoi mesh scheme (paper Section 2).  FP64 throughput on this
// part is ~1.2 TFLOP/s, so the kernels compute every FP64 quantity once and
// keep it in HBM for the next kernel (circumcentres per triangle, edge
// geometry per edge, one HLLC flux per edge), avoid re-evaluating divisions
// and square roots, and gather fluxes per cell in a fixed order (no atomics).
#include <cfloat>
#include <cmath>

#include "sweep.cuh"

namespace rich {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double px_of(const SweepParams &p, int32_t q) { return q < p.n ? p.x[q] : p.gx[q - p.n]; }
__device__ __forceinline__ double py_of(const SweepParams &p, int32_t q) { return q < p.n ? p.y[q] : p.gy[q - p.n]; }

// real cell behind point q and its mirror flags
__device__ __forceinline__ int32_t src_of(const SweepParams &p, int32_t q, int32_t &xf)
{
    if (q < p.n) { xf = 0; return q; }
    xf = p.ghost_xf[q - p.n];
    return p.ghost_src[q - p.n];
}

// primitives of point q (a ghost mirrors the velocity of its source)
__device__ __forceinline__ void load_W(const SweepParams &p, int32_t q, double W[4])
{
    int32_t xf;
    int32_t k = src_of(p, q, xf);
    const int32_t n = p.n;
    W[0] = p.W[k];
    W[1] = p.W[n + k];
    W[2] = p.W[2 * n + k];
    W[3] = p.W[3 * n + k];
    if (xf & 1) W[1] = -W[1];
    if (xf & 2) W[2] = -W[2];
}

// ---------------------------------------------------------------------------
// a1: circumcentre of every triangle touching a real cell (Voronoi vertices)
__global__ void k_circumcentre(SweepParams p)
{
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.T) return;
    int32_t a = p.tri[3 * t], b = p.tri[3 * t + 1], c = p.tri[3 * t + 2];
    double ax = px_of(p, a), ay = py_of(p, a);
    double bx = px_of(p, b) - ax, by = py_of(p, b) - ay;
    double cx = px_of(p, c) - ax, cy = py_of(p, c) - ay;
    double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    double inv = 0.5 / (bx * cy - by * cx);
    p.ccx[t] = ax + (cy * b2 - by * c2) * inv;
    p.ccy[t] = ay + (bx * c2 - cx * b2) * inv;
}

// a1: per-edge geometry, relative to the edge's left generator
__global__ void k_edge_geometry(SweepParams p)
{
    int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.E) return;
    int32_t l = p.edge_l[e], r = p.edge_r[e];
    double xl = p.x[l], yl = p.y[l];
    double ax = p.ccx[p.edge_ta[e]] - xl, ay = p.ccy[p.edge_ta[e]] - yl;
    double bx = p.ccx[p.edge_tb[e]] - xl, by = p.ccy[p.edge_tb[e]] - yl;
    double dx = px_of(p, r) - xl, dy = py_of(p, r) - yl;
    double ex = bx - ax, ey = by - ay;
    double L = sqrt(ex * ex + ey * ey);
    double mx = 0.5 * (ax + bx), my = 0.5 * (ay + by);
    double rinv = 1.0 / sqrt(dx * dx + dy * dy);
    p.eL[e] = L;
    p.emlx[e] = mx;
    p.emly[e] = my;
    p.emrx[e] = mx - dx;
    p.emry[e] = my - dy;
    p.enx[e] = dx * rinv;
    p.eny[e] = dy * rinv;
    p.eqx[e] = (mx - 0.5 * dx) * rinv;
    p.eqy[e] = (my - 0.5 * dy) * rinv;
}

// a1 + a2: area and centre of mass (shoelace about the generator), then the
// primitive variables.  With init_W the conserved variables are set instead.
__global__ void k_cell_geometry(SweepParams p, const double *__restrict__ init_W)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int32_t lo = p.cell_ptr[i], hi = p.cell_ptr[i + 1];
    const double xi = p.x[i], yi = p.y[i];
    int32_t tl = p.slot_tri[hi - 1];
    double ax = p.ccx[tl] - xi, ay = p.ccy[tl] - yi;
    double A2 = 0.0, sx = 0.0, sy = 0.0;
    for (int32_t s = lo; s < hi; s++) {
        int32_t t = p.slot_tri[s];
        double bx = p.ccx[t] - xi, by = p.ccy[t] - yi;
        double cr = ax * by - ay * bx;
        A2 += cr;
        sx += (ax + bx) * cr;
        sy += (ay + by) * cr;
        ax = bx;
        ay = by;
    }
    const double A = 0.5 * A2;
    const double inv3 = 1.0 / (3.0 * A2);
    p.A[i] = A;
    p.ox[i] = sx * inv3;
    p.oy[i] = sy * inv3;
    const int32_t n = p.n;
    const double gm1 = p.gamma - 1.0;
    if (init_W) {
        double rho = init_W[i], vx = init_W[n + i], vy = init_W[2 * n + i], pr = init_W[3 * n + i];
        double m = rho * A;
        p.Un[i] = m;
        p.Un[n + i] = m * vx;
        p.Un[2 * n + i] = m * vy;
        p.Un[3 * n + i] = (pr / gm1 + 0.5 * rho * (vx * vx + vy * vy)) * A;
        return;
    }
    double m = p.U[i], Px = p.U[n + i], Py = p.U[2 * n + i], E = p.U[3 * n + i];
    double invA = 1.0 / A, invm = 1.0 / m;
    double rho = m * invA, vx = Px * invm, vy = Py * invm;
    double pr = gm1 * (E - 0.5 * (Px * vx + Py * vy)) * invA;
    p.W[i] = rho;
    p.W[n + i] = vx;
    p.W[2 * n + i] = vy;
    p.W[3 * n + i] = pr;
    p.cs[i] = sqrt(p.gamma * pr / rho);
}

__device__ __forceinline__ void warp_block_min(double v, unsigned long long *dst)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    __shared__ double red[kBlock / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : DBL_MAX;
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
        if (lane == 0 && v >= 0.0) atomicMin(dst, (unsigned long long)__double_as_longlong(v));
    }
}

// a3-a6: Green-Gauss gradient (Eq. 1), limiter with the shock switch
// (Eqs. 3-8), cell-rounding mesh velocity (Section 6), per-cell time step.
__global__ void __launch_bounds__(kBlock) k_cell_gradient(SweepParams p)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double dt_cell = DBL_MAX;
    if (i < p.n) {
        const int32_t n = p.n;
        const int32_t lo = p.cell_ptr[i], hi = p.cell_ptr[i + 1];
        double Wi[4] = {p.W[i], p.W[n + i], p.W[2 * n + i], p.W[3 * n + i]};
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        double fmx[4] = {Wi[0], Wi[1], Wi[2], Wi[3]};
        double fmn[4] = {Wi[0], Wi[1], Wi[2], Wi[3]};
        bool shock = false;
        const double A = p.A[i];
        // Eqs. 3-8 look at the cells sharing an edge longer than 1e-9 sqrt(A):
        // shorter edges are point contacts whose presence depends on round-off
        const double Lmin = 1e-9 * sqrt(A);
        for (int32_t s = lo; s < hi; s++) {
            int32_t es = p.slot_edge[s];
            int32_t e = es >> 1;
            double sg = (es & 1) ? -1.0 : 1.0;
            double L = p.eL[e];
            double nx = sg * p.enx[e], ny = sg * p.eny[e];
            double qx = p.eqx[e], qy = p.eqy[e];
            double Wj[4];
            load_W(p, p.slot_nb[s], Wj);
#pragma unroll
            for (int v = 0; v < 4; v++) {
                double d = Wj[v] - Wi[v], a = 0.5 * (Wi[v] + Wj[v]);
                acc[2 * v] += L * (d * qx + a * nx);
                acc[2 * v + 1] += L * (d * qy + a * ny);
            }
            if (L > Lmin) {
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    fmx[v] = fmax(fmx[v], Wj[v]);
                    fmn[v] = fmin(fmn[v], Wj[v]);
                }
                if (fmin(Wi[3], Wj[3]) < p.delta_p * fmax(Wi[3], Wj[3])) shock = true;
            }
        }
        const double invA = 1.0 / A;
        double g[8];
#pragma unroll
        for (int c = 0; c < 8; c++) g[c] = acc[c] * invA;
        const double cs = p.cs[i];
        const double R = sqrt(A * (1.0 / M_PI));
        if (-(g[2] + g[5]) * R > p.delta_v * cs) shock = true;
        const bool use_tess = p.limiter == 2 || (p.limiter == 0 && shock);
        const double ox = p.ox[i], oy = p.oy[i];
        // alpha = min(1, min_j psi_ij) without a division per edge.
        // AREPO (Eqs. 4-5): psi_ij = (phi_max - phi_i)/dphi for dphi > 0, so the
        // minimum over those edges sits at the largest dphi (likewise for
        // dphi < 0); one division per sign and variable.
        // TESS (Eq. 6): psi_ij = max(theta (phi_j - phi_i)/dphi, 0); the
        // smallest ratio is found by cross-multiplication, divided once.
        double alpha[4];
        if (!use_tess) {
            double dpos[4] = {0, 0, 0, 0}, dneg[4] = {0, 0, 0, 0};
            for (int32_t s = lo; s < hi; s++) {
                int32_t es = p.slot_edge[s];
                int32_t e = es >> 1;
                if (!(p.eL[e] > Lmin)) continue;
                double offx = ((es & 1) ? p.emrx[e] : p.emlx[e]) - ox;
                double offy = ((es & 1) ? p.emry[e] : p.emly[e]) - oy;
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    double dphi = g[2 * v] * offx + g[2 * v + 1] * offy;
                    dpos[v] = fmax(dpos[v], dphi);
                    dneg[v] = fmin(dneg[v], dphi);
                }
            }
#pragma unroll
            for (int v = 0; v < 4; v++) {
                double a = 1.0;
                if (dpos[v] > 0.0) a = fmin(a, (fmx[v] - Wi[v]) / dpos[v]);
                if (dneg[v] < 0.0) a = fmin(a, (fmn[v] - Wi[v]) / dneg[v]);
                alpha[v] = a;
            }
        } else {
            double bn[4] = {0, 0, 0, 0}, bd[4] = {0, 0, 0, 0};  // smallest |N|/|D| so far (bd == 0: none)
            bool zero[4] = {false, false, false, false};
            for (int32_t s = lo; s < hi; s++) {
                int32_t es = p.slot_edge[s];
                int32_t e = es >> 1;
                if (!(p.eL[e] > Lmin)) continue;
                double offx = ((es & 1) ? p.emrx[e] : p.emlx[e]) - ox;
                double offy = ((es & 1) ? p.emry[e] : p.emly[e]) - oy;
                double Wj[4];
                load_W(p, p.slot_nb[s], Wj);
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    double dphi = g[2 * v] * offx + g[2 * v + 1] * offy;
                    if (dphi == 0.0) continue;
                    double num = Wj[v] - Wi[v];
                    if (!(num * dphi > 0.0)) { zero[v] = true; continue; }
                    double an = fabs(num), ad = fabs(dphi);
                    if (bd[v] == 0.0 || an * bd[v] < bn[v] * ad) { bn[v] = an; bd[v] = ad; }
                }
            }
#pragma unroll
            for (int v = 0; v < 4; v++) {
                double a = 1.0;
                if (zero[v]) a = 0.0;
                else if (bd[v] > 0.0) a = fmin(a, p.theta * bn[v] / bd[v]);
                alpha[v] = a;
            }
        }
#pragma unroll
        for (int c = 0; c < 8; c++) {
            p.g[c * n + i] = g[c];
            p.gl[c * n + i] = alpha[c >> 1] * g[c];
        }
#pragma unroll
        for (int v = 0; v < 4; v++) p.alpha[v * n + i] = alpha[v];
        p.tess[i] = use_tess ? 1 : 0;
        // Section 6: mesh-generating point velocity
        double wx = 0.0, wy = 0.0;
        if (p.motion == 0) {
            wx = Wi[1];
            wy = Wi[2];
            double d = sqrt(ox * ox + oy * oy);
            if (d > p.eta * R) {
                double f = p.chi * cs / d;
                wx += f * ox;
                wy += f * oy;
            }
        }
        p.wx[i] = wx;
        p.wy[i] = wy;
        double rx = Wi[1] - wx, ry = Wi[2] - wy;
        dt_cell = R / (cs + sqrt(rx * rx + ry * ry));
    }
    warp_block_min(dt_cell, p.dtmin_bits);
}

__device__ __forceinline__ double step_dt(const SweepParams &p)
{
    double dt = p.cfl * __longlong_as_double((long long)*p.dtmin_bits);
    return dt > p.remaining ? p.remaining : dt;
}

// half-step prediction of one side's edge state in the frame moving with wf
__device__ __forceinline__ void predict(double gam, double hdt, const double W[4], const double g[8], double offx,
                                        double offy, double wfx, double wfy, double out[4])
{
    double ux = W[1] - wfx, uy = W[2] - wfy;
    double div = g[2] + g[5];
    double irho = 1.0 / W[0];
    out[0] = W[0] + g[0] * offx + g[1] * offy - hdt * (ux * g[0] + uy * g[1] + W[0] * div);
    out[1] = W[1] + g[2] * offx + g[3] * offy - hdt * (ux * g[2] + uy * g[3] + g[6] * irho);
    out[2] = W[2] + g[4] * offx + g[5] * offy - hdt * (ux * g[4] + uy * g[5] + g[7] * irho);
    out[3] = W[3] + g[6] * offx + g[7] * offy - hdt * (ux * g[6] + uy * g[7] + gam * W[3] * div);
}

// HLLC (Toro) in the edge frame, states (rho, u_n, u_t, p)
__device__ __forceinline__ void hllc(double gam, const double L[4], const double R[4], double F[4])
{
    const double rL = L[0], uL = L[1], tL = L[2], pL = L[3];
    const double rR = R[0], uR = R[1], tR = R[2], pR = R[3];
    const double cL = sqrt(gam * pL / rL), cR = sqrt(gam * pR / rR);
    const double igm1 = 1.0 / (gam - 1.0);
    const double EL = pL * igm1 + 0.5 * rL * (uL * uL + tL * tL);
    const double ER = pR * igm1 + 0.5 * rR * (uR * uR + tR * tR);
    const double SL = fmin(uL - cL, uR - cR);
    const double SR = fmax(uL + cL, uR + cR);
    if (SL >= 0.0) {
        F[0] = rL * uL; F[1] = rL * uL * uL + pL; F[2] = rL * uL * tL; F[3] = uL * (EL + pL);
        return;
    }
    if (SR <= 0.0) {
        F[0] = rR * uR; F[1] = rR * uR * uR + pR; F[2] = rR * uR * tR; F[3] = uR * (ER + pR);
        return;
    }
    const double mL = rL * (SL - uL), mR = rR * (SR - uR);
    const double Ss = (pR - pL + uL * mL - uR * mR) / (mL - mR);
    if (Ss >= 0.0) {
        const double f = mL / (SL - Ss);
        const double Es = f * (EL / rL + (Ss - uL) * (Ss + pL / mL));
        F[0] = rL * uL + SL * (f - rL);
        F[1] = rL * uL * uL + pL + SL * (f * Ss - rL * uL);
        F[2] = rL * uL * tL + SL * (f * tL - rL * tL);
        F[3] = uL * (EL + pL) + SL * (Es - EL);
    } else {
        const double f = mR / (SR - Ss);
        const double Es = f * (ER / rR + (Ss - uR) * (Ss + pR / mR));
        F[0] = rR * uR + SR * (f - rR);
        F[1] = rR * uR * uR + pR + SR * (f * Ss - rR * uR);
        F[2] = rR * uR * tR + SR * (f * tR - rR * tR);
        F[3] = uR * (ER + pR) + SR * (Es - ER);
    }
}

// a7: one flux per edge in the frame of the moving edge
__global__ void __launch_bounds__(kBlock) k_edge_flux(SweepParams p)
{
    int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.E) return;
    const int32_t n = p.n;
    const double dt = step_dt(p);
    const double hdt = 0.5 * dt;
    const int32_t l = p.edge_l[e];
    int32_t xf;
    const int32_t k = src_of(p, p.edge_r[e], xf);
    const double sx = (xf & 1) ? -1.0 : 1.0, sy = (xf & 2) ? -1.0 : 1.0;
    double Wl[4] = {p.W[l], p.W[n + l], p.W[2 * n + l], p.W[3 * n + l]};
    double Wr[4] = {p.W[k], sx * p.W[n + k], sy * p.W[2 * n + k], p.W[3 * n + k]};
    double gl[8], gr[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
        gl[c] = p.gl[c * n + l];
        gr[c] = p.gl[c * n + k];
    }
    // mirrored source: each derivative takes the flip of its axis, velocity
    // components also the flip of their own axis
    gr[0] *= sx; gr[1] *= sy;
    gr[3] *= sx * sy;
    gr[4] *= sx * sy;
    gr[6] *= sx; gr[7] *= sy;
    const double wlx = p.wx[l], wly = p.wy[l];
    const double wrx = sx * p.wx[k], wry = sy * p.wy[k];
    const double orx = sx * p.ox[k], ory = sy * p.oy[k];
    const double L = p.eL[e];
    const double nx = p.enx[e], ny = p.eny[e];
    const double qx = p.eqx[e], qy = p.eqy[e];
    // velocity of the perpendicular bisector at the edge midpoint
    const double dwc = (wrx - wlx) * qx + (wry - wly) * qy;
    const double wfx = 0.5 * (wlx + wrx) - dwc * nx;
    const double wfy = 0.5 * (wly + wry) - dwc * ny;
    double Sl[4], Sr[4];
    predict(p.gamma, hdt, Wl, gl, p.emlx[e] - p.ox[l], p.emly[e] - p.oy[l], wfx, wfy, Sl);
    predict(p.gamma, hdt, Wr, gr, p.emrx[e] - orx, p.emry[e] - ory, wfx, wfy, Sr);
    const double tx = -ny, ty = nx;
    double WL[4] = {Sl[0], (Sl[1] - wfx) * nx + (Sl[2] - wfy) * ny, (Sl[1] - wfx) * tx + (Sl[2] - wfy) * ty, Sl[3]};
    double WR[4] = {Sr[0], (Sr[1] - wfx) * nx + (Sr[2] - wfy) * ny, (Sr[1] - wfx) * tx + (Sr[2] - wfy) * ty, Sr[3]};
    double Fe[4];
    hllc(p.gamma, WL, WR, Fe);
    const double Fmx = Fe[1] * nx + Fe[2] * tx, Fmy = Fe[1] * ny + Fe[2] * ty;
    p.F[e] = L * Fe[0];
    p.F[p.E + e] = L * (Fmx + Fe[0] * wfx);
    p.F[2 * p.E + e] = L * (Fmy + Fe[0] * wfy);
    p.F[3 * p.E + e] = L * (Fe[3] + Fmx * wfx + Fmy * wfy + 0.5 * (wfx * wfx + wfy * wfy) * Fe[0]);
}

// a8 + a9: conservative update (fixed CSR order, no atomics), advance points
__global__ void __launch_bounds__(kBlock) k_cell_update(SweepParams p)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int32_t n = p.n;
    const double dt = step_dt(p);
    if (i == 0) *p.dt_out = dt;
    const int32_t lo = p.cell_ptr[i], hi = p.cell_ptr[i + 1];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int32_t s = lo; s < hi; s++) {
        int32_t es = p.slot_edge[s];
        int32_t e = es >> 1;
        double f0 = p.F[e], f1 = p.F[p.E + e], f2 = p.F[2 * p.E + e], f3 = p.F[3 * p.E + e];
        if (es & 1) { s0 -= f0; s1 -= f1; s2 -= f2; s3 -= f3; }
        else { s0 += f0; s1 += f1; s2 += f2; s3 += f3; }
    }
    double m = p.U[i] - dt * s0;
    double Px = p.U[n + i] - dt * s1;
    double Py = p.U[2 * n + i] - dt * s2;
    double E = p.U[3 * n + i] - dt * s3;
    p.Un[i] = m;
    p.Un[n + i] = Px;
    p.Un[2 * n + i] = Py;
    p.Un[3 * n + i] = E;
    int32_t st = 0;
    if (!(isfinite(m) && isfinite(Px) && isfinite(Py) && isfinite(E))) st |= ST_NAN;
    else if (!(m > 0.0) || !(E - 0.5 * (Px * Px + Py * Py) / m > 0.0)) st |= ST_NEGATIVE;
    double xn = p.x[i] + dt * p.wx[i], yn = p.y[i] + dt * p.wy[i];
    if (p.boundary == 1) {
        const double Lx = p.x1 - p.x0, Ly = p.y1 - p.y0;
        if (xn < p.x0) xn += Lx;
        else if (xn >= p.x1) xn -= Lx;
        if (yn < p.y0) yn += Ly;
        else if (yn >= p.y1) yn -= Ly;
    } else if (!(xn > p.x0 && xn < p.x1 && yn > p.y0 && yn < p.y1)) {
        st |= ST_LEFT_BOX;
    }
    p.xn[i] = xn;
    p.yn[i] = yn;
    if (st) atomicOr(p.status, st);
}

inline int blocks(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }

}  // namespace

const char *stage_name(int k)
{
    static const char *names[NUM_STAGES] = {"k_circumcentre", "k_edge_geometry", "k_cell_geometry", "dt_reset",
                                            "k_cell_gradient", "k_edge_flux", "k_cell_update"};
    return k >= 0 && k < NUM_STAGES ? names[k] : "";
}

void launch_stage(int k, const SweepParams &p, const double *init_W, cudaStream_t st)
{
    switch (k) {
    case K_CIRCUMCENTRE:
        if (p.T > 0) k_circumcentre<<<blocks(p.T), kBlock, 0, st>>>(p);
        break;
    case K_EDGE_GEOMETRY:
        if (p.E > 0) k_edge_geometry<<<blocks(p.E), kBlock, 0, st>>>(p);
        break;
    case K_CELL_GEOMETRY:
        if (p.n > 0) k_cell_geometry<<<blocks(p.n), kBlock, 0, st>>>(p, init_W);
        break;
    case K_DT_RESET:
        cudaMemsetAsync(p.dtmin_bits, 0x7f, sizeof(unsigned long long), st);
        break;
    case K_CELL_GRADIENT:
        if (p.n > 0) k_cell_gradient<<<blocks(p.n), kBlock, 0, st>>>(p);
        break;
    case K_EDGE_FLUX:
        if (p.E > 0) k_edge_flux<<<blocks(p.E), kBlock, 0, st>>>(p);
        break;
    case K_CELL_UPDATE:
        if (p.n > 0) k_cell_update<<<blocks(p.n), kBlock, 0, st>>>(p);
        break;
    default:
        break;
    }
}

}  // namespace rich
