// C ABI of the library (include/rich.h): owns the device memory of a
// simulation, runs the host tessellation (a0) and enqueues the device sweep
// (a1-a9) on a CUDA stream.  There is no CPU fallback: without a CUDA device
// rich_init_mesh fails with RICH_ENODEV.
#include <array>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rich.h"
#include "api_internal.h"
#include "mesh.h"
#include "sweep.cuh"
#include "threadpool.h"

namespace rich {
namespace {
thread_local std::string g_last_error;
}
int set_error(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}
const char *last_error() { return g_last_error.c_str(); }
}  // namespace rich

namespace {

using rich::DBuf;
using rich::now_ms;
using rich::upload;
#define CUDA_TRY RICH_CUDA_TRY

int fail(int code, const std::string &msg) { return rich::set_error(code, msg); }

int mesh_rc(int rc)
{
    switch (rc) {
    case 0: return RICH_OK;
    case -2: return fail(RICH_EDUPLICATE, "two generating points coincide");
    case -4: return fail(RICH_ETOOFEW, "too few points: the ghost band cannot close every cell");
    default: return fail(RICH_ETESS, "tessellation failed");
    }
}

}  // namespace

namespace rich {
bool valid_config(const rich_config *c)
{
    return c && c->gamma > 1.0 && std::isfinite(c->gamma) && c->cfl > 0.0 && c->x1 > c->x0 && c->y1 > c->y0 &&
           (c->boundary == RICH_BC_REFLECTIVE || c->boundary == RICH_BC_PERIODIC) &&
           (c->motion == RICH_MESH_LAGRANGIAN || c->motion == RICH_MESH_EULERIAN) && c->limiter >= 0 &&
           c->limiter <= 2 && (c->scheme == RICH_SCHEME_EXTRAPOLATED || c->scheme == RICH_SCHEME_TIME_CENTRED) && (c->precision == RICH_FP64 || c->precision == RICH_FP32_SPLIT) && c->chi >= 0 &&
           c->eta >= 0 && c->theta >= 0 && c->delta_p >= 0 && c->delta_v >= 0;
}

bool point_inside(const rich_config *c, double x, double y)
{
    if (c->boundary == RICH_BC_PERIODIC) return x >= c->x0 && x < c->x1 && y >= c->y0 && y < c->y1;
    return x > c->x0 && x < c->x1 && y > c->y0 && y < c->y1;
}

}  // namespace rich
using rich::point_inside;
using rich::valid_config;

struct rich_sim {
    rich_config cfg{};
    int32_t n = 0;
    std::vector<int32_t> perm;  // internal -> caller index
    // host copy of the points (internal order), page-locked: x at [0, n),
    // y at [n, 2n), then the dt of the sweep that moved them
    rich::HBuf hpts;
    double *hx() const { return hpts.as<double>(); }
    double *hy() const { return hpts.as<double>() + n; }
    rich::MeshWork mw;  // (edge list built on the device: see tessellate)
    rich::HostMesh hm;
    std::unique_ptr<rich::ThreadPool> pool;  // host threads of the tile-parallel tessellation
    rich_sim() { mw.host_edges = false; }
    double t = 0.0;
    int cur = 0;
    // time-centred scheme: 1 between its two sweeps (buffers [2] then hold
    // the half-step points and state)
    int tc_phase = 0;
    bool tess_current = false;
    bool pending = false;
    bool geometry_current = false;
    int diag_pts = 0;  // points buffer of the last completed sweep
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // early read of a sweep's new points (rich_step): copied on their own
    // stream once the point motion is done, while the sweep goes on
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_moved = nullptr, ev_copied = nullptr;
    bool profiling = false;
    cudaEvent_t kev[rich::NUM_STAGES + 1] = {};
    double kms[rich::NUM_STAGES] = {};
    double last_dt = 0.0;
    // device buffers
    DBuf x[3], y[3], U[3];
    DBuf A, o, W, cs, g, gl, alpha, w, tess, cell_ptr, corder, initW, rounding, p64, psrc;
    bool diagnostics = true;
    DBuf gx, gy, gsrc, gxf, gshift, eoff, toff;
    DBuf perm_dev, unperm;  // caller index of each internal cell; reordered state for reads
    DBuf tri, ccx, ccy;
    DBuf slot_nb, slot_tri, slot_edge;
    DBuf edge_l, edge_r, edge_ta, edge_tb, eL, emlx, emly, emrx, emry, enx, eny, eqx, eqy, F, ePM;
    DBuf scal;   // dtmin bits, dt, status
    DBuf instp;  // one InstParams
    rich::InstParams inst_host{};  // staging for the parameter upload

    ~rich_sim()
    {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (ev_moved) cudaEventDestroy(ev_moved);
        if (ev_copied) cudaEventDestroy(ev_copied);
        if (copy_stream) cudaStreamDestroy(copy_stream);
        for (cudaEvent_t e : kev)
            if (e) cudaEventDestroy(e);
        if (own_stream) cudaStreamDestroy(own_stream);
    }

    template <class R> rich::SweepParams<R> params() const
    {
        rich::SweepParams<R> p{};
        p.inst = instp.as<rich::InstParams>();
        p.cell_inst = nullptr;
        p.n_inst = 1;
        p.diagnostics = diagnostics ? 1 : 0;
        p.motion = 1;
        p.n = n;
        p.ng = hm.g;
        p.T = hm.n_tris;
        p.E = hm.n_edges;
        p.S = (int32_t)hm.slot_nb.size();
        // extrapolated fluxes: [cur] -> [1 - cur].  Time-centred: [cur] -> [2]
        // by half a step, then primitives and mesh of [2], update of [cur]
        // into [1 - cur]
        const int src = pts(), dst = next_pts();
        p.x = x[src].as<double>(); p.y = y[src].as<double>();
        p.xn = x[dst].as<double>(); p.yn = y[dst].as<double>();
        p.x0 = x[cur].as<double>(); p.y0 = y[cur].as<double>();
        p.gx = gx.as<double>(); p.gy = gy.as<double>();
        p.tri = tri.as<int32_t>(); p.cell_ptr = cell_ptr.as<int32_t>(); p.cell_order = corder.as<int32_t>();
        p.slot_nb = slot_nb.as<int32_t>(); p.slot_tri = slot_tri.as<int32_t>(); p.slot_edge = slot_edge.as<int32_t>();
        p.edge_l = edge_l.as<int32_t>(); p.edge_r = edge_r.as<int32_t>();
        p.edge_ta = edge_ta.as<int32_t>(); p.edge_tb = edge_tb.as<int32_t>();
        p.ghost_src = gsrc.as<int32_t>(); p.ghost_xf = gxf.as<int32_t>();
        p.ccx = ccx.as<double>(); p.ccy = ccy.as<double>(); p.A = A.as<double>();
        p.eL = eL.as<R>(); p.emlx = emlx.as<R>(); p.emly = emly.as<R>();
        p.emrx = emrx.as<R>(); p.emry = emry.as<R>();
        p.enx = enx.as<R>(); p.eny = eny.as<R>(); p.eqx = eqx.as<R>(); p.eqy = eqy.as<R>();
        p.ePM = ePM.as<rich::Vec4<R>>();
        p.U = U[src].as<double>(); p.Un = U[dst].as<double>(); p.U0 = U[cur].as<double>();
        p.W = W.as<rich::Vec4<R>>(); p.o = o.as<rich::Vec2<R>>(); p.cs = cs.as<R>();
        p.g = g.as<rich::Vec4<R>>(); p.gl = gl.as<rich::Vec4<R>>(); p.alpha = alpha.as<rich::Vec4<R>>();
        p.w = w.as<rich::Vec2<R>>();
        p.rounding = rounding.as<uint8_t>(); p.p64 = p64.as<double>();
        p.tess = tess.as<int32_t>(); p.F = F.as<rich::Vec4<R>>(); p.psrc = psrc.as<rich::Vec4<R>>();
        char *sc = scal.as<char>();
        p.dtmin_bits = reinterpret_cast<unsigned long long *>(sc);
        p.dt_out = reinterpret_cast<double *>(sc + 8);
        p.status = reinterpret_cast<int32_t *>(sc + 16);
        return p;
    }

    size_t rsize() const { return cfg.precision == RICH_FP32_SPLIT ? sizeof(float) : sizeof(double); }
    bool time_centred() const { return cfg.scheme == RICH_SCHEME_TIME_CENTRED; }
    // buffer of the points (and state) that the current mesh and sweep describe
    int pts() const { return tc_phase == 1 ? 2 : cur; }
    // buffer the sweep writes its moved points (and state) to
    int next_pts() const { return time_centred() && tc_phase == 0 ? 2 : 1 - cur; }

    // scheme parameters of this simulation with the time left to t_end
    rich::InstParams inst_params(double remaining, bool init = false) const
    {
        rich::InstParams ip{};
        ip.init = init ? 1 : 0;
        ip.gamma = cfg.gamma; ip.igm1 = 1.0 / (cfg.gamma - 1.0); ip.gamma_f = (float)ip.gamma; ip.igm1_f = (float)ip.igm1; ip.cfl = cfg.cfl; ip.chi = cfg.chi; ip.eta = cfg.eta; ip.theta = cfg.theta;
        ip.delta_v = cfg.delta_v; ip.delta_p = cfg.delta_p; ip.chi_f = (float)ip.chi; ip.theta_f = (float)ip.theta; ip.delta_v_f = (float)ip.delta_v;
        ip.x0 = cfg.x0; ip.x1 = cfg.x1; ip.y0 = cfg.y0; ip.y1 = cfg.y1;
        ip.remaining = remaining;
        ip.boundary = cfg.boundary; ip.motion = cfg.motion; ip.limiter = cfg.limiter;
        ip.phase = time_centred() ? 1 + tc_phase : 0;
        return ip;
    }

    // launch stage k of the sweep in the handle's precision (motion false:
    // the geometry stage leaves the mesh velocity and time step alone)
    void launch(int k, const double *init_W, double *Un_override = nullptr, bool motion = true) const
    {
        if (cfg.precision == RICH_FP32_SPLIT) {
            rich::SweepParams<float> p = params<float>();
            if (Un_override) p.Un = Un_override;
            p.motion = motion ? 1 : 0;
            rich::launch_stage<float>(k, p, init_W, stream);
        } else {
            rich::SweepParams<double> p = params<double>();
            if (Un_override) p.Un = Un_override;
            p.motion = motion ? 1 : 0;
            rich::launch_stage<double>(k, p, init_W, stream);
        }
    }

    // the mesh sizes of the current tessellation
    int32_t nT() const { return hm.n_tris; }
    int32_t nE() const { return hm.n_edges; }
};

namespace {

int alloc_cells(rich_sim *s)
{
    const size_t n = (size_t)s->n, d = sizeof(double), r = s->rsize();
    for (int k = 0; k < (s->time_centred() ? 3 : 2); k++) {
        CUDA_TRY(s->x[k].ensure(n * d));
        CUDA_TRY(s->y[k].ensure(n * d));
        CUDA_TRY(s->U[k].ensure(4 * n * d));
    }
    CUDA_TRY(s->A.ensure(n * d)); CUDA_TRY(s->o.ensure(2 * n * r));
    CUDA_TRY(s->W.ensure(4 * n * r)); CUDA_TRY(s->cs.ensure(n * r));
    CUDA_TRY(s->g.ensure(8 * n * r)); CUDA_TRY(s->gl.ensure(8 * n * r)); CUDA_TRY(s->alpha.ensure(4 * n * r));
    CUDA_TRY(s->w.ensure(2 * n * r)); CUDA_TRY(s->tess.ensure(n * 4)); CUDA_TRY(s->psrc.ensure(4 * n * r));
    CUDA_TRY(s->rounding.ensure(n)); CUDA_TRY(s->p64.ensure(n * d));
    CUDA_TRY(s->scal.ensure(64));
    CUDA_TRY(cudaMemsetAsync(s->scal.p, 0, 64, s->stream));
    CUDA_TRY(s->instp.ensure(sizeof(rich::InstParams)));
    return RICH_OK;
}

// a0 on the host: the mesh of the points in hx, hy (the device mesh is
// then out of date until upload_mesh)
int build_mesh(rich_sim *s, rich_step_info *info)
{
    rich::Range range("rich tessellate (a0)");
    const double t1 = now_ms();
    rich::BoxConfig box{s->cfg.boundary, s->cfg.x0, s->cfg.x1, s->cfg.y0, s->cfg.y1};
    const int rc = rich::build_host_mesh(box, s->n, s->hx(), s->hy(), s->mw, s->hm, s->pool.get());
    if (info) info->tess_ms += now_ms() - t1;
    return rc ? mesh_rc(rc) : RICH_OK;
}

// upload of the host mesh; the triangle and edge lists are built on the
// device from the rings (the host sends each cell's first owned triangle
// and edge, and the ghosts' periodic shifts).  Nothing on the stream may
// still read the old mesh: buffers that grow are reallocated.
int upload_mesh(rich_sim *s, rich_step_info *info)
{
    const double t2 = now_ms();
    const rich::HostMesh &m = s->hm;
    const size_t T = (size_t)m.n_tris, E = (size_t)m.n_edges, d = sizeof(double);
    CUDA_TRY(upload(s->gx, m.gx, s->stream));
    CUDA_TRY(upload(s->gy, m.gy, s->stream));
    CUDA_TRY(upload(s->gsrc, m.ghost_src, s->stream));
    CUDA_TRY(upload(s->gxf, m.ghost_xf, s->stream));
    CUDA_TRY(upload(s->cell_ptr, m.cell_ptr, s->stream));
    CUDA_TRY(upload(s->corder, m.cell_order, s->stream));
    CUDA_TRY(upload(s->slot_nb, m.slot_nb, s->stream));
    CUDA_TRY(upload(s->toff, m.tri_off, s->stream));
    CUDA_TRY(upload(s->eoff, m.edge_off, s->stream));
    CUDA_TRY(upload(s->gshift, m.ghost_shift, s->stream));
    const size_t S = m.slot_nb.size();
    CUDA_TRY(s->tri.ensure((3 * T + 3) * sizeof(int32_t)));
    CUDA_TRY(s->slot_tri.ensure((S + 1) * sizeof(int32_t)));
    CUDA_TRY(s->slot_edge.ensure((S + 1) * sizeof(int32_t)));
    for (DBuf *b : {&s->edge_l, &s->edge_r, &s->edge_ta, &s->edge_tb}) CUDA_TRY(b->ensure((E + 1) * sizeof(int32_t)));
    int32_t *bad = reinterpret_cast<int32_t *>(s->scal.as<char>() + 24);
    int32_t *bad_tri = reinterpret_cast<int32_t *>(s->scal.as<char>() + 28);
    CUDA_TRY(rich::launch_build_tris(s->n, (int32_t)S, s->cell_ptr.as<int32_t>(), s->slot_nb.as<int32_t>(),
                                     s->toff.as<int32_t>(), s->tri.as<int32_t>(), s->slot_tri.as<int32_t>(), bad_tri,
                                     s->stream));
    CUDA_TRY(rich::launch_build_edges(s->n, (int32_t)S, s->cell_ptr.as<int32_t>(), s->slot_nb.as<int32_t>(),
                                      s->slot_tri.as<int32_t>(), s->gsrc.as<int32_t>(), s->gshift.as<int32_t>(),
                                      s->eoff.as<int32_t>(), s->cfg.boundary == RICH_BC_PERIODIC ? 1 : 0,
                                      nullptr, nullptr, s->slot_edge.as<int32_t>(), s->edge_l.as<int32_t>(), s->edge_r.as<int32_t>(),
                                      s->edge_ta.as<int32_t>(), s->edge_tb.as<int32_t>(), bad, s->stream));
    int32_t bad_h[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(bad_h, bad, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    const size_t r = s->rsize();
    CUDA_TRY(s->ccx.ensure((T + 1) * d)); CUDA_TRY(s->ccy.ensure((T + 1) * d));
    for (DBuf *b : {&s->eL, &s->emlx, &s->emly, &s->emrx, &s->emry, &s->enx, &s->eny, &s->eqx, &s->eqy})
        CUDA_TRY(b->ensure((E + 1) * r));
    CUDA_TRY(s->F.ensure((4 * E + 4) * sizeof(double)));
    CUDA_TRY(s->ePM.ensure((4 * E + 4) * r));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    const double t3 = now_ms();
    if (bad_h[1]) return fail(RICH_ETESS, "a triangle of a ring is missing from its owner's ring");
    if (bad_h[0]) return fail(RICH_ETESS, "an edge of a ring has no partner in the other cell's ring");
    s->tess_current = true;
    if (info) {
        info->copy_ms += t3 - t2;
        info->n_ghost = m.g;
        info->n_tri = (int64_t)T;
        info->n_edges = (int64_t)E;
        info->n_slots = (int64_t)m.slot_nb.size();
    }
    return RICH_OK;
}

// host tessellation of the current points + upload of the connectivity
int tessellate(rich_sim *s, rich_step_info *info, bool fetch_points)
{
    if (fetch_points) {
        const double t0 = now_ms();
        const int q = s->pts();
        CUDA_TRY(cudaMemcpyAsync(s->hx(), s->x[q].p, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaMemcpyAsync(s->hy(), s->y[q].p, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (info) info->copy_ms += now_ms() - t0;
    }
    s->tess_current = false;
    int rc = build_mesh(s, info);
    if (rc) return rc;
    return upload_mesh(s, info);
}

}  // namespace

extern "C" {

void rich_default_config(rich_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->gamma = 5.0 / 3.0;
    c->cfl = 0.3;
    c->boundary = RICH_BC_PERIODIC;
    c->x0 = 0.0; c->x1 = 1.0; c->y0 = 0.0; c->y1 = 1.0;
    c->motion = RICH_MESH_LAGRANGIAN;
    c->chi = 0.15; c->eta = 0.02;
    c->theta = 0.5; c->delta_v = 0.2; c->delta_p = 0.7;
    c->limiter = RICH_LIM_SWITCHED;
    c->scheme = RICH_SCHEME_EXTRAPOLATED;
    c->precision = RICH_FP64;
}

const char *rich_strerror(int code)
{
    switch (code) {
    case RICH_OK: return "ok";
    case RICH_EINVAL: return "invalid argument";
    case RICH_EDUPLICATE: return "coincident generating points";
    case RICH_ETESS: return "tessellation failed";
    case RICH_ETOOFEW: return "too few points for the ghost band";
    case RICH_ENEGATIVE: return "non-positive mass or thermal energy, or a point left the box";
    case RICH_ENAN: return "non-finite value";
    case RICH_ENOMEM: return "out of memory";
    case RICH_ECUDA: return "CUDA error";
    case RICH_ENODEV: return "no CUDA device";
    case RICH_ESTATE: return "call not valid in the current state";
    default: return "unknown error";
    }
}

const char *rich_last_error(void) { return rich::last_error(); }

int64_t rich_num_cells(const rich_sim *s) { return s ? s->n : -1; }

// Shared by rich_init_mesh (f = primitives rho, vx, vy, p) and
// rich_init_conserved (f = extensive m, px, py, E at time t0, cells in the
// internal order `order` when given).
static int create_sim(const rich_config *cfg, int64_t n, const double *x, const double *y, const double *const f[4],
                      bool conserved, double t0, const int64_t *order, rich_sim **out)
{
    if (!out) return fail(RICH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!valid_config(cfg)) return fail(RICH_EINVAL, "invalid configuration");
    if (n < 3 || n > (int64_t)1 << 30) return fail(RICH_EINVAL, "n must be in [3, 2^30]");
    if (!x || !y || !f[0] || !f[1] || !f[2] || !f[3]) return fail(RICH_EINVAL, "NULL input array");
    if (!std::isfinite(t0)) return fail(RICH_EINVAL, "bad start time");
    for (int64_t i = 0; i < n; i++) {
        if (!std::isfinite(x[i]) || !std::isfinite(y[i]) || !point_inside(cfg, x[i], y[i]))
            return fail(RICH_EINVAL, "point " + std::to_string(i) + " outside the box");
        bool good = std::isfinite(f[0][i]) && std::isfinite(f[1][i]) && std::isfinite(f[2][i]) && std::isfinite(f[3][i]);
        if (conserved) good = good && f[0][i] > 0 && 2.0 * f[0][i] * f[3][i] - (f[1][i] * f[1][i] + f[2][i] * f[2][i]) > 0;
        else good = good && f[0][i] > 0 && f[3][i] > 0;
        if (!good) return fail(RICH_EINVAL, "bad field values at point " + std::to_string(i));
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(RICH_ENODEV, "no CUDA device");
    rich_sim *s = new (std::nothrow) rich_sim();
    if (!s) return fail(RICH_ENOMEM, "host allocation");
    s->cfg = *cfg;
    s->n = (int32_t)n;
    s->t = t0;
    s->pool.reset(new (std::nothrow) rich::ThreadPool((int)std::max(1u, std::thread::hardware_concurrency())));
    if (!s->pool) {
        delete s;
        return fail(RICH_ENOMEM, "host thread pool");
    }
    if (order) {
        // the caller's internal order (a checkpoint's): must be a permutation
        s->perm.resize(n);
        std::vector<char> seen(n, 0);
        for (int64_t k = 0; k < n; k++) {
            if (order[k] < 0 || order[k] >= n || seen[order[k]]) {
                delete s;
                return fail(RICH_EINVAL, "order is not a permutation");
            }
            seen[order[k]] = 1;
            s->perm[k] = (int32_t)order[k];
        }
    } else {
        // renumber cells along a Hilbert curve for locality
        rich::hilbert_order(s->n, x, y, s->perm);
    }
    int rc = RICH_OK;
    auto bail = [&](int code) { delete s; return code; };
    if (s->hpts.ensure((2 * (size_t)n + 1) * sizeof(double)) != cudaSuccess)
        return bail(fail(RICH_ENOMEM, "page-locked host points"));
    std::vector<double> Fh(4 * (size_t)n);
    double *hx = s->hx(), *hy = s->hy();
    for (int32_t k = 0; k < s->n; k++) {
        int32_t u = s->perm[k];
        hx[k] = x[u];
        hy[k] = y[u];
        for (int c = 0; c < 4; c++) Fh[(size_t)c * n + k] = f[c][u];
    }
    if (cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(RICH_ECUDA, "stream creation failed"));
    s->stream = s->own_stream;
    if (cudaEventCreate(&s->ev0) != cudaSuccess || cudaEventCreate(&s->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_moved, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_copied, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(RICH_ECUDA, "event creation failed"));
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(RICH_ECUDA, "stream creation failed"));
    if ((rc = alloc_cells(s)) != RICH_OK) return bail(rc);
    if (s->x[0].ensure(n * 8) != cudaSuccess) return bail(fail(RICH_ENOMEM, "device points"));
    if (upload(s->perm_dev, s->perm, s->stream) != cudaSuccess) return bail(fail(RICH_ENOMEM, "device order"));
    cudaMemcpyAsync(s->x[0].p, hx, n * 8, cudaMemcpyHostToDevice, s->stream);
    cudaMemcpyAsync(s->y[0].p, hy, n * 8, cudaMemcpyHostToDevice, s->stream);
    if ((rc = tessellate(s, nullptr, false)) != RICH_OK) return bail(rc);
    if (conserved) {
        if (cudaMemcpyAsync(s->U[0].p, Fh.data(), 4 * n * 8, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            return bail(fail(RICH_ECUDA, "state upload"));
    } else {
        if (s->initW.ensure(4 * n * 8) != cudaSuccess) return bail(fail(RICH_ENOMEM, "device primitives"));
        cudaMemcpyAsync(s->initW.p, Fh.data(), 4 * n * 8, cudaMemcpyHostToDevice, s->stream);
        s->inst_host = s->inst_params(0.0, true);
        if (cudaMemcpyAsync(s->instp.p, &s->inst_host, sizeof(rich::InstParams), cudaMemcpyHostToDevice,
                            s->stream) != cudaSuccess)
            return bail(fail(RICH_ECUDA, "parameter upload"));
        for (int k = 0; k < rich::GEOMETRY_STAGES; k++) s->launch(k, s->initW.as<double>(), s->U[0].as<double>());
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(fail(RICH_ECUDA, std::string("init: ") + cudaGetErrorString(e)));
    s->geometry_current = false;  // W not yet derived from U
    *out = s;
    return RICH_OK;
}

int rich_init_mesh(const rich_config *cfg, int64_t n, const double *x, const double *y, const double *rho,
                   const double *vx, const double *vy, const double *p, rich_sim **out)
{
    const double *f[4] = {rho, vx, vy, p};
    return create_sim(cfg, n, x, y, f, false, 0.0, nullptr, out);
}

int rich_init_conserved(const rich_config *cfg, int64_t n, const double *x, const double *y, const double *m,
                        const double *px, const double *py, const double *E, double t, const int64_t *order,
                        rich_sim **out)
{
    const double *f[4] = {m, px, py, E};
    return create_sim(cfg, n, x, y, f, true, t, order, out);
}

int rich_get_order(const rich_sim *s, int64_t n, int64_t *order)
{
    if (!s || n != s->n || !order) return fail(RICH_EINVAL, "bad arguments");
    for (int32_t k = 0; k < s->n; k++) order[k] = s->perm[k];
    return RICH_OK;
}

double rich_time(const rich_sim *s) { return s ? s->t : -1.0; }

void rich_destroy(rich_sim *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    delete s;
}

int rich_set_stream(rich_sim *s, void *stream)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->stream = stream ? static_cast<cudaStream_t>(stream) : s->own_stream;
    return RICH_OK;
}

int rich_set_diagnostics(rich_sim *s, int32_t on)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    if (s->pending) return fail(RICH_ESTATE, "a sweep is pending; call rich_sync first");
    s->diagnostics = on != 0;
    return RICH_OK;
}

int rich_set_profiling(rich_sim *s, int32_t on)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    if (on && !s->kev[0])
        for (cudaEvent_t &e : s->kev) CUDA_TRY(cudaEventCreate(&e));
    s->profiling = on != 0;
    return RICH_OK;
}

int rich_kernel_times(rich_sim *s, int32_t cap, double *ms, int32_t *count)
{
    if (!s || !count) return fail(RICH_EINVAL, "bad arguments");
    *count = rich::NUM_STAGES;
    if (!s->profiling) return fail(RICH_ESTATE, "profiling is off");
    for (int k = 0; k < rich::NUM_STAGES && k < cap; k++) ms[k] = s->kms[k];
    return RICH_OK;
}

const char *rich_kernel_name(int32_t k) { return rich::stage_name(k); }

int rich_tessellate(rich_sim *s, rich_step_info *info)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    if (s->pending) return fail(RICH_ESTATE, "a sweep is pending; call rich_sync first");
    return tessellate(s, info, true);
}

// Launch the sweep; with read_points the moved points and the step's dt
// are copied into hpts on the copy stream as soon as the point motion is
// done (ev_copied marks their arrival) while the rest of the sweep runs.
static int launch_sweep(rich_sim *s, double t_end, bool read_points)
{
    rich::Range range("rich sweep launch (a1-a9)");
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    if (!s->tess_current) return fail(RICH_ESTATE, "no current tessellation");
    if (s->pending) return fail(RICH_ESTATE, "a sweep is pending; call rich_sync first");
    if (!(t_end > s->t)) return fail(RICH_EINVAL, "t_end must exceed the current time");
    CUDA_TRY(cudaStreamSynchronize(s->stream));  // the staging struct may be in flight
    s->inst_host = s->inst_params(t_end - s->t);
    CUDA_TRY(cudaMemcpyAsync(s->instp.p, &s->inst_host, sizeof(rich::InstParams), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaEventRecord(s->ev0, s->stream));
    for (int k = 0; k < rich::NUM_STAGES; k++) {
        if (s->profiling) CUDA_TRY(cudaEventRecord(s->kev[k], s->stream));
        s->launch(k, nullptr);
        if (read_points && k == rich::K_ADVANCE) {
            const size_t N = (size_t)s->n;
            const int q = s->next_pts();
            CUDA_TRY(cudaEventRecord(s->ev_moved, s->stream));
            CUDA_TRY(cudaStreamWaitEvent(s->copy_stream, s->ev_moved, 0));
            CUDA_TRY(cudaMemcpyAsync(s->hx(), s->x[q].p, N * 8, cudaMemcpyDeviceToHost, s->copy_stream));
            CUDA_TRY(cudaMemcpyAsync(s->hy(), s->y[q].p, N * 8, cudaMemcpyDeviceToHost, s->copy_stream));
            CUDA_TRY(cudaMemcpyAsync(s->hy() + N, s->scal.as<char>() + 8, 8, cudaMemcpyDeviceToHost, s->copy_stream));
            CUDA_TRY(cudaEventRecord(s->ev_copied, s->copy_stream));
        }
    }
    if (s->profiling) CUDA_TRY(cudaEventRecord(s->kev[rich::NUM_STAGES], s->stream));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(s->ev1, s->stream));
    s->pending = true;
    return RICH_OK;
}

int rich_sweep(rich_sim *s, double t_end) { return launch_sweep(s, t_end, false); }

int rich_sync(rich_sim *s, rich_step_info *info)
{
    rich::Range range("rich sync");
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    if (!s->pending) return fail(RICH_ESTATE, "no sweep pending");
    double t0 = now_ms();
    double dt = 0.0;
    int32_t status = 0;
    char *sc = s->scal.as<char>();
    CUDA_TRY(cudaMemcpyAsync(&dt, sc + 8, 8, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaMemcpyAsync(&status, sc + 16, 4, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->pending = false;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, s->ev0, s->ev1);
    if (s->profiling)
        for (int k = 0; k < rich::NUM_STAGES; k++) {
            float km = 0.0f;
            cudaEventElapsedTime(&km, s->kev[k], s->kev[k + 1]);
            s->kms[k] = km;
        }
    if (info) {
        info->sweep_ms += ms;
        info->copy_ms += now_ms() - t0;
    }
    s->geometry_current = true;  // diagnostics describe this sweep
    s->diag_pts = s->pts();
    if (status) {
        CUDA_TRY(cudaMemsetAsync(sc + 16, 0, 4, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (s->tc_phase == 1) {
            // the full step failed: start the step again from [cur]
            s->tc_phase = 0;
            s->tess_current = false;
        }
        if (status & rich::ST_NAN) return fail(RICH_ENAN, "non-finite state after the step");
        if (status & rich::ST_LEFT_BOX) return fail(RICH_ENEGATIVE, "a generating point left the box");
        return fail(RICH_ENEGATIVE, "non-positive mass or thermal energy after the step");
    }
    s->last_dt = dt;
    s->tess_current = false;
    if (s->time_centred() && s->tc_phase == 0) {
        // half step done: the next sweep is the full step on the half-step mesh
        s->tc_phase = 1;
        return RICH_OK;
    }
    s->tc_phase = 0;
    s->cur = 1 - s->cur;
    s->t += dt;
    if (info) {
        info->steps_done += 1;
        info->t = s->t;
        info->dt_last = dt;
    }
    return RICH_OK;
}

// One sweep of rich_step: while the device computes the gradients, fluxes
// and update, the host builds the mesh of the moved points (which it reads
// as soon as the point motion is done) unless the sweep ends the run at
// t_end; after the sweep that mesh is uploaded.  A failed sweep leaves the
// host mesh ahead of the device one: the next use tessellates again.
static int pipelined_sweep(rich_sim *s, double t_end, rich_step_info *info)
{
    int rc = launch_sweep(s, t_end, true);
    if (rc != RICH_OK) return rc;
    const double t0 = now_ms();
    CUDA_TRY(cudaEventSynchronize(s->ev_copied));
    if (info) info->copy_ms += now_ms() - t0;
    const double dt = s->hy()[s->n];
    // the half-step points always get a mesh; after a full step, the points
    // get one unless the step lands on t_end
    const bool build = (s->time_centred() && s->tc_phase == 0) || dt < t_end - s->t;
    int brc = RICH_OK;
    if (build) {
        s->tess_current = false;
        brc = build_mesh(s, info);
    }
    rc = rich_sync(s, info);
    if (rc != RICH_OK) return rc;
    // (a mesh that could not be built is reported by the next step's
    // tessellation of the same points, as without the early build)
    if (!build || brc != RICH_OK) return RICH_OK;
    return upload_mesh(s, info);
}

int rich_step(rich_sim *s, int32_t max_steps, double t_end, rich_step_info *info)
{
    rich::Range range("rich step");
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    if (s->pending) return fail(RICH_ESTATE, "a sweep is pending; call rich_sync first");
    if (info) std::memset(info, 0, sizeof(*info));
    for (int32_t k = 0; k < max_steps; k++) {
        if (!(s->t < t_end)) break;
        int rc;
        if (!s->tess_current && (rc = tessellate(s, info, true)) != RICH_OK) return rc;
        double before = s->t;
        if ((rc = pipelined_sweep(s, t_end, info)) != RICH_OK) return rc;
        if (s->tc_phase == 1) {
            // time-centred: the full step on the mesh of the half-step points
            // (meshed again here, to report its error, if the early build failed)
            if (!s->tess_current && (rc = tessellate(s, info, true)) != RICH_OK) return rc;
            if ((rc = pipelined_sweep(s, t_end, info)) != RICH_OK) return rc;
        }
        if (s->last_dt >= t_end - before) s->t = t_end;  // landed on t_end
        if (info) info->t = s->t;
    }
    if (info) {
        info->t = s->t;
        info->dt_last = s->last_dt;
    }
    return RICH_OK;
}

static int ensure_geometry(rich_sim *s)
{
    if (s->pending) return fail(RICH_ESTATE, "a sweep is pending; call rich_sync first");
    if (!s->tess_current) {
        int rc = tessellate(s, nullptr, true);
        if (rc) return rc;
    }
    for (int k = 0; k < rich::GEOMETRY_STAGES; k++) s->launch(k, nullptr, nullptr, false);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    // the cell geometry and primitives now describe the current points
    s->geometry_current = true;
    s->diag_pts = s->pts();
    return RICH_OK;
}

static void unpermute(const rich_sim *s, const double *internal, double *out)
{
    for (int32_t k = 0; k < s->n; k++) out[s->perm[k]] = internal[k];
}

static int fetch(rich_sim *s, const void *dev, std::vector<double> &h, size_t count)
{
    h.resize(count);
    CUDA_TRY(cudaMemcpyAsync(h.data(), dev, count * 8, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return RICH_OK;
}

// fetch count values stored in the handle's reconstruction precision
static int fetch_r(rich_sim *s, const void *dev, std::vector<double> &h, size_t count)
{
    if (s->rsize() == sizeof(double)) return fetch(s, dev, h, count);
    std::vector<float> f(count);
    CUDA_TRY(cudaMemcpyAsync(f.data(), dev, count * 4, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    h.assign(f.begin(), f.end());
    return RICH_OK;
}

int rich_get_state(rich_sim *s, int64_t n, double *x, double *y, double *rho, double *vx, double *vy, double *p,
                   double *area)
{
    if (!s || n != s->n) return fail(RICH_EINVAL, "bad handle or size");
    int rc = ensure_geometry(s);
    if (rc) return rc;
    std::vector<double> h;
    const size_t N = (size_t)s->n;
    const int q = s->pts();
    if (x) { if ((rc = fetch(s, s->x[q].p, h, N))) return rc; unpermute(s, h.data(), x); }
    if (y) { if ((rc = fetch(s, s->y[q].p, h, N))) return rc; unpermute(s, h.data(), y); }
    double *outs[4] = {rho, vx, vy, p};
    if (rho || vx || vy || p) {
        if ((rc = fetch_r(s, s->W.p, h, 4 * N))) return rc;
        std::vector<double> comp(N);
        for (int v = 0; v < 4; v++) {
            if (!outs[v]) continue;
            for (size_t k = 0; k < N; k++) comp[k] = h[4 * k + v];
            unpermute(s, comp.data(), outs[v]);
        }
    }
    if (area) { if ((rc = fetch(s, s->A.p, h, N))) return rc; unpermute(s, h.data(), area); }
    return RICH_OK;
}

int rich_get_conserved(rich_sim *s, int64_t n, double *x, double *y, double *m, double *px, double *py, double *E)
{
    if (!s || n != s->n) return fail(RICH_EINVAL, "bad handle or size");
    if (s->pending) return fail(RICH_ESTATE, "a sweep is pending; call rich_sync first");
    const size_t N = (size_t)s->n;
    const int q = s->pts();
    // points and state put in the caller's order on the device, then copied
    // straight into the caller's arrays with one wait
    double *outs[6] = {x, y, m, px, py, E};
    const double *src[6] = {s->x[q].as<double>(), s->y[q].as<double>(), s->U[q].as<double>(),
                            s->U[q].as<double>() + N, s->U[q].as<double>() + 2 * N, s->U[q].as<double>() + 3 * N};
    for (int f = 0; f < 6; f++)
        if (!outs[f]) src[f] = nullptr;
    CUDA_TRY(s->unperm.ensure(6 * N * sizeof(double)));
    double *st = s->unperm.as<double>();
    CUDA_TRY(rich::launch_unpermute(s->n, s->perm_dev.as<int32_t>(), src, st, s->stream));
    for (int f = 0; f < 6; f++)
        if (outs[f]) CUDA_TRY(cudaMemcpyAsync(outs[f], st + (size_t)f * N, N * 8, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return RICH_OK;
}

int rich_get_field(rich_sim *s, int32_t f, int64_t n, double *out)
{
    if (!s || n != s->n || !out) return fail(RICH_EINVAL, "bad arguments");
    if (s->pending) return fail(RICH_ESTATE, "a sweep is pending; call rich_sync first");
    const size_t N = (size_t)s->n;
    std::vector<double> h, h2;
    int rc;
    // the diagnostics refer to the points of the last sweep (or of the last
    // geometry pass on the current points)
    const int prev = s->geometry_current ? s->diag_pts : s->pts();
    // gather component c of an array-of-structures field with `stride` values per cell
    auto comp_of = [&](const DBuf &b, int stride, int c) {
        int r2 = fetch_r(s, b.p, h2, stride * N);
        if (r2) return r2;
        h.resize(N);
        for (size_t k = 0; k < N; k++) h[k] = h2[stride * k + c];
        return RICH_OK;
    };
    if (f == 0) rc = fetch(s, s->A.p, h, N);
    else if (f == 1 || f == 2) {
        if ((rc = comp_of(s->o, 2, f - 1))) return rc;
        std::vector<double> xs;
        rc = fetch(s, (f == 1 ? s->x[prev] : s->y[prev]).p, xs, N);
        for (size_t k = 0; k < N; k++) h[k] += xs[k];
    } else if (f >= 3 && f <= 6) rc = comp_of(s->W, 4, f - 3);
    else if (f == 7) rc = fetch_r(s, s->cs.p, h, N);
    else if (f >= 8 && f <= 23) rc = comp_of(f < 16 ? s->g : s->gl, 8, (f - 8) % 8);
    else if (f == 24 || f == 25) rc = comp_of(s->w, 2, f - 24);
    else if (f == 26) {
        std::vector<int32_t> ti(N);
        CUDA_TRY(cudaMemcpyAsync(ti.data(), s->tess.p, N * 4, cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        h.resize(N);
        for (size_t k = 0; k < N; k++) h[k] = ti[k];
        rc = RICH_OK;
    } else if (f >= 27 && f <= 30) rc = comp_of(s->alpha, 4, f - 27);
    else if (f == 31) {
        h.assign(N, s->last_dt);
        rc = RICH_OK;
    } else
        return fail(RICH_EINVAL, "unknown field");
    if (rc) return rc;
    unpermute(s, h.data(), out);
    return RICH_OK;
}

int rich_delaunay_host(int64_t n, const double *x, const double *y, int64_t cap, int32_t *tris, int64_t *ntri)
{
    if (n < 1 || !x || !y || !ntri) return fail(RICH_EINVAL, "bad arguments");
    rich::Delaunay dt;
    int rc = dt.build(x, y, (int32_t)n);
    if (rc == -2) return fail(RICH_EDUPLICATE, "two points coincide");
    if (rc) return fail(RICH_ETESS, "triangulation failed");
    *ntri = (int64_t)dt.tris.size();
    if (cap < *ntri || !tris) return fail(RICH_EINVAL, "capacity too small");
    for (size_t t = 0; t < dt.tris.size(); t++)
        for (int k = 0; k < 3; k++) tris[3 * t + k] = dt.tris[t].v[k];
    return RICH_OK;
}

int rich_rings_host(const rich_config *cfg, int64_t n, const double *x, const double *y, int64_t cap, int64_t *ptr,
                    double *nbx, double *nby, int64_t *nbsrc, int64_t *nslots)
{
    if (!valid_config(cfg) || n < 3 || !x || !y || !nslots || !ptr) return fail(RICH_EINVAL, "bad arguments");
    for (int64_t i = 0; i < n; i++)
        if (!point_inside(cfg, x[i], y[i])) return fail(RICH_EINVAL, "point outside the box");
    rich::MeshWork mw;
    rich::HostMesh m;
    rich::BoxConfig box{cfg->boundary, cfg->x0, cfg->x1, cfg->y0, cfg->y1};
    rich::ThreadPool pool((int)std::max(1u, std::thread::hardware_concurrency()));
    int rc = rich::build_host_mesh(box, (int32_t)n, x, y, mw, m, &pool);
    if (rc) return mesh_rc(rc);
    *nslots = (int64_t)m.slot_nb.size();
    for (int64_t i = 0; i <= n; i++) ptr[i] = m.cell_ptr[i];
    if (cap < *nslots || !nbx || !nby || !nbsrc) return fail(RICH_EINVAL, "capacity too small");
    for (size_t s = 0; s < m.slot_nb.size(); s++) {
        int32_t q = m.slot_nb[s];
        if (q < n) { nbx[s] = x[q]; nby[s] = y[q]; nbsrc[s] = q; }
        else { nbx[s] = m.gx[q - n]; nby[s] = m.gy[q - n]; nbsrc[s] = m.ghost_src[q - n]; }
    }
    return RICH_OK;
}

int rich_tess_phases(const rich_sim *s, double *ms)
{
    if (!s || !ms) return fail(RICH_EINVAL, "bad arguments");
    for (int k = 0; k < 4; k++) ms[k] = s->mw.phase_ms[k];
    return RICH_OK;
}

int rich_edge_list_check(const rich_config *cfg, int64_t n, const double *x, const double *y, int64_t *edges,
                         int64_t *mismatched)
{
    if (!valid_config(cfg) || n < 3 || n > INT32_MAX || !x || !y || !edges || !mismatched)
        return fail(RICH_EINVAL, "bad arguments");
    for (int64_t i = 0; i < n; i++)
        if (!point_inside(cfg, x[i], y[i])) return fail(RICH_EINVAL, "point outside the box");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(RICH_ENODEV, "no CUDA device");
    const rich::BoxConfig box{cfg->boundary, cfg->x0, cfg->x1, cfg->y0, cfg->y1};
    rich::ThreadPool pool((int)std::max(1u, std::thread::hardware_concurrency()));
    rich::MeshWork mw;  // host_edges: the host builds the reference lists too
    rich::HostMesh m;
    int rc = rich::build_host_mesh(box, (int32_t)n, x, y, mw, m, &pool);
    if (rc) return mesh_rc(rc);
    // the same points as a simulation builds them: rings and tri_off only
    rich::MeshWork mw2;
    mw2.host_edges = false;
    rich::HostMesh m2;
    rc = rich::build_host_mesh(box, (int32_t)n, x, y, mw2, m2, &pool);
    if (rc) return mesh_rc(rc);
    if (m2.slot_nb != m.slot_nb || m2.cell_ptr != m.cell_ptr) return fail(RICH_ETESS, "rings differ between builds");
    const size_t S = m.slot_nb.size(), E = (size_t)m.n_edges, T2 = (size_t)m2.n_tris;
    cudaStream_t st = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    DBuf cell_ptr, slot_nb, slot_tri, gsrc, gshift, eoff, slot_edge, el, er, eta, etb, bad, toff, dtri, dslot_tri, bad2;
    auto up = [&](DBuf &d, const std::vector<int32_t> &h) -> cudaError_t {
        cudaError_t e = d.ensure((h.size() + 1) * sizeof(int32_t));
        if (e == cudaSuccess && !h.empty())
            e = cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        return e;
    };
    std::vector<int32_t> dse(S), del(E), der(E), deta(E), detb(E), dt(3 * T2), dst(S);
    int32_t bad_h = 0, bad2_h = 0;
    cudaError_t e = up(cell_ptr, m.cell_ptr);
    if (e == cudaSuccess) e = up(slot_nb, m.slot_nb);
    if (e == cudaSuccess) e = up(slot_tri, m.slot_tri);
    if (e == cudaSuccess) e = up(gsrc, m.ghost_src);
    if (e == cudaSuccess) e = up(gshift, m.ghost_shift);
    if (e == cudaSuccess) e = up(eoff, m.edge_off);
    for (DBuf *b : {&slot_edge}) if (e == cudaSuccess) e = b->ensure((S + 1) * sizeof(int32_t));
    for (DBuf *b : {&el, &er, &eta, &etb}) if (e == cudaSuccess) e = b->ensure((E + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = bad.ensure(sizeof(int32_t));
    if (e == cudaSuccess) e = up(toff, m2.tri_off);
    if (e == cudaSuccess) e = dtri.ensure((3 * T2 + 3) * sizeof(int32_t));
    if (e == cudaSuccess) e = dslot_tri.ensure((S + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = bad2.ensure(sizeof(int32_t));
    if (e == cudaSuccess)
        e = rich::launch_build_tris((int32_t)n, (int32_t)S, cell_ptr.as<int32_t>(), slot_nb.as<int32_t>(),
                                    toff.as<int32_t>(), dtri.as<int32_t>(), dslot_tri.as<int32_t>(),
                                    bad2.as<int32_t>(), st);
    if (e == cudaSuccess)
        e = rich::launch_build_edges((int32_t)n, (int32_t)S, cell_ptr.as<int32_t>(), slot_nb.as<int32_t>(),
                                     slot_tri.as<int32_t>(), gsrc.as<int32_t>(), gshift.as<int32_t>(),
                                     eoff.as<int32_t>(), cfg->boundary == RICH_BC_PERIODIC ? 1 : 0, nullptr, nullptr,
                                     slot_edge.as<int32_t>(), el.as<int32_t>(), er.as<int32_t>(), eta.as<int32_t>(),
                                     etb.as<int32_t>(), bad.as<int32_t>(), st);
    auto down = [&](std::vector<int32_t> &h, DBuf &d) {
        if (e == cudaSuccess && !h.empty())
            e = cudaMemcpyAsync(h.data(), d.p, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    };
    down(dse, slot_edge);
    down(del, el);
    down(der, er);
    down(deta, eta);
    down(detb, etb);
    down(dt, dtri);
    down(dst, dslot_tri);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad2_h, bad2.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(RICH_ECUDA, cudaGetErrorString(e));
    int64_t bad_count = (bad_h ? 1 : 0) + (bad2_h ? 1 : 0);
    for (size_t k = 0; k < S; k++) bad_count += dse[k] != m.slot_edge[k];
    // the device's triangle of every slot: the host's, vertex for vertex
    // (the numbering differs: the host's is per tile)
    for (size_t k = 0; k < S; k++) {
        const int32_t a = dst[k], h = m.slot_tri[k];
        if (a < 0 || (size_t)a >= T2) {
            bad_count++;
            continue;
        }
        for (int c = 0; c < 3; c++) bad_count += dt[3 * (size_t)a + c] != m.tri[3 * (size_t)h + c];
    }
    for (size_t k = 0; k < E; k++)
        bad_count += (del[k] != m.edge_l[k]) + (der[k] != m.edge_r[k]) + (deta[k] != m.edge_ta[k]) +
                     (detb[k] != m.edge_tb[k]);
    *edges = (int64_t)E;
    *mismatched = bad_count;
    return RICH_OK;
}

int rich_mesh_update_check(const rich_config *cfg, int64_t n, int32_t steps, const double *xs, const double *ys,
                           int32_t threads, int32_t *mismatched, int64_t *updated, int64_t *rebuilt,
                           int64_t *reinserted)
{
    if (!valid_config(cfg) || n < 3 || n > INT32_MAX || steps < 1 || !xs || !ys || !mismatched || !updated ||
        !rebuilt || !reinserted || threads < 1)
        return fail(RICH_EINVAL, "bad arguments");
    for (int64_t i = 0; i < (int64_t)steps * n; i++)
        if (!point_inside(cfg, xs[i], ys[i])) return fail(RICH_EINVAL, "point outside the box");
    const rich::BoxConfig box{cfg->boundary, cfg->x0, cfg->x1, cfg->y0, cfg->y1};
    rich::ThreadPool pool(threads);
    rich::MeshWork kept;
    // the same sequence as a simulation builds it (no host lists: the rings
    // are read off incrementally and copied where unchanged)
    rich::MeshWork kept_dev;
    kept_dev.host_edges = false;
    *mismatched = 0;
    // a triangle's vertices (smallest id first in both builds)
    auto tri_of = [](const rich::HostMesh &m, int32_t t) {
        return std::array<int32_t, 3>{m.tri[3 * (size_t)t], m.tri[3 * (size_t)t + 1], m.tri[3 * (size_t)t + 2]};
    };
    for (int32_t k = 0; k < steps; k++) {
        const double *x = xs + (size_t)k * n, *y = ys + (size_t)k * n;
        rich::HostMesh a, b, c;
        rich::MeshWork fresh;
        int rc = rich::build_host_mesh(box, (int32_t)n, x, y, kept, a, &pool);
        if (rc) return mesh_rc(rc);
        rc = rich::build_host_mesh(box, (int32_t)n, x, y, fresh, b, &pool);
        if (rc) return mesh_rc(rc);
        rc = rich::build_host_mesh(box, (int32_t)n, x, y, kept_dev, c, &pool);
        if (rc) return mesh_rc(rc);
        if (!(c.g == b.g && c.gx == b.gx && c.gy == b.gy && c.ghost_src == b.ghost_src && c.cell_ptr == b.cell_ptr &&
              c.slot_nb == b.slot_nb && c.edge_off == b.edge_off && c.n_edges == b.n_edges &&
              c.cell_order == b.cell_order && (int64_t)c.tri_off.size() == n + 1 && c.tri_off[n] == c.n_tris))
            (*mismatched)++;
        bool same = a.g == b.g && a.gx == b.gx && a.gy == b.gy && a.ghost_src == b.ghost_src &&
                    a.cell_ptr == b.cell_ptr && a.slot_nb == b.slot_nb && a.slot_edge == b.slot_edge &&
                    a.edge_l == b.edge_l && a.edge_r == b.edge_r && a.cell_order == b.cell_order &&
                    a.edge_off == b.edge_off && a.n_edges == b.n_edges && (size_t)b.n_edges == b.edge_l.size();
        // the per-cell first edges (what the device builder numbers from)
        // agree with the host's list: cell i owns edges [edge_off[i], edge_off[i + 1])
        for (int64_t i = 0; same && i < n; i++)
            for (int32_t e = b.edge_off[i]; same && e < b.edge_off[i + 1]; e++) same = b.edge_l[e] == (int32_t)i;
        for (size_t s = 0; same && s < a.slot_tri.size(); s++) same = tri_of(a, a.slot_tri[s]) == tri_of(b, b.slot_tri[s]);
        for (size_t e = 0; same && e < a.edge_ta.size(); e++)
            same = tri_of(a, a.edge_ta[e]) == tri_of(b, b.edge_ta[e]) && tri_of(a, a.edge_tb[e]) == tri_of(b, b.edge_tb[e]);
        if (!same) (*mismatched)++;
    }
    *updated = kept.kinetic_tiles;
    *rebuilt = kept.fresh_tiles;
    *reinserted = kept.reinserted;
    return RICH_OK;
}

}  // extern "C"
