// Batched simulations (include/rich.h, rich_batch_*): many independent
// moving-mesh simulations of different sizes and parameters advanced
// together, one device sweep per step over all of them.
//
// Every step:
//   1. the generating points of all running simulations come back to the
//      host in one copy;
//   2. each simulation is tessellated on a host worker thread (a0), newly
//      admitted ones included;
//   3. the meshes are packed into one index space (cells of simulation k
//      follow those of k-1; ghosts, triangles, edges and ring slots likewise)
//      with a per-cell simulation id and a per-simulation parameter table;
//      when membership changed, the FP64 conserved state is regathered on
//      the device;
//   4. newly admitted simulations get their conserved variables from their
//      initial primitives and first areas (geometry stage in init mode);
//   5. one sweep (a1-a9) runs over all cells; each simulation keeps its own
//      time step, remaining time and status flags;
//   6. simulations that reached t_end or their step budget are copied out
//      and leave the batch; a failed step rolls back that simulation only.
// The arithmetic of every cell depends only on its own simulation, so a
// simulation's results do not depend on what else is in the batch.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "api_internal.h"
#include "mesh.h"
#include "sweep.cuh"
#include "threadpool.h"

namespace {

using rich::DBuf;
using rich::now_ms;
using rich::upload;
#define CUDA_TRY RICH_CUDA_TRY

int fail(int code, const std::string &msg) { return rich::set_error(code, msg); }

enum SimState { PENDING = 0, RUNNING = 1, DONE = 2, FAILED = 3, REMOVED = 4 };

struct BatchSim {
    int32_t id = -1;
    rich_config cfg{};
    int32_t n = 0;
    std::vector<int32_t> perm;  // internal (Hilbert) -> caller index
    std::vector<double> hx, hy;  // points, internal order
    std::vector<double> W0;      // initial primitives (4n, component-major) until admitted
    rich::MeshWork mw;           // (edge lists built on the device, packed)
    rich::HostMesh hm;
    int mesh_rc = 0;
    // the mesh of its current points was built during the last step's sweep
    // (mesh_rc is that build's result)
    bool prebuilt = false;
    double t = 0.0, t_end = 0.0, last_dt = 0.0;
    int64_t steps = 0, max_steps = 0;
    int state = PENDING;
    int err = RICH_OK;
    std::string err_msg;
    // offsets in the packed arrays of the current step
    int64_t cell_off = -1, ghost_off = 0, tri_off = 0, edge_off = 0, slot_off = 0;
    int64_t prev_cell_off = -1;  // offset in the previous packing (-1: not packed)
    // results of a finished simulation (caller order is applied on read)
    std::vector<double> fin;  // x, y, m, px, py, E (n each, internal order)
    double t_submit = 0.0, t_admit = 0.0, t_finish = 0.0;
    BatchSim() { mw.host_edges = false; }
};

// One way of launching the sweep: stage by stage, or as one persistent
// cooperative kernel (replayed from a recorded CUDA graph) with a block size.
struct LaunchShape {
    bool persistent;
    int block;
};

int mesh_code(int rc, std::string &msg)
{
    if (rc == -2) { msg = "two generating points coincide"; return RICH_EDUPLICATE; }
    if (rc == -4) { msg = "too few points for the ghost band"; return RICH_ETOOFEW; }
    msg = "tessellation failed";
    return RICH_ETESS;
}

}  // namespace

struct rich_batch {
    int32_t precision = RICH_FP64;
    int64_t max_cells = 0;
    int64_t cells_admitted = 0;  // cells of pending + running simulations
    std::vector<std::unique_ptr<BatchSim>> sims;
    std::vector<BatchSim *> packed;  // running simulations in packed order (last step)
    int64_t n_packed = 0;            // cells in the packed arrays
    // host workers: the batch's own, or a pool it shares with other
    // batches (the server's lanes)
    std::unique_ptr<rich::ThreadPool> own_pool;
    rich::ThreadPool *pool = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // early read of a staged sweep's moved points and time steps (copied on
    // their own stream once the point motion is done) into page-locked
    // memory: x, y of the packed cells, then dt per simulation
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_moved = nullptr, ev_copied = nullptr;
    rich::HBuf h_moved;
    bool diagnostics = false;
    int cur = 0;
    // device
    DBuf x[2], y[2], U[2], A, o, W, cs, g, gl, alpha, w, tess, rounding, p64, cell_ptr, cell_inst, initW, src;
    DBuf corder, psrc;
    DBuf gx, gy, gsrc, gxf, tri, ccx, ccy, slot_nb, slot_tri, slot_edge;
    DBuf edge_l, edge_r, edge_ta, edge_tb, eL, emlx, emly, emrx, emry, enx, eny, eqx, eqy, F, ePM;
    DBuf instp, dtmin, dtout, status, dsizes, gsync, eoff, toff, gshift, edgebad;
    // launch shape: autotuned over the first steps unless fixed by the caller
    int launch_mode = 0;  // 0 autotune, 1 staged, 2 persistent
    int fixed_block = 256;
    std::vector<LaunchShape> cands;
    std::vector<double> cand_ms;
    size_t cand_next = 0;
    bool tuned = false;
    LaunchShape chosen{false, 256};
    int last_grid = 0;
    bool graph_ok = true;
    std::string graph_note;
    // one recorded graph per ping-pong parity (the buffers swap roles each step)
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::vector<unsigned char> graph_sig[2];
    int64_t graph_records = 0;
    int64_t persistent_launches = 0, graph_launches = 0, staged_launches = 0;
    // persistent sweeps whose barrier wait gave up (each step redone staged);
    // inject_spin > 0 makes the next persistent sweep's barrier wait for one
    // block more than it launched and give up after that many polls
    int64_t barrier_timeouts = 0;
    int32_t inject_spin = 0;
    // host staging of the packed mesh
    std::vector<double> h_x, h_y, h_gx, h_gy, h_W0;
    std::vector<double> h_dlx, h_dly;  // the points downloaded at the start of a step
    std::vector<int32_t> h_gsrc, h_gxf, h_cell_ptr, h_slot_nb, h_cell_inst;
    std::vector<int32_t> h_corder;
    std::vector<int32_t> h_src, h_eoff, h_toff, h_gshift;
    std::vector<rich::InstParams> h_inst;
    std::vector<double> h_dt;
    std::vector<int32_t> h_status;
    int64_t nG = 0, nT = 0, nE = 0, nS = 0;

    explicit rich_batch(int threads) : own_pool(new rich::ThreadPool(threads)), pool(own_pool.get()) {}
    explicit rich_batch(rich::ThreadPool *shared) : pool(shared) {}
    ~rich_batch()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (int k = 0; k < 2; k++) {
            if (gexec[k]) cudaGraphExecDestroy(gexec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
        }
        if (copy_stream) cudaStreamSynchronize(copy_stream);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (ev_moved) cudaEventDestroy(ev_moved);
        if (ev_copied) cudaEventDestroy(ev_copied);
        if (copy_stream) cudaStreamDestroy(copy_stream);
        if (stream) cudaStreamDestroy(stream);
    }

    size_t rsize() const { return precision == RICH_FP32_SPLIT ? sizeof(float) : sizeof(double); }

    template <class R> rich::SweepParams<R> params() const
    {
        rich::SweepParams<R> p{};
        p.inst = instp.as<rich::InstParams>();
        p.cell_inst = cell_inst.as<int32_t>();
        p.n_inst = (int32_t)packed.size();
        p.diagnostics = diagnostics ? 1 : 0;
        p.motion = 1;
        p.n = (int32_t)n_packed;
        p.ng = (int32_t)nG;
        p.T = (int32_t)nT;
        p.E = (int32_t)nE;
        p.S = (int32_t)nS;
        p.x = x[cur].as<double>(); p.y = y[cur].as<double>();
        p.xn = x[1 - cur].as<double>(); p.yn = y[1 - cur].as<double>();
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
        p.U = U[cur].as<double>(); p.Un = U[1 - cur].as<double>();
        p.U0 = p.U; p.x0 = p.x; p.y0 = p.y;
        p.W = W.as<rich::Vec4<R>>(); p.o = o.as<rich::Vec2<R>>(); p.cs = cs.as<R>();
        p.g = g.as<rich::Vec4<R>>(); p.gl = gl.as<rich::Vec4<R>>(); p.alpha = alpha.as<rich::Vec4<R>>();
        p.w = w.as<rich::Vec2<R>>();
        p.rounding = rounding.as<uint8_t>(); p.p64 = p64.as<double>();
        p.tess = tess.as<int32_t>(); p.F = F.as<rich::Vec4<R>>(); p.psrc = psrc.as<rich::Vec4<R>>();
        p.dtmin_bits = dtmin.as<unsigned long long>();
        p.dt_out = dtout.as<double>();
        p.status = status.as<int32_t>();
        return p;
    }

    void launch(int k, const double *init_W, double *Un_override = nullptr) const
    {
        if (precision == RICH_FP32_SPLIT) {
            rich::SweepParams<float> p = params<float>();
            if (Un_override) p.Un = Un_override;
            rich::launch_stage<float>(k, p, init_W, stream);
        } else {
            rich::SweepParams<double> p = params<double>();
            if (Un_override) p.Un = Un_override;
            rich::launch_stage<double>(k, p, init_W, stream);
        }
    }

    BatchSim *find(int32_t id) const
    {
        if (id < 0 || (size_t)id >= sims.size()) return nullptr;
        BatchSim *s = sims[id].get();
        return s->state == REMOVED ? nullptr : s;
    }
};

namespace {

rich::InstParams inst_params(const BatchSim &s, bool init)
{
    rich::InstParams ip{};
    const rich_config &c = s.cfg;
    ip.gamma = c.gamma; ip.igm1 = 1.0 / (c.gamma - 1.0); ip.gamma_f = (float)ip.gamma; ip.igm1_f = (float)ip.igm1; ip.cfl = c.cfl; ip.chi = c.chi; ip.eta = c.eta; ip.theta = c.theta;
    ip.delta_v = c.delta_v; ip.delta_p = c.delta_p; ip.chi_f = (float)ip.chi; ip.theta_f = (float)ip.theta; ip.delta_v_f = (float)ip.delta_v;
    ip.x0 = c.x0; ip.x1 = c.x1; ip.y0 = c.y0; ip.y1 = c.y1;
    ip.remaining = s.t_end - s.t;
    ip.boundary = c.boundary; ip.motion = c.motion; ip.limiter = c.limiter;
    ip.init = init ? 1 : 0;
    return ip;
}

// Fill the staging arrays of simulation s (index k in packing order) at its offsets.
// One piece of the packing of simulation k into the batch's index space:
// part 0 its cells [i0, i1) (points, simulation id, ring offsets, order,
// first owned edges, state sources, initial primitives), part 1 its ring
// slots [i0, i1), part 2 its triangle corners [i0, i1), part 3 its ghosts.
struct PackTask {
    int32_t k, part;
    int64_t i0, i1;
};

void pack_part(rich_batch *b, BatchSim &s, const PackTask &t)
{
    const rich::HostMesh &m = s.hm;
    const int32_t n = s.n;
    const int64_t co = s.cell_off, go = s.ghost_off, to = s.tri_off, eo = s.edge_off, so = s.slot_off;
    const int64_t N = b->n_packed;
    auto pid = [&](int32_t q) -> int32_t {
        return q < n ? (int32_t)(co + q) : (int32_t)(N + go + (q - n));
    };
    const int64_t i0 = t.i0, i1 = t.i1;
    switch (t.part) {
    case 0:
        std::memcpy(&b->h_x[co + i0], s.hx.data() + i0, sizeof(double) * (i1 - i0));
        std::memcpy(&b->h_y[co + i0], s.hy.data() + i0, sizeof(double) * (i1 - i0));
        for (int64_t i = i0; i < i1; i++) {
            b->h_cell_inst[co + i] = t.k;
            b->h_cell_ptr[co + i] = (int32_t)(so + m.cell_ptr[i]);
            b->h_corder[co + i] = (int32_t)(co + m.cell_order[i]);
            b->h_eoff[co + i] = (int32_t)(eo + m.edge_off[i]);
            b->h_toff[co + i] = (int32_t)(to + m.tri_off[i]);
            // conserved state: continuing simulations gather from their previous slot
            b->h_src[co + i] = s.prev_cell_off >= 0 ? (int32_t)(s.prev_cell_off + i) : -1;
        }
        if (s.state == PENDING)
            for (int c = 0; c < 4; c++)
                for (int64_t i = i0; i < i1; i++) b->h_W0[(size_t)c * N + co + i] = s.W0[(size_t)c * n + i];
        break;
    case 1:
        for (int64_t q = i0; q < i1; q++) b->h_slot_nb[so + q] = pid(m.slot_nb[q]);
        break;
    default:
        for (int64_t q = i0; q < i1; q++) {
            b->h_gx[go + q] = m.gx[q];
            b->h_gy[go + q] = m.gy[q];
            b->h_gsrc[go + q] = (int32_t)(co + m.ghost_src[q]);
            b->h_gxf[go + q] = m.ghost_xf[q];
            b->h_gshift[go + q] = m.ghost_shift[q];
        }
        break;
    }
}

// The packing of every simulation as pieces of bounded size, so that one
// large simulation packs on all the pool's threads.
void pack_all(rich_batch *b, const std::vector<BatchSim *> &ok)
{
    constexpr int64_t kPiece = 1 << 16;
    std::vector<PackTask> tasks;
    auto split = [&](int32_t k, int32_t part, int64_t len, int64_t piece) {
        for (int64_t i = 0; i < len; i += piece) tasks.push_back(PackTask{k, part, i, std::min(len, i + piece)});
    };
    for (size_t k = 0; k < ok.size(); k++) {
        const BatchSim &s = *ok[k];
        split((int32_t)k, 0, s.n, kPiece);
        split((int32_t)k, 1, (int64_t)s.hm.slot_nb.size(), 4 * kPiece);
        split((int32_t)k, 3, s.hm.g, 4 * kPiece);
    }
    b->pool->parallel_for((int64_t)tasks.size(), [&](int64_t j) { pack_part(b, *ok[tasks[j].k], tasks[j]); });
}

int ensure_device(rich_batch *b)
{
    const size_t N = (size_t)b->n_packed, d = sizeof(double), r = b->rsize();
    const size_t G = (size_t)b->nG, T = (size_t)b->nT, E = (size_t)b->nE, K = b->packed.size();
    for (int k = 0; k < 2; k++) {
        CUDA_TRY(b->x[k].ensure(N * d + 8));
        CUDA_TRY(b->y[k].ensure(N * d + 8));
    }
    // U is grown by the caller: one of its two buffers may hold the live state
    CUDA_TRY(b->A.ensure(N * d + 8)); CUDA_TRY(b->o.ensure(2 * N * r + 16));
    CUDA_TRY(b->W.ensure(4 * N * r + 32)); CUDA_TRY(b->cs.ensure(N * r + 8));
    CUDA_TRY(b->g.ensure(8 * N * r + 64)); CUDA_TRY(b->gl.ensure(8 * N * r + 64));
    CUDA_TRY(b->alpha.ensure(4 * N * r + 32)); CUDA_TRY(b->w.ensure(2 * N * r + 16));
    CUDA_TRY(b->tess.ensure(N * 4 + 4)); CUDA_TRY(b->rounding.ensure(N + 8)); CUDA_TRY(b->p64.ensure(N * d + 8));
    CUDA_TRY(b->psrc.ensure(4 * N * r + 32));
    CUDA_TRY(b->ccx.ensure(T * d + 8)); CUDA_TRY(b->ccy.ensure(T * d + 8));
    for (DBuf *e : {&b->eL, &b->emlx, &b->emly, &b->emrx, &b->emry, &b->enx, &b->eny, &b->eqx, &b->eqy})
        CUDA_TRY(e->ensure(E * r + 8));
    CUDA_TRY(b->F.ensure(4 * E * sizeof(double) + 32));
    CUDA_TRY(b->ePM.ensure(4 * E * r + 32));
    CUDA_TRY(b->instp.ensure(K * sizeof(rich::InstParams) + 8));
    CUDA_TRY(b->dtmin.ensure(K * 8 + 8)); CUDA_TRY(b->dtout.ensure(K * 8 + 8)); CUDA_TRY(b->status.ensure(K * 4 + 8));
    CUDA_TRY(b->dsizes.ensure(sizeof(rich::DeviceSizes))); CUDA_TRY(b->gsync.ensure(sizeof(rich::GridSync)));
    (void)G;
    return RICH_OK;
}

void finish_copy_out(rich_batch *b, BatchSim &s, int which)
{
    // x, y and U of simulation s from packed buffer set `which` (synchronous)
    const size_t n = (size_t)s.n, N = (size_t)b->n_packed;
    s.fin.assign(6 * n, 0.0);
    cudaMemcpyAsync(&s.fin[0], b->x[which].as<double>() + s.cell_off, n * 8, cudaMemcpyDeviceToHost, b->stream);
    cudaMemcpyAsync(&s.fin[n], b->y[which].as<double>() + s.cell_off, n * 8, cudaMemcpyDeviceToHost, b->stream);
    for (int c = 0; c < 4; c++)
        cudaMemcpyAsync(&s.fin[(2 + c) * n], b->U[which].as<double>() + c * N + s.cell_off, n * 8,
                        cudaMemcpyDeviceToHost, b->stream);
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class R> int persistent_grid(int block)
{
    return rich::persistent_blocks_per_sm<R>(block) * sm_count();
}

// Enqueue the whole sweep as one persistent cooperative launch, from a
// recorded CUDA graph when possible.  The graph holds the barrier and status
// resets and the launch; it is recorded again only when a device buffer moved
// (the mesh sizes come from device memory).
template <class R> int run_persistent(rich_batch *b, int block)
{
    const int grid = persistent_grid<R>(block);
    if (grid <= 0) return fail(RICH_ECUDA, "persistent sweep cannot be resident");
    b->last_grid = grid;
    rich::SweepParams<R> p = b->params<R>();
    p.n = p.ng = p.T = p.E = p.S = p.n_inst = 0;  // read from device memory
    rich::DeviceSizes sz{};
    sz.n = (int32_t)b->n_packed;
    sz.ng = (int32_t)b->nG;
    sz.T = (int32_t)b->nT;
    sz.E = (int32_t)b->nE;
    sz.n_inst = (int32_t)b->packed.size();
    CUDA_TRY(cudaMemcpyAsync(b->dsizes.p, &sz, sizeof(sz), cudaMemcpyHostToDevice, b->stream));
    auto *gs = b->gsync.as<rich::GridSync>();
    auto *ds = b->dsizes.as<rich::DeviceSizes>();
    if (b->inject_spin > 0) {
        // a barrier that cannot complete: every wait runs out after
        // inject_spin polls and the sweep stops (launched directly, not from
        // the recorded graph)
        rich::GridSync g{};
        g.spin_limit = b->inject_spin;
        g.extra = 1;
        b->inject_spin = 0;
        CUDA_TRY(cudaMemcpyAsync(gs, &g, sizeof(g), cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(cudaMemsetAsync(b->status.p, 0, b->status.cap, b->stream));
        CUDA_TRY(rich::launch_persistent<R>(p, ds, gs, block, grid, b->stream));
        b->persistent_launches++;
        return RICH_OK;
    }
    if (b->graph_ok) {
        std::vector<unsigned char> sig(sizeof(p) + 3 * sizeof(int));
        std::memcpy(sig.data(), &p, sizeof(p));
        int extra[3] = {block, grid, (int)sizeof(R)};
        std::memcpy(sig.data() + sizeof(p), extra, sizeof(extra));
        const int par = b->cur;
        cudaGraph_t &graph = b->graph[par];
        cudaGraphExec_t &gexec = b->gexec[par];
        if (!gexec || sig != b->graph_sig[par]) {
            if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
            if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
            bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                cudaMemsetAsync(gs, 0, sizeof(rich::GridSync), b->stream);
                cudaMemsetAsync(b->status.p, 0, b->status.cap, b->stream);
                cudaError_t le = rich::launch_persistent<R>(p, ds, gs, block, grid, b->stream);
                cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
                ok = le == cudaSuccess && ce == cudaSuccess && graph &&
                     cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
                if (!ok) b->graph_note = std::string("graph capture failed: ") + cudaGetErrorString(le != cudaSuccess ? le : ce);
            }
            cudaGetLastError();
            if (!ok) {
                b->graph_ok = false;
                if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
                if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
            } else {
                b->graph_sig[par] = sig;
                b->graph_records++;
            }
        }
        if (b->graph_ok) {
            CUDA_TRY(cudaGraphLaunch(gexec, b->stream));
            b->graph_launches++;
            b->persistent_launches++;
            return RICH_OK;
        }
    }
    CUDA_TRY(cudaMemsetAsync(gs, 0, sizeof(rich::GridSync), b->stream));
    CUDA_TRY(cudaMemsetAsync(b->status.p, 0, b->status.cap, b->stream));
    CUDA_TRY(rich::launch_persistent<R>(p, ds, gs, block, grid, b->stream));
    b->persistent_launches++;
    return RICH_OK;
}

// The sweep stage by stage; with read_moved the moved points and each
// simulation's dt are copied into h_moved as soon as the point motion is
// done (ev_copied marks their arrival) while the other stages run.
int run_staged(rich_batch *b, bool read_moved = false)
{
    CUDA_TRY(cudaMemsetAsync(b->status.p, 0, b->status.cap, b->stream));
    for (int k = 0; k < rich::NUM_STAGES; k++) {
        b->launch(k, nullptr);
        if (read_moved && k == rich::K_ADVANCE) {
            const size_t N = (size_t)b->n_packed, I = b->packed.size();
            double *h = b->h_moved.as<double>();
            CUDA_TRY(cudaEventRecord(b->ev_moved, b->stream));
            CUDA_TRY(cudaStreamWaitEvent(b->copy_stream, b->ev_moved, 0));
            CUDA_TRY(cudaMemcpyAsync(h, b->x[1 - b->cur].p, N * 8, cudaMemcpyDeviceToHost, b->copy_stream));
            CUDA_TRY(cudaMemcpyAsync(h + N, b->y[1 - b->cur].p, N * 8, cudaMemcpyDeviceToHost, b->copy_stream));
            CUDA_TRY(cudaMemcpyAsync(h + 2 * N, b->dtout.p, I * 8, cudaMemcpyDeviceToHost, b->copy_stream));
            CUDA_TRY(cudaEventRecord(b->ev_copied, b->copy_stream));
        }
    }
    CUDA_TRY(cudaGetLastError());
    b->staged_launches++;
    return RICH_OK;
}

// the launch shape of this step: the next untried candidate while tuning
LaunchShape pick_shape(rich_batch *b)
{
    if (b->launch_mode == 1) return LaunchShape{false, 256};
    if (b->launch_mode == 2) return LaunchShape{true, b->fixed_block};
    if (b->tuned) return b->chosen;
    if (b->cands.empty()) {
        // every candidate twice; the faster of its two timings counts
        for (int rep = 0; rep < 2; rep++) {
            b->cands.push_back(LaunchShape{false, 256});
            for (int bs : {128, 256, 512}) b->cands.push_back(LaunchShape{true, bs});
        }
        b->cand_ms.assign(b->cands.size(), 0.0);
    }
    return b->cands[b->cand_next];
}

void record_timing(rich_batch *b, const LaunchShape &s, double ms)
{
    if (b->launch_mode != 0 || b->tuned) return;
    b->cand_ms[b->cand_next++] = ms;
    if (b->cand_next < b->cands.size()) return;
    const size_t half = b->cands.size() / 2;
    double best = 1e300;
    for (size_t k = 0; k < half; k++) {
        double t = std::min(b->cand_ms[k], b->cand_ms[k + half]);
        if (t < best) { best = t; b->chosen = b->cands[k]; }
    }
    b->tuned = true;
    (void)s;
}

}  // namespace

namespace rich {
// A batch whose host work runs on `shared` (owned by the caller, who keeps
// it alive longer than the batch); host_threads <= 0 and shared == nullptr:
// its own pool of one thread per hardware thread.
int batch_create(int32_t precision, int64_t max_cells, int32_t host_threads, ThreadPool *shared, rich_batch **out)
{
    if (!out) return fail(RICH_EINVAL, "out is NULL");
    *out = nullptr;
    if ((precision != RICH_FP64 && precision != RICH_FP32_SPLIT) || max_cells < 3 || max_cells > ((int64_t)1 << 30))
        return fail(RICH_EINVAL, "bad precision or cell budget");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(RICH_ENODEV, "no CUDA device");
    int threads = host_threads > 0 ? host_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    rich_batch *b = shared ? new (std::nothrow) rich_batch(shared) : new (std::nothrow) rich_batch(threads);
    if (!b) return fail(RICH_ENOMEM, "host allocation");
    b->precision = precision;
    b->max_cells = max_cells;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_moved, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_copied, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return fail(RICH_ECUDA, "stream or event creation failed");
    }
    *out = b;
    return RICH_OK;
}
}  // namespace rich

extern "C" {


int rich_batch_create(int32_t precision, int64_t max_cells, int32_t host_threads, rich_batch **out)
{
    return rich::batch_create(precision, max_cells, host_threads, nullptr, out);
}

void rich_batch_destroy(rich_batch *b) { delete b; }

int rich_batch_add(rich_batch *b, const rich_config *cfg, int64_t n, const double *x, const double *y,
                   const double *rho, const double *vx, const double *vy, const double *p, double t_end,
                   int64_t max_steps, int32_t *id)
{
    if (!b || !id) return fail(RICH_EINVAL, "NULL argument");
    if (cfg && cfg->scheme != RICH_SCHEME_EXTRAPOLATED)
        return fail(RICH_EINVAL, "batches run the extrapolated-fluxes scheme only");
    if (!rich::valid_config(cfg) || cfg->precision != b->precision)
        return fail(RICH_EINVAL, "invalid configuration or precision differs from the batch");
    if (n < 3 || n > ((int64_t)1 << 30) || !x || !y || !rho || !vx || !vy || !p) return fail(RICH_EINVAL, "bad arrays");
    if (!(t_end > 0.0) || max_steps < 1) return fail(RICH_EINVAL, "t_end must be > 0 and max_steps >= 1");
    for (int64_t i = 0; i < n; i++) {
        if (!std::isfinite(x[i]) || !std::isfinite(y[i]) || !rich::point_inside(cfg, x[i], y[i]))
            return fail(RICH_EINVAL, "point " + std::to_string(i) + " outside the box");
        if (!(rho[i] > 0) || !(p[i] > 0) || !std::isfinite(rho[i]) || !std::isfinite(p[i]) || !std::isfinite(vx[i]) ||
            !std::isfinite(vy[i]))
            return fail(RICH_EINVAL, "bad primitive values at point " + std::to_string(i));
    }
    if (b->cells_admitted + n > b->max_cells) return fail(RICH_ENOMEM, "the batch's cell budget is full");
    auto s = std::make_unique<BatchSim>();
    s->cfg = *cfg;
    s->n = (int32_t)n;
    rich::hilbert_order(s->n, x, y, s->perm);
    s->hx.resize(n);
    s->hy.resize(n);
    s->W0.resize(4 * (size_t)n);
    for (int32_t k = 0; k < s->n; k++) {
        int32_t u = s->perm[k];
        s->hx[k] = x[u];
        s->hy[k] = y[u];
        s->W0[k] = rho[u];
        s->W0[n + k] = vx[u];
        s->W0[2 * n + k] = vy[u];
        s->W0[3 * n + k] = p[u];
    }
    s->t_end = t_end;
    s->max_steps = max_steps;
    s->t_submit = now_ms();
    s->id = (int32_t)b->sims.size();  // ids index the simulation list
    *id = s->id;
    b->cells_admitted += n;
    b->sims.push_back(std::move(s));
    return RICH_OK;
}

// Simulations of at least this many cells are tessellated in tiles over the
// whole pool (four or more tiles of 16,384 points).
constexpr int32_t kTiledMember = 65536;

namespace {
// a0 for the given simulations on the pool, from the points in their hx, hy
// (results in mesh_rc): largest first, since the pool hands out tasks in
// order, so the longest tessellations start first and the makespan stays
// near the largest one (or the mean load per thread).  A simulation large
// enough for several tiles is tessellated with the whole pool (its tiles in
// parallel, as a single simulation is), one after another; the others in
// parallel, one per pool thread.  The mesh the sweep sees does not depend
// on the tiling.
void tessellate_members(rich_batch *b, const std::vector<BatchSim *> &sims)
{
    rich::Range range("rich batch tessellate (a0)");
    std::vector<BatchSim *> by_size(sims);
    std::stable_sort(by_size.begin(), by_size.end(), [](const BatchSim *a, const BatchSim *c) { return a->n > c->n; });
    size_t n_large = 0;
    while (n_large < by_size.size() && by_size[n_large]->n >= kTiledMember) n_large++;
    for (size_t k = 0; k < n_large; k++) {
        BatchSim *s = by_size[k];
        rich::BoxConfig box{s->cfg.boundary, s->cfg.x0, s->cfg.x1, s->cfg.y0, s->cfg.y1};
        s->mesh_rc = rich::build_host_mesh(box, s->n, s->hx.data(), s->hy.data(), s->mw, s->hm, b->pool);
    }
    b->pool->parallel_for((int64_t)(by_size.size() - n_large), [&](int64_t k) {
        BatchSim *s = by_size[n_large + k];
        rich::BoxConfig box{s->cfg.boundary, s->cfg.x0, s->cfg.x1, s->cfg.y0, s->cfg.y1};
        s->mesh_rc = rich::build_host_mesh(box, s->n, s->hx.data(), s->hy.data(), s->mw, s->hm);
    });
}

}  // namespace

int rich_batch_step(rich_batch *b, rich_step_info *info)
{
    rich::Range range("rich batch step");
    if (!b) return fail(RICH_EINVAL, "NULL handle");
    if (info) std::memset(info, 0, sizeof(*info));
    const double t0 = now_ms();
    // 1. points of the running simulations back to the host (those whose
    //    mesh was built during the last sweep have them already)
    bool need_points = false;
    for (BatchSim *s : b->packed) need_points |= s->state == RUNNING && !s->prebuilt;
    if (b->n_packed > 0 && need_points) {
        // (kept between steps: a fresh vector would zero 16 B per cell first)
        std::vector<double> &hx = b->h_dlx, &hy = b->h_dly;
        if (hx.size() < (size_t)b->n_packed) {
            hx.resize(b->n_packed);
            hy.resize(b->n_packed);
        }
        CUDA_TRY(cudaMemcpyAsync(hx.data(), b->x[b->cur].p, b->n_packed * 8, cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaMemcpyAsync(hy.data(), b->y[b->cur].p, b->n_packed * 8, cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        // to each simulation's own arrays, on the pool
        b->pool->parallel_for((int64_t)b->packed.size(), [&](int64_t k) {
            BatchSim *s = b->packed[k];
            if (s->state != RUNNING || s->prebuilt) return;
            std::memcpy(s->hx.data(), &hx[s->cell_off], sizeof(double) * s->n);
            std::memcpy(s->hy.data(), &hy[s->cell_off], sizeof(double) * s->n);
        });
    }
    // the simulations of this step: running ones in their previous order, then new ones
    std::vector<BatchSim *> list;
    for (BatchSim *s : b->packed)
        if (s->state == RUNNING) list.push_back(s);
    for (auto &s : b->sims)
        if (s->state == PENDING) list.push_back(s.get());
    for (BatchSim *s : list) s->prev_cell_off = s->state == RUNNING ? s->cell_off : -1;
    if (list.empty()) {
        b->packed.clear();
        b->n_packed = 0;
        return RICH_OK;
    }
    // 2. tessellations in parallel (of the simulations without a mesh
    //    built during the last sweep)
    const double t1 = now_ms();
    {
        std::vector<BatchSim *> todo;
        for (BatchSim *s : list)
            if (!s->prebuilt) todo.push_back(s);
        tessellate_members(b, todo);
        for (BatchSim *s : list) s->prebuilt = false;
    }
    const double t2 = now_ms();
    std::vector<BatchSim *> ok;
    for (BatchSim *s : list) {
        if (s->mesh_rc == 0) {
            ok.push_back(s);
            continue;
        }
        s->err = mesh_code(s->mesh_rc, s->err_msg);
        if (s->state == RUNNING) {
            // keep its last good state for the caller
            s->cell_off = s->prev_cell_off;
            finish_copy_out(b, *s, b->cur);
        }
        s->state = FAILED;
        s->t_finish = now_ms();
        b->cells_admitted -= s->n;
    }
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    // 3. packing offsets
    const int64_t n_old = b->n_packed;
    bool same_layout = ok.size() == b->packed.size();
    int64_t co = 0, go = 0, to = 0, eo = 0, so = 0;
    for (size_t k = 0; k < ok.size(); k++) {
        BatchSim *s = ok[k];
        if (same_layout && (b->packed[k] != s || s->prev_cell_off != co)) same_layout = false;
        s->cell_off = co; s->ghost_off = go; s->tri_off = to; s->edge_off = eo; s->slot_off = so;
        co += s->n;
        go += s->hm.g;
        to += (int64_t)s->hm.n_tris;
        eo += (int64_t)s->hm.n_edges;
        so += (int64_t)s->hm.slot_nb.size();
    }
    if (co + go > ((int64_t)1 << 31) - 1 || 3 * to > ((int64_t)1 << 31) - 1 || 2 * eo > ((int64_t)1 << 31) - 1)
        return fail(RICH_ENOMEM, "batch exceeds 32-bit indexing");
    b->packed = ok;
    b->n_packed = co;
    b->nG = go;
    b->nT = to;
    b->nE = eo;
    b->nS = so;
    const size_t N = (size_t)co;
    bool any_pending = false;
    for (BatchSim *s : ok) any_pending |= s->state == PENDING;
    b->h_x.resize(N); b->h_y.resize(N); b->h_cell_inst.resize(N); b->h_src.resize(N);
    b->h_gx.resize(go); b->h_gy.resize(go); b->h_gsrc.resize(go); b->h_gxf.resize(go);
    b->h_cell_ptr.resize(N + 1); b->h_corder.resize(N);
    b->h_slot_nb.resize(so);
    b->h_eoff.resize(N + 1); b->h_toff.resize(N + 1); b->h_gshift.resize(go);
    if (any_pending) b->h_W0.assign(4 * N, 0.0);
    pack_all(b, ok);
    b->h_cell_ptr[N] = (int32_t)so;
    b->h_eoff[N] = (int32_t)eo;
    b->h_toff[N] = (int32_t)to;
    b->h_inst.resize(ok.size());
    for (size_t k = 0; k < ok.size(); k++) b->h_inst[k] = inst_params(*ok[k], ok[k]->state == PENDING);
    // 4. device buffers and uploads
    int rc = ensure_device(b);
    if (rc) return rc;
    const int nxt = 1 - b->cur;
    if (!same_layout && n_old > 0) {
        // regather the conserved state of continuing simulations into the other
        // buffer (grown first: U[cur] holds the live state and is not touched)
        CUDA_TRY(b->U[nxt].ensure(4 * N * sizeof(double) + 8));
        CUDA_TRY(upload(b->src, b->h_src, b->stream));
        rich::launch_repack(b->src.as<int32_t>(), (int32_t)N, (int32_t)n_old, b->U[b->cur].as<double>(),
                            b->U[nxt].as<double>(), b->stream);
        CUDA_TRY(cudaGetLastError());
        b->cur = nxt;
    } else if (n_old == 0) {
        CUDA_TRY(b->U[b->cur].ensure(4 * N * sizeof(double) + 8));  // nothing live yet
    }
    // the buffer the sweep writes; its old contents are dead
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    CUDA_TRY(b->U[1 - b->cur].ensure(4 * N * sizeof(double) + 8));
    CUDA_TRY(upload(b->x[b->cur], b->h_x, b->stream));
    CUDA_TRY(upload(b->y[b->cur], b->h_y, b->stream));
    CUDA_TRY(upload(b->cell_inst, b->h_cell_inst, b->stream));
    CUDA_TRY(upload(b->gx, b->h_gx, b->stream));
    CUDA_TRY(upload(b->gy, b->h_gy, b->stream));
    CUDA_TRY(upload(b->gsrc, b->h_gsrc, b->stream));
    CUDA_TRY(upload(b->gxf, b->h_gxf, b->stream));
    CUDA_TRY(upload(b->cell_ptr, b->h_cell_ptr, b->stream));
    CUDA_TRY(upload(b->corder, b->h_corder, b->stream));
    CUDA_TRY(upload(b->slot_nb, b->h_slot_nb, b->stream));
    CUDA_TRY(upload(b->toff, b->h_toff, b->stream));
    CUDA_TRY(upload(b->eoff, b->h_eoff, b->stream));
    CUDA_TRY(upload(b->gshift, b->h_gshift, b->stream));
    CUDA_TRY(upload(b->instp, b->h_inst, b->stream));
    // the packed triangle and edge lists, built on the device from the rings
    // (each cell's box type from its simulation's parameters); checked before
    // any kernel reads them
    {
        CUDA_TRY(b->tri.ensure((size_t)to * 12 + 12));
        CUDA_TRY(b->slot_tri.ensure((size_t)so * 4 + 4));
        CUDA_TRY(b->slot_edge.ensure((size_t)so * 4 + 4));
        for (DBuf *e : {&b->edge_l, &b->edge_r, &b->edge_ta, &b->edge_tb}) CUDA_TRY(e->ensure((size_t)eo * 4 + 4));
        CUDA_TRY(b->edgebad.ensure(8));
        int32_t *bad = b->edgebad.as<int32_t>();
        CUDA_TRY(rich::launch_build_tris((int32_t)N, (int32_t)so, b->cell_ptr.as<int32_t>(), b->slot_nb.as<int32_t>(),
                                         b->toff.as<int32_t>(), b->tri.as<int32_t>(), b->slot_tri.as<int32_t>(),
                                         bad + 1, b->stream));
        CUDA_TRY(rich::launch_build_edges((int32_t)N, (int32_t)so, b->cell_ptr.as<int32_t>(), b->slot_nb.as<int32_t>(),
                                          b->slot_tri.as<int32_t>(), b->gsrc.as<int32_t>(), b->gshift.as<int32_t>(),
                                          b->eoff.as<int32_t>(), 0, b->instp.as<rich::InstParams>(),
                                          b->cell_inst.as<int32_t>(), b->slot_edge.as<int32_t>(),
                                          b->edge_l.as<int32_t>(), b->edge_r.as<int32_t>(), b->edge_ta.as<int32_t>(),
                                          b->edge_tb.as<int32_t>(), bad, b->stream));
        int32_t bad_h[2] = {0, 0};
        CUDA_TRY(cudaMemcpyAsync(bad_h, bad, 8, cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        if (bad_h[1]) return fail(RICH_ETESS, "a triangle of a ring is missing from its owner's ring");
        if (bad_h[0]) return fail(RICH_ETESS, "an edge of a ring has no partner in the other cell's ring");
    }
    CUDA_TRY(cudaMemsetAsync(b->status.p, 0, ok.size() * 4, b->stream));
    if (any_pending) CUDA_TRY(upload(b->initW, b->h_W0, b->stream));
    // 5. admission: conserved variables of new simulations from their first geometry
    if (any_pending) {
        b->launch(rich::K_CIRCUMCENTRE, nullptr);
        b->launch(rich::K_GEOMETRY, b->initW.as<double>(), b->U[b->cur].as<double>());
        for (BatchSim *s : ok)
            if (s->state == PENDING) {
                s->state = RUNNING;
                s->t_admit = now_ms();
                s->W0.clear();
                s->W0.shrink_to_fit();
            }
        for (size_t k = 0; k < ok.size(); k++) b->h_inst[k].init = 0;
        CUDA_TRY(upload(b->instp, b->h_inst, b->stream));
    }
    const double t3 = now_ms();
    // 6. the sweep over every cell of every simulation; staged, its moved
    //    points are read back once the point motion is done, and the host
    //    tessellates them for the next step while the device finishes
    const LaunchShape shape = pick_shape(b);
    if (!shape.persistent) CUDA_TRY(b->h_moved.ensure((2 * N + ok.size() + 1) * sizeof(double)));
    CUDA_TRY(cudaEventRecord(b->ev0, b->stream));
    if (shape.persistent) {
        rc = b->precision == RICH_FP32_SPLIT ? run_persistent<float>(b, shape.block) : run_persistent<double>(b, shape.block);
    } else {
        rc = run_staged(b, true);
    }
    if (rc) return rc;
    CUDA_TRY(cudaEventRecord(b->ev1, b->stream));
    double t_pre = 0.0;
    if (!shape.persistent) {
        CUDA_TRY(cudaEventSynchronize(b->ev_copied));
        const double tp = now_ms();
        const double *h = b->h_moved.as<double>();
        // the simulations that go on after this step (the bookkeeping below
        // takes the same decision), unless the step fails
        std::vector<BatchSim *> next;
        for (size_t k = 0; k < ok.size(); k++) {
            BatchSim *s = ok[k];
            const double dt = h[2 * N + k], rem = s->t_end - s->t;
            const double tn = dt >= rem ? s->t_end : s->t + dt;
            if (tn >= s->t_end || s->steps + 1 >= s->max_steps) continue;
            next.push_back(s);
        }
        b->pool->parallel_for((int64_t)next.size(), [&](int64_t k) {
            BatchSim *s = next[k];
            std::memcpy(s->hx.data(), h + s->cell_off, sizeof(double) * s->n);
            std::memcpy(s->hy.data(), h + N + s->cell_off, sizeof(double) * s->n);
        });
        tessellate_members(b, next);
        for (BatchSim *s : next) s->prebuilt = true;
        t_pre = now_ms() - tp;
    }
    if (shape.persistent) {
        int32_t timeout = 0;
        CUDA_TRY(cudaMemcpyAsync(&timeout, (char *)b->gsync.p + offsetof(rich::GridSync, timeout), 4,
                                 cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        if (timeout) {
            // a barrier wait gave up: the inputs of the step are untouched, so
            // redo it stage by stage and keep the staged launch from now on
            b->launch_mode = 1;
            b->barrier_timeouts++;
            b->graph_note = "persistent sweep barrier timed out; staged launches used";
            CUDA_TRY(cudaEventRecord(b->ev0, b->stream));
            if ((rc = run_staged(b))) return rc;
            CUDA_TRY(cudaEventRecord(b->ev1, b->stream));
        }
    }
    b->h_dt.resize(ok.size());
    b->h_status.resize(ok.size());
    CUDA_TRY(cudaMemcpyAsync(b->h_dt.data(), b->dtout.p, ok.size() * 8, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaMemcpyAsync(b->h_status.data(), b->status.p, ok.size() * 4, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    record_timing(b, shape, ms);
    // 7. per-simulation bookkeeping; a failed step keeps that simulation's old state
    const int nxt2 = 1 - b->cur;
    const double tnow = now_ms();
    for (size_t k = 0; k < ok.size(); k++) {
        BatchSim *s = ok[k];
        if (b->h_status[k]) {
            s->prebuilt = false;
            s->err = (b->h_status[k] & rich::ST_NAN) ? RICH_ENAN : RICH_ENEGATIVE;
            s->err_msg = "step rejected (non-finite, non-positive mass or thermal energy, or a point left the box)";
            finish_copy_out(b, *s, b->cur);
            s->state = FAILED;
            s->t_finish = tnow;
            b->cells_admitted -= s->n;
            continue;
        }
        const double rem = s->t_end - s->t;
        s->last_dt = b->h_dt[k];
        s->t = s->last_dt >= rem ? s->t_end : s->t + s->last_dt;
        s->steps++;
        if (s->t >= s->t_end || s->steps >= s->max_steps) {
            finish_copy_out(b, *s, nxt2);
            s->state = DONE;
            s->t_finish = tnow;
            b->cells_admitted -= s->n;
        }
    }
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->cur = nxt2;
    if (info) {
        info->steps_done = (int64_t)ok.size();
        info->sweep_ms = ms;
        info->tess_ms = (t2 - t1) + t_pre;
        info->copy_ms = (t1 - t0) + (t3 - t2) + (now_ms() - tnow);
        info->n_ghost = b->nG;
        info->n_tri = b->nT;
        info->n_edges = b->nE;
        info->n_slots = b->nS;
        info->t = 0.0;
        info->dt_last = 0.0;
    }
    return RICH_OK;
}

int rich_batch_query(rich_batch *b, int32_t id, int32_t *state, int32_t *error, double *t, int64_t *steps,
                     double *latency_ms)
{
    if (!b) return fail(RICH_EINVAL, "NULL handle");
    BatchSim *s = b->find(id);
    if (!s) return fail(RICH_EINVAL, "unknown simulation id");
    if (state) *state = s->state;
    if (error) *error = s->err;
    if (t) *t = s->t;
    if (steps) *steps = s->steps;
    if (latency_ms)
        *latency_ms = (s->state == DONE || s->state == FAILED) ? s->t_finish - s->t_submit : -1.0;
    return RICH_OK;
}

int rich_batch_get_conserved(rich_batch *b, int32_t id, int64_t n, double *x, double *y, double *m, double *px,
                             double *py, double *E)
{
    if (!b) return fail(RICH_EINVAL, "NULL handle");
    BatchSim *s = b->find(id);
    if (!s || n != s->n) return fail(RICH_EINVAL, "unknown simulation id or wrong size");
    std::vector<double> buf;
    const double *src = nullptr;
    if (s->state == DONE || s->state == FAILED) {
        if (s->fin.empty()) return fail(RICH_ESTATE, "no state recorded");
        src = s->fin.data();
    } else if (s->state == RUNNING) {
        const size_t nn = (size_t)s->n, N = (size_t)b->n_packed;
        buf.resize(6 * nn);
        CUDA_TRY(cudaMemcpyAsync(&buf[0], b->x[b->cur].as<double>() + s->cell_off, nn * 8, cudaMemcpyDeviceToHost,
                                 b->stream));
        CUDA_TRY(cudaMemcpyAsync(&buf[nn], b->y[b->cur].as<double>() + s->cell_off, nn * 8, cudaMemcpyDeviceToHost,
                                 b->stream));
        for (int c = 0; c < 4; c++)
            CUDA_TRY(cudaMemcpyAsync(&buf[(2 + c) * nn], b->U[b->cur].as<double>() + c * N + s->cell_off, nn * 8,
                                     cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        src = buf.data();
    } else {
        return fail(RICH_ESTATE, "simulation not admitted yet");
    }
    double *outs[6] = {x, y, m, px, py, E};
    for (int f = 0; f < 6; f++) {
        if (!outs[f]) continue;
        for (int32_t k = 0; k < s->n; k++) outs[f][s->perm[k]] = src[(size_t)f * s->n + k];
    }
    return RICH_OK;
}

int rich_batch_remove(rich_batch *b, int32_t id)
{
    if (!b) return fail(RICH_EINVAL, "NULL handle");
    BatchSim *s = b->find(id);
    if (!s) return fail(RICH_EINVAL, "unknown simulation id");
    if (s->state == PENDING || s->state == RUNNING) b->cells_admitted -= s->n;
    s->state = REMOVED;
    s->fin.clear();
    s->fin.shrink_to_fit();
    s->hm = rich::HostMesh();
    s->mw = rich::MeshWork();
    s->hx = std::vector<double>();
    s->hy = std::vector<double>();
    s->perm = std::vector<int32_t>();
    s->W0 = std::vector<double>();
    return RICH_OK;
}

int rich_batch_set_diagnostics(rich_batch *b, int32_t on)
{
    if (!b) return fail(RICH_EINVAL, "NULL handle");
    b->diagnostics = on != 0;
    return RICH_OK;
}

int64_t rich_batch_cells(const rich_batch *b) { return b ? b->cells_admitted : -1; }

int rich_batch_set_launch(rich_batch *b, int32_t mode, int32_t block)
{
    if (!b) return fail(RICH_EINVAL, "NULL handle");
    if (mode < 0 || mode > 2 || (mode == 2 && block != 128 && block != 256 && block != 512))
        return fail(RICH_EINVAL, "mode 0 (autotune), 1 (staged) or 2 (persistent, block 128/256/512)");
    b->launch_mode = mode;
    b->fixed_block = block;
    b->tuned = false;
    b->cands.clear();
    b->cand_next = 0;
    return RICH_OK;
}

int rich_batch_inject_barrier_timeout(rich_batch *b, int32_t spin_limit, int64_t *timeouts_seen)
{
    if (!b || spin_limit < 0) return fail(RICH_EINVAL, "bad arguments");
    if (spin_limit > 0) b->inject_spin = spin_limit;
    if (timeouts_seen) *timeouts_seen = b->barrier_timeouts;
    return RICH_OK;
}

int rich_batch_launch_info(const rich_batch *b, int32_t *persistent, int32_t *block, int32_t *grid, int32_t *tuned,
                           int32_t *graph, int64_t *counts)
{
    if (!b) return fail(RICH_EINVAL, "NULL handle");
    LaunchShape s = b->launch_mode == 1 ? LaunchShape{false, 256}
                    : b->launch_mode == 2 ? LaunchShape{true, b->fixed_block}
                                          : b->chosen;
    if (persistent) *persistent = s.persistent ? 1 : 0;
    if (block) *block = s.block;
    if (grid) *grid = b->last_grid;
    if (tuned) *tuned = (b->launch_mode != 0 || b->tuned) ? 1 : 0;
    if (graph) *graph = b->graph_ok ? 1 : 0;
    if (counts) {
        counts[0] = b->staged_launches;
        counts[1] = b->persistent_launches;
        counts[2] = b->graph_launches;
        counts[3] = b->graph_records;
    }
    return RICH_OK;
}

}  // extern "C"
