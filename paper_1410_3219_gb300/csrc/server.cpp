// Continuous-batching simulation server (include/rich.h, rich_server_*).
//
// Requests (a simulation: points, initial fields, scheme parameters, end
// time or step budget) are queued on submission with host copies of their
// inputs.  Admission takes queued requests in arrival order while their
// cells fit in the device budget; every admitted simulation advances one
// step per batched device sweep (rich_batch_step).  Simulations that finish
// leave the batch at once, so their cells become free for the next
// admissions; requests that arrive while others run join at the next step.
// Per request the server records queueing time (submission to admission)
// and latency (submission to the end of its last step).
//
// Two ways of driving it:
//   ticks  the caller's thread admits and steps one batch (rich_server_tick);
//   lanes  rich_server_start hands the work to lane threads, each stepping
//          its own batch (own CUDA stream) in a loop; the lanes share one
//          pool of host workers task by task, the lanes of larger requests
//          first.  Requests go to a lane by size, so a small request's step
//          never waits for the whole host tessellation of a large one, and
//          one lane's host work overlaps another lane's device sweep.
//          Admission against the shared cell budget stays in arrival order
//          within a lane.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "api_internal.h"
#include "threadpool.h"

namespace {

int fail(int code, const std::string &msg) { return rich::set_error(code, msg); }

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3 };

struct Request {
    int64_t id = 0;
    rich_config cfg{};
    int64_t n = 0;
    std::vector<double> in;  // x, y, rho, vx, vy, p
    double t_end = 0.0;
    int64_t max_steps = 0;
    int state = QUEUED;
    int lane = 0;
    int32_t sim = -1;  // batch simulation id once admitted
    int64_t steps = 0;  // steps taken, as of the lane's last step
    int32_t error = RICH_OK;
    double t_submit = 0.0, t_admit = 0.0, t_finish = 0.0;
};

struct Lane {
    rich_batch *batch = nullptr;
    std::deque<int64_t> queue;  // requests routed here, arrival order (server mutex)
    std::mutex mu;              // guards the batch: steps, reads, removals
    std::thread th;
    int64_t cells = 0;  // cells of its running requests (server mutex)
    // totals of the lane's steps (server mutex)
    int64_t steps = 0;
    double sweep_ms = 0.0, tess_ms = 0.0, other_ms = 0.0;
    ~Lane()
    {
        if (batch) rich_batch_destroy(batch);
    }
};

}  // namespace

struct rich_server {
    int32_t precision = RICH_FP64;
    int32_t host_threads = 0;
    int64_t max_cells = 0;
    int64_t next_id = 1;
    int64_t cells_admitted = 0;  // running requests over all lanes
    std::vector<std::unique_ptr<Lane>> lanes;
    int64_t split_cells = 0;  // lane of a request: number of lane thresholds at or below its n
    int64_t top_lane_cells = 0;  // cells the lane of the largest requests holds at once (0: the budget)
    bool async = false;
    int device = 0;
    std::atomic<bool> stop{false};
    std::mutex mu;  // requests, queues, admission count, lane totals
    std::condition_variable cv;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    double t_start = 0.0;
    // lanes mode: one pool of host workers for every lane, shared task by
    // task (larger lanes first), so a lane alone gets all of it
    std::unique_ptr<rich::ThreadPool> pool;

    ~rich_server()
    {
        stop.store(true);
        cv.notify_all();
        for (auto &l : lanes)
            if (l->th.joinable()) l->th.join();
        lanes.clear();  // the batches before the pool they share
    }

    int lane_of(int64_t n) const
    {
        if (lanes.size() < 2) return 0;
        int k = 0;
        int64_t t = split_cells;
        while (k + 1 < (int)lanes.size() && n >= t) {
            k++;
            t *= 8;
        }
        return k;
    }

    // Admit queued requests of lane k in arrival order while the budget
    // allows (server mutex held; takes the lane's batch mutex).
    int admit(int k)
    {
        Lane &L = *lanes[k];
        const bool top = lanes.size() > 1 && k + 1 == (int)lanes.size() && top_lane_cells > 0;
        int adm = 0;
        while (!L.queue.empty()) {
            Request &r = *reqs[L.queue.front()];
            if (cells_admitted + r.n > max_cells) break;
            if (top && L.cells > 0 && L.cells + r.n > top_lane_cells) break;
            const size_t n = (size_t)r.n;
            int rc;
            {
                std::lock_guard<std::mutex> lk(L.mu);
                rc = rich_batch_add(L.batch, &r.cfg, r.n, &r.in[0], &r.in[n], &r.in[2 * n], &r.in[3 * n],
                                    &r.in[4 * n], &r.in[5 * n], r.t_end, r.max_steps, &r.sim);
            }
            L.queue.pop_front();
            if (rc) {
                r.state = FAILED;
                r.error = rc;
                r.t_finish = rich::now_ms();
            } else {
                r.state = RUNNING;
                r.t_admit = rich::now_ms();
                cells_admitted += r.n;
                L.cells += r.n;
                adm++;
            }
            r.in.clear();
            r.in.shrink_to_fit();
        }
        return adm;
    }

    // After a step of lane k: finished requests leave (server mutex held).
    int settle(int k)
    {
        Lane &L = *lanes[k];
        int run = 0;
        for (auto &kv : reqs) {
            Request &r = *kv.second;
            if (r.state != RUNNING || r.lane != k) continue;
            int32_t st = 0, err = 0;
            {
                std::lock_guard<std::mutex> lk(L.mu);
                rich_batch_query(L.batch, r.sim, &st, &err, nullptr, &r.steps, nullptr);
            }
            if (st == RICH_SIM_DONE || st == RICH_SIM_FAILED) {
                r.state = st == RICH_SIM_DONE ? DONE : FAILED;
                r.error = err;
                r.t_finish = rich::now_ms();
                cells_admitted -= r.n;
                L.cells -= r.n;
            } else {
                run++;
            }
        }
        return run;
    }

    static void account(Lane &L, const rich_step_info &info)
    {
        L.steps++;
        L.sweep_ms += info.sweep_ms;
        L.tess_ms += info.tess_ms;
        L.other_ms += info.copy_ms;
    }

    void lane_loop(int k)
    {
        cudaSetDevice(device);
        // the lanes of larger requests get the shared workers first: their
        // steps are long and sequential, the small lane fills idle workers
        rich::ThreadPool::set_priority(k);
        Lane &L = *lanes[k];
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            if (stop.load()) return;
            admit(k);
            int64_t live;
            {
                std::lock_guard<std::mutex> bl(L.mu);
                live = rich_batch_cells(L.batch);
            }
            if (live <= 0) {
                // nothing admitted here: wait for a submission or for cells
                // freed by another lane
                cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            lk.unlock();
            rich_step_info info{};
            int rc;
            {
                std::lock_guard<std::mutex> bl(L.mu);
                rc = rich_batch_step(L.batch, &info);
            }
            lk.lock();
            if (rc == RICH_OK) {
                account(L, info);
            } else {
                // a batch-level failure (a device error): every running
                // request of this lane fails with it and leaves the batch
                for (auto &kv : reqs) {
                    Request &r = *kv.second;
                    if (r.lane == k && r.state == RUNNING) {
                        r.state = FAILED;
                        r.error = rc;
                        r.t_finish = rich::now_ms();
                        cells_admitted -= r.n;
                        L.cells -= r.n;
                        std::lock_guard<std::mutex> bl(L.mu);
                        rich_batch_remove(L.batch, r.sim);
                        r.sim = -1;
                    }
                }
                cv.notify_all();
                continue;
            }
            const int64_t before = cells_admitted;
            settle(k);
            if (cells_admitted != before) cv.notify_all();
        }
    }
};

extern "C" {

int rich_server_create(int32_t precision, int64_t max_cells, int32_t host_threads, rich_server **out)
{
    if (!out) return fail(RICH_EINVAL, "out is NULL");
    *out = nullptr;
    rich_server *s = new (std::nothrow) rich_server();
    if (!s) return fail(RICH_ENOMEM, "host allocation");
    auto lane = std::make_unique<Lane>();
    int rc = rich_batch_create(precision, max_cells, host_threads, &lane->batch);
    if (rc) {
        delete s;
        return rc;
    }
    s->lanes.push_back(std::move(lane));
    s->precision = precision;
    s->host_threads = host_threads > 0 ? host_threads : (int32_t)std::max(1u, std::thread::hardware_concurrency());
    s->max_cells = max_cells;
    cudaGetDevice(&s->device);
    *out = s;
    return RICH_OK;
}

void rich_server_destroy(rich_server *s) { delete s; }

int rich_server_start(rich_server *s, int32_t lanes, int64_t split_cells, int64_t top_lane_cells)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    if (lanes < 1 || lanes > 4 || (lanes > 1 && split_cells < 3) || top_lane_cells < 0)
        return fail(RICH_EINVAL, "1-4 lanes, split >= 3, top_lane_cells >= 0");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->async) return fail(RICH_ESTATE, "the server's lanes run already");
    // (a request that ran in tick mode keeps its results in the tick batch,
    // which the lanes replace)
    bool ran = s->cells_admitted > 0 || rich_batch_cells(s->lanes[0]->batch) > 0;
    for (auto &kv : s->reqs) ran = ran || kv.second->state != QUEUED;
    if (ran) return fail(RICH_ESTATE, "start the lanes before any request is admitted");
    s->lanes.clear();
    if (!s->pool) s->pool = std::make_unique<rich::ThreadPool>(s->host_threads);
    for (int k = 0; k < lanes; k++) {
        auto lane = std::make_unique<Lane>();
        int rc = rich::batch_create(s->precision, s->max_cells, 0, s->pool.get(), &lane->batch);
        if (rc) {
            s->lanes.clear();
            rich_batch *b = nullptr;
            if (rich_batch_create(s->precision, s->max_cells, s->host_threads, &b) == RICH_OK) {
                auto l0 = std::make_unique<Lane>();
                l0->batch = b;
                s->lanes.push_back(std::move(l0));
            }
            return rc;
        }
        s->lanes.push_back(std::move(lane));
    }
    s->split_cells = split_cells;
    s->top_lane_cells = top_lane_cells;
    // requests queued before the start move to their lanes
    std::vector<int64_t> queued;
    for (auto &kv : s->reqs)
        if (kv.second->state == QUEUED) queued.push_back(kv.first);
    for (int64_t id : queued) {
        Request &r = *s->reqs[id];
        r.lane = s->lane_of(r.n);
        s->lanes[r.lane]->queue.push_back(id);
    }
    s->async = true;
    s->t_start = rich::now_ms();
    for (int k = 0; k < lanes; k++) s->lanes[k]->th = std::thread([s, k] { s->lane_loop(k); });
    return RICH_OK;
}

int rich_server_submit(rich_server *s, const rich_config *cfg, int64_t n, const double *x, const double *y,
                       const double *rho, const double *vx, const double *vy, const double *p, double t_end,
                       int64_t max_steps, int64_t *req)
{
    if (!s || !cfg || !req) return fail(RICH_EINVAL, "NULL argument");
    if (n < 3 || n > s->max_cells) return fail(RICH_EINVAL, "n must be in [3, the server's cell budget]");
    if (!x || !y || !rho || !vx || !vy || !p) return fail(RICH_EINVAL, "NULL input array");
    if (cfg->scheme != RICH_SCHEME_EXTRAPOLATED)
        return fail(RICH_EINVAL, "the server runs the extrapolated-fluxes scheme only");
    auto r = std::make_unique<Request>();
    r->cfg = *cfg;
    r->n = n;
    r->in.resize(6 * (size_t)n);
    const double *src[6] = {x, y, rho, vx, vy, p};
    for (int f = 0; f < 6; f++) std::memcpy(&r->in[(size_t)f * n], src[f], sizeof(double) * n);
    r->t_end = t_end;
    r->max_steps = max_steps;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        r->t_submit = rich::now_ms();
        r->lane = s->lane_of(n);
        *req = r->id;
        s->lanes[r->lane]->queue.push_back(r->id);
        s->reqs[r->id] = std::move(r);
    }
    s->cv.notify_all();
    return RICH_OK;
}

int rich_server_tick(rich_server *s, rich_step_info *info, int32_t *admitted, int32_t *running, int32_t *queued)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->async) return fail(RICH_ESTATE, "the server's lanes step it (rich_server_start)");
    const int32_t adm = s->admit(0);
    lk.unlock();
    rich_step_info local{};
    int rc;
    {
        std::lock_guard<std::mutex> bl(s->lanes[0]->mu);
        rc = rich_batch_step(s->lanes[0]->batch, &local);
    }
    lk.lock();
    if (rc) return rc;
    if (info) *info = local;
    s->account(*s->lanes[0], local);
    const int32_t run = s->settle(0);
    if (admitted) *admitted = adm;
    if (running) *running = run;
    if (queued) *queued = (int32_t)s->lanes[0]->queue.size();
    return RICH_OK;
}

int rich_server_query(rich_server *s, int64_t req, int32_t *state, int32_t *error, int64_t *steps, double *queue_ms,
                      double *latency_ms)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(RICH_EINVAL, "unknown request");
    Request &r = *it->second;
    if (state) *state = r.state;
    if (error) *error = r.error;
    if (steps) *steps = r.steps;
    if (queue_ms) *queue_ms = r.state == QUEUED ? -1.0 : (r.t_admit > 0 ? r.t_admit : r.t_finish) - r.t_submit;
    if (latency_ms) *latency_ms = (r.state == DONE || r.state == FAILED) ? r.t_finish - r.t_submit : -1.0;
    return RICH_OK;
}

int rich_server_fetch(rich_server *s, int64_t req, int64_t n, double *x, double *y, double *m, double *px,
                      double *py, double *E)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    Lane *L = nullptr;
    int32_t sim = -1;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(req);
        if (it == s->reqs.end()) return fail(RICH_EINVAL, "unknown request");
        Request &r = *it->second;
        if (r.state != DONE && r.state != FAILED) return fail(RICH_ESTATE, "request not finished");
        if (r.sim < 0) return fail(RICH_ESTATE, "request never ran");
        L = s->lanes[r.lane].get();
        sim = r.sim;
    }
    {
        // the lane may be stepping: wait for it without holding the server
        // mutex, so the other lanes keep admitting and settling
        std::lock_guard<std::mutex> bl(L->mu);
        int rc = rich_batch_get_conserved(L->batch, sim, n, x, y, m, px, py, E);
        if (rc) return rc;
        rich_batch_remove(L->batch, sim);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->reqs.erase(req);
    return RICH_OK;
}

int rich_server_stats(rich_server *s, int64_t *steps, double *sweep_ms, double *tess_ms, double *other_ms,
                      double *wall_ms)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t st = 0;
    double sw = 0.0, te = 0.0, ot = 0.0;
    for (auto &l : s->lanes) {
        st += l->steps;
        sw += l->sweep_ms;
        te += l->tess_ms;
        ot += l->other_ms;
    }
    if (steps) *steps = st;
    if (sweep_ms) *sweep_ms = sw;
    if (tess_ms) *tess_ms = te;
    if (other_ms) *other_ms = ot;
    if (wall_ms) *wall_ms = s->async ? rich::now_ms() - s->t_start : 0.0;
    return RICH_OK;
}

rich_batch *rich_server_batch(rich_server *s) { return s && !s->lanes.empty() ? s->lanes[0]->batch : nullptr; }

}  // extern "C"
