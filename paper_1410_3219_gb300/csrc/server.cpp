// Continuous-batching simulation server (include/rich.h, rich_server_*).
//
// Requests (a simulation: points, initial fields, scheme parameters, end
// time or step budget) are queued on submission with host copies of their
// inputs.  Each tick admits queued requests in arrival order while their
// cells fit in the device budget, then advances every admitted simulation by
// one step in one batched device sweep (rich_batch_step).  Simulations that
// finish leave the batch at once, so their cells become free for the next
// admissions; requests that arrive while others run join at the next tick.
// Per request the server records queueing time (submission to admission) and
// latency (submission to the end of its last step).
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "api_internal.h"

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
    int32_t sim = -1;  // batch simulation id once admitted
    int32_t error = RICH_OK;
    double t_submit = 0.0, t_admit = 0.0, t_finish = 0.0;
};

}  // namespace

struct rich_server {
    rich_batch *batch = nullptr;
    int64_t max_cells = 0;
    int64_t next_id = 1;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    ~rich_server()
    {
        if (batch) rich_batch_destroy(batch);
    }
};

extern "C" {

int rich_server_create(int32_t precision, int64_t max_cells, int32_t host_threads, rich_server **out)
{
    if (!out) return fail(RICH_EINVAL, "out is NULL");
    *out = nullptr;
    rich_server *s = new (std::nothrow) rich_server();
    if (!s) return fail(RICH_ENOMEM, "host allocation");
    int rc = rich_batch_create(precision, max_cells, host_threads, &s->batch);
    if (rc) {
        delete s;
        return rc;
    }
    s->max_cells = max_cells;
    *out = s;
    return RICH_OK;
}

void rich_server_destroy(rich_server *s) { delete s; }

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
    r->id = s->next_id++;
    r->cfg = *cfg;
    r->n = n;
    r->in.resize(6 * (size_t)n);
    const double *src[6] = {x, y, rho, vx, vy, p};
    for (int f = 0; f < 6; f++) std::memcpy(&r->in[(size_t)f * n], src[f], sizeof(double) * n);
    r->t_end = t_end;
    r->max_steps = max_steps;
    r->t_submit = rich::now_ms();
    *req = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    return RICH_OK;
}

int rich_server_tick(rich_server *s, rich_step_info *info, int32_t *admitted, int32_t *running, int32_t *queued)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    int32_t adm = 0;
    // admit in arrival order while the budget allows
    while (!s->queue.empty()) {
        Request &r = *s->reqs[s->queue.front()];
        if (rich_batch_cells(s->batch) + r.n > s->max_cells) break;
        const size_t n = (size_t)r.n;
        int rc = rich_batch_add(s->batch, &r.cfg, r.n, &r.in[0], &r.in[n], &r.in[2 * n], &r.in[3 * n], &r.in[4 * n],
                                &r.in[5 * n], r.t_end, r.max_steps, &r.sim);
        s->queue.pop_front();
        if (rc) {
            r.state = FAILED;
            r.error = rc;
            r.t_finish = rich::now_ms();
        } else {
            r.state = RUNNING;
            r.t_admit = rich::now_ms();
            adm++;
        }
        r.in.clear();
        r.in.shrink_to_fit();
    }
    int rc = rich_batch_step(s->batch, info);
    if (rc) return rc;
    int32_t run = 0;
    for (auto &kv : s->reqs) {
        Request &r = *kv.second;
        if (r.state != RUNNING) continue;
        int32_t st = 0, err = 0;
        rich_batch_query(s->batch, r.sim, &st, &err, nullptr, nullptr, nullptr);
        if (st == RICH_SIM_DONE || st == RICH_SIM_FAILED) {
            r.state = st == RICH_SIM_DONE ? DONE : FAILED;
            r.error = err;
            r.t_finish = rich::now_ms();
        } else {
            run++;
        }
    }
    if (admitted) *admitted = adm;
    if (running) *running = run;
    if (queued) *queued = (int32_t)s->queue.size();
    return RICH_OK;
}

int rich_server_query(rich_server *s, int64_t req, int32_t *state, int32_t *error, int64_t *steps, double *queue_ms,
                      double *latency_ms)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(RICH_EINVAL, "unknown request");
    Request &r = *it->second;
    if (state) *state = r.state;
    if (error) *error = r.error;
    if (steps) {
        *steps = 0;
        if (r.sim >= 0) rich_batch_query(s->batch, r.sim, nullptr, nullptr, nullptr, steps, nullptr);
    }
    if (queue_ms) *queue_ms = r.state == QUEUED ? -1.0 : (r.t_admit > 0 ? r.t_admit : r.t_finish) - r.t_submit;
    if (latency_ms) *latency_ms = (r.state == DONE || r.state == FAILED) ? r.t_finish - r.t_submit : -1.0;
    return RICH_OK;
}

int rich_server_fetch(rich_server *s, int64_t req, int64_t n, double *x, double *y, double *m, double *px,
                      double *py, double *E)
{
    if (!s) return fail(RICH_EINVAL, "NULL handle");
    auto it = s->reqs.find(req);
    if (it == s->reqs.end()) return fail(RICH_EINVAL, "unknown request");
    Request &r = *it->second;
    if (r.state != DONE && r.state != FAILED) return fail(RICH_ESTATE, "request not finished");
    if (r.sim < 0) return fail(RICH_ESTATE, "request never ran");
    int rc = rich_batch_get_conserved(s->batch, r.sim, n, x, y, m, px, py, E);
    if (rc) return rc;
    rich_batch_remove(s->batch, r.sim);
    s->reqs.erase(it);
    return RICH_OK;
}

rich_batch *rich_server_batch(rich_server *s) { return s ? s->batch : nullptr; }

}  // extern "C"
