"""GPU tests of the continuous-batching server (rich_server_*): requests
arriving while others run are admitted as the cell budget frees up, their
work shares one batched sweep per tick, and each result is the same alone
and in the mix (bit for bit)."""
import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_3219_gb300 import rich
    return rich


def requests():
    out = []
    for k in range(9):
        kind = k % 3
        if kind == 0:
            wl = W.sod(n_side=16 + 2 * k, seed=100 + k)
        elif kind == 1:
            wl = W.sedov(n=600 + 150 * k, seed=100 + k)
        else:
            wl = W.gresho(n_side=14 + k, seed=100 + k, eta=0.01 + 0.01 * k, chi=0.5 + 0.1 * k)
        out.append((wl, 3 + (k % 4)))
    return out


def solo(R, wl, steps):
    s = R.Sim(wl)
    s.step(steps)
    c = s.conserved()
    s.close()
    return c


def test_server_results_equal_solo_runs(R):
    reqs = requests()
    budget = 3500  # forces queueing: the requests hold 256..1800 cells each
    srv = R.Server(max_cells=budget)
    ids, arrival_tick, finished = [], {}, {}
    tick = 0
    pending = list(enumerate(reqs))
    max_cells_seen = 0
    while pending or any(srv.query(r)["state"] in ("queued", "running") for r in ids):
        # two new requests arrive every tick while others are on the GPU
        for _ in range(2):
            if pending:
                k, (wl, steps) = pending.pop(0)
                rid = srv.submit(wl, max_steps=steps)
                ids.append(rid)
                arrival_tick[rid] = (k, tick)
        t = srv.tick()
        max_cells_seen = max(max_cells_seen, sum(len(reqs[arrival_tick[r][0]][0]["x"]) for r in ids
                                                 if srv.query(r)["state"] == "running"))
        tick += 1
        assert tick < 200
    assert max_cells_seen <= budget
    for rid in ids:
        q = srv.query(rid)
        k, _ = arrival_tick[rid]
        wl, steps = reqs[k]
        assert q["state"] == "done" and q["steps"] == steps
        assert q["latency_ms"] >= q["queue_ms"] >= 0
        got = srv.fetch(rid)
        ref = solo(R, wl, steps)
        for f in ref:
            assert np.array_equal(got[f], ref[f]), (k, f)
    srv.close()


def test_server_fifo_admission_and_oversize_reject(R):
    srv = R.Server(max_cells=1000)
    big = W.sod(n_side=30, seed=1)  # 900 cells
    small = W.sod(n_side=10, seed=2)  # 100 cells
    a = srv.submit(big, max_steps=2)
    b = srv.submit(big, max_steps=2)
    c = srv.submit(small, max_steps=1)
    srv.tick()
    assert srv.query(a)["state"] == "running"
    # strict arrival order: the small request waits behind the second big one
    assert srv.query(b)["state"] == "queued" and srv.query(c)["state"] == "queued"
    for _ in range(6):
        srv.tick()
    assert all(srv.query(r)["state"] == "done" for r in (a, b, c))
    with pytest.raises(R.RichError):
        srv.submit(W.sod(n_side=40, seed=3), max_steps=1)  # 1600 cells > budget
    srv.close()


def test_server_isolates_a_failing_request(R):
    """A request whose simulation fails (the Sedov blast with 16,384 points
    empties a cell at step 21: the scheme has no floor) ends as 'failed'
    with RICH_ENEGATIVE and its last good state; the requests sharing its
    ticks finish and equal their solo runs."""
    srv = R.Server(max_cells=1 << 20)
    crash = W.sedov(n=16384, seed=2)
    others = [W.sod(n_side=16, seed=7), W.gresho(n_side=14, seed=8)]
    rc = srv.submit(crash, max_steps=40)
    ro = [srv.submit(wl, max_steps=30) for wl in others]
    for _ in range(60):
        srv.tick()
        if all(srv.query(r)["state"] in ("done", "failed") for r in [rc] + ro):
            break
    q = srv.query(rc)
    assert q["state"] == "failed" and q["error"] == R.RICH_ENEGATIVE, q
    assert q["steps"] == 20, q
    got = srv.fetch(rc)
    ref = solo(R, crash, 20)
    for f in ref:
        assert np.array_equal(got[f], ref[f]), f
    for rid, wl in zip(ro, others):
        assert srv.query(rid)["state"] == "done"
        got = srv.fetch(rid)
        ref = solo(R, wl, 30)
        for f in ref:
            assert np.array_equal(got[f], ref[f]), f
    srv.close()


def test_served_mix_matches_the_oracle(R, oracle):
    """Requests served together, admitted as the budget frees up, each end
    within the FP64 parity tolerance of the oracle run of the same request
    (conserved variables and points, element by element)."""
    from tests.gpu_common import compare_conserved
    reqs = [(W.sod(n_side=18, seed=201), 3), (W.sedov(n=1500, seed=202), 4),
            (W.gresho(n_side=16, seed=203, eta=0.05, chi=1.2), 5), (W.kelvin_helmholtz(n_side=24, seed=204), 3)]
    srv = R.Server(max_cells=1600)  # the requests hold 256..1500 cells: some wait for others to finish
    ids = []
    for wl, steps in reqs:
        ids.append(srv.submit(wl, max_steps=steps))
        srv.tick()  # each arrives while the earlier ones are on the GPU
    for _ in range(100):
        if all(srv.query(r)["state"] in ("done", "failed") for r in ids):
            break
        srv.tick()

    class Fetched:
        def __init__(self, c):
            self.c = c

        def conserved(self):
            return self.c

    for (wl, steps), rid in zip(reqs, ids):
        q = srv.query(rid)
        assert q["state"] == "done" and q["steps"] == steps, (wl["name"], q)
        ref = oracle.Sim(wl)
        for _ in range(steps):
            ref.step()
        compare_conserved(Fetched(srv.fetch(rid)), ref, wl["cfg"])
    srv.close()


def wait_all(srv, ids, limit_s=120.0):
    import time
    t0 = time.time()
    while not all(srv.query(r)["state"] in ("done", "failed") for r in ids):
        assert time.time() - t0 < limit_s, [srv.query(r) for r in ids]
        time.sleep(0.005)


def test_lanes_results_equal_solo_runs(R):
    """Asynchronous lanes: requests of both size classes, submitted while
    others run, end bit for bit as their solo runs, within the budget."""
    import time
    reqs = requests() + [(W.kelvin_helmholtz(n_side=48, seed=150), 4), (W.sedov(n=3000, seed=151), 3)]
    srv = R.Server(max_cells=6000)
    # the KH and Sedov requests go to lane 1, which holds at most 3000 cells at once
    srv.start(lanes=2, split_cells=2000, top_lane_cells=3000)
    ids = []
    for wl, steps in reqs:
        ids.append(srv.submit(wl, max_steps=steps))
        time.sleep(0.002)
    wait_all(srv, ids)
    for (wl, steps), rid in zip(reqs, ids):
        q = srv.query(rid)
        assert q["state"] == "done" and q["steps"] == steps, (wl["name"], q)
        got = srv.fetch(rid)
        ref = solo(R, wl, steps)
        for f in ref:
            assert np.array_equal(got[f], ref[f]), (wl["name"], f)
    st = srv.stats()
    assert st["steps"] > 0 and st["sweep_ms"] > 0 and st["tess_ms"] > 0
    with pytest.raises(R.RichError):
        srv.tick()  # the lanes own the stepping
    srv.close()


def test_lanes_small_requests_do_not_wait_for_large_ones(R):
    """A large request submitted first does not hold back small ones in the
    other lane: they finish while it is still running."""
    srv = R.Server(max_cells=1 << 20)
    srv.start(lanes=2, split_cells=20000)
    big = srv.submit(W.kelvin_helmholtz(n_side=256, seed=160), max_steps=40)
    small = [srv.submit(W.sod(n_side=16, seed=161 + k), max_steps=3) for k in range(4)]
    wait_all(srv, small)
    assert srv.query(big)["state"] == "running", srv.query(big)
    wait_all(srv, [big])
    lat_small = max(srv.query(r)["latency_ms"] for r in small)
    assert lat_small < srv.query(big)["latency_ms"]
    for r in small + [big]:
        srv.fetch(r)
    srv.close()


def test_lanes_isolate_a_failing_request_and_admit_an_oversized_one(R):
    """Lanes: a request whose simulation fails (the Sedov blast with 16,384
    points empties a cell at step 21) ends failed with its last good state
    while the others finish and equal their solo runs; a request larger
    than the top lane's cell cap still runs, alone in its lane."""
    srv = R.Server(max_cells=1 << 20)
    srv.start(lanes=2, split_cells=4000, top_lane_cells=5000)
    crash = W.sedov(n=16384, seed=2)  # lane 1, above the cap: admitted alone
    others = [W.sod(n_side=16, seed=7), W.gresho(n_side=14, seed=8), W.kelvin_helmholtz(n_side=64, seed=9)]
    rc = srv.submit(crash, max_steps=40)
    ro = [srv.submit(wl, max_steps=12) for wl in others]
    wait_all(srv, [rc] + ro)
    q = srv.query(rc)
    assert q["state"] == "failed" and q["error"] == R.RICH_ENEGATIVE and q["steps"] == 20, q
    got = srv.fetch(rc)
    ref = solo(R, crash, 20)
    for f in ref:
        assert np.array_equal(got[f], ref[f]), f
    for rid, wl in zip(ro, others):
        assert srv.query(rid)["state"] == "done"
        got = srv.fetch(rid)
        ref = solo(R, wl, 12)
        for f in ref:
            assert np.array_equal(got[f], ref[f]), (wl["name"], f)
    srv.close()


def test_lanes_start_only_before_any_admission(R):
    """The lanes replace the tick-mode batch, so they start only while no
    request has been admitted yet; queued requests move to their lanes."""
    srv = R.Server(max_cells=4000)
    a = srv.submit(W.sod(n_side=12, seed=21), max_steps=2)
    srv.tick()
    with pytest.raises(R.RichError) as e:
        srv.start(lanes=2, split_cells=1000)
    assert e.value.code == R.RICH_ESTATE
    srv.close()
    srv = R.Server(max_cells=4000)
    b = srv.submit(W.sod(n_side=12, seed=22), max_steps=2)  # queued before the start
    srv.start(lanes=2, split_cells=1000)
    wait_all(srv, [b])
    got = srv.fetch(b)
    ref = solo(R, W.sod(n_side=12, seed=22), 2)
    for f in ref:
        assert np.array_equal(got[f], ref[f]), f
    srv.close()
