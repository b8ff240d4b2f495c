"""GPU tests of batched simulations (rich_batch_*): one device sweep per
step over many independent simulations.  Every simulation in a batch must
give bit-for-bit the same state as when run alone through rich_step, for
any batch composition, including simulations that join mid-run, finish,
or fail."""
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


def mix(precision):
    wls = [W.sod(n_side=24, seed=11), W.sedov(n=2000, seed=12), W.gresho(n_side=20, seed=13),
           W.kelvin_helmholtz(n_side=32, seed=14), W.random_smooth(n=900, seed=15),
           W.random_smooth(n=700, seed=16, boundary=W.BC_REFLECTIVE)]  # a point reaches a wall at step 9
    for wl in wls:
        wl["cfg"]["precision"] = precision
    return wls


def solo(R, wl, steps, t_end=np.inf):
    s = R.Sim(wl)
    s.step(steps, t_end)
    c = s.conserved()
    s.close()
    return c


@pytest.mark.parametrize("precision", [W.FP64, W.FP32_SPLIT])
def test_batch_equals_solo_runs(R, precision):
    wls = mix(precision)
    b = R.Batch(precision=precision)
    ids = [b.add(wl, max_steps=12) for wl in wls]
    for _ in range(12):  # the launch autotuner tries its 8 shapes during these steps
        b.step()
    info = b.launch_info()
    assert info["tuned"] == 1 and info["staged_steps"] >= 2 and info["persistent_steps"] >= 6
    for wl, sid in zip(wls, ids):
        q = b.query(sid)
        assert q["state"] == "done" and q["steps"] == 12, (wl["name"], q)
        got, ref = b.conserved(sid), solo(R, wl, 12)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (wl["name"], k)
    b.close()


def test_batch_admission_mid_run_and_uneven_budgets(R):
    wls = mix(W.FP64)
    b = R.Batch()
    first = [b.add(wl, max_steps=4) for wl in wls[:2]]
    b.step()
    b.step()
    later = [b.add(wl, max_steps=3) for wl in wls[2:4]]
    t_end_sim = b.add(wls[4], t_end=0.004)
    for _ in range(6):
        b.step()
    for wl, sid in zip(wls[:2], first):
        assert b.query(sid)["steps"] == 4
        ref = solo(R, wl, 4)
        got = b.conserved(sid)
        assert all(np.array_equal(got[k], ref[k]) for k in ref)
    for wl, sid in zip(wls[2:4], later):
        assert b.query(sid)["steps"] == 3
        ref = solo(R, wl, 3)
        got = b.conserved(sid)
        assert all(np.array_equal(got[k], ref[k]) for k in ref)
    q = b.query(t_end_sim)
    assert q["state"] == "done" and q["t"] == 0.004
    ref = solo(R, wls[4], 1000, t_end=0.004)
    got = b.conserved(t_end_sim)
    assert all(np.array_equal(got[k], ref[k]) for k in ref)
    b.close()


@pytest.mark.parametrize("mode,block", [(1, 256), (2, 128), (2, 256), (2, 512)])
def test_batch_launch_shapes_give_identical_results(R, mode, block):
    wls = mix(W.FP64)[:4]
    b = R.Batch()
    b.set_launch(mode, block)
    ids = [b.add(wl, max_steps=5) for wl in wls]
    for _ in range(5):
        b.step()
    info = b.launch_info()
    if mode == 2:
        assert info["persistent_steps"] == 5 and info["block"] == block
        if info["graph"]:
            # one recording per ping-pong parity, plus re-recordings when a buffer grows
            assert info["graph_replays"] == 5 and info["graph_recordings"] <= 4
    for wl, sid in zip(wls, ids):
        ref = solo(R, wl, 5)
        got = b.conserved(sid)
        assert all(np.array_equal(got[k], ref[k]) for k in ref), (mode, block, wl["name"])
    b.close()


def test_batch_failure_is_isolated(R):
    good = W.sod(n_side=20, seed=3)
    bad = W.random_mixed(n=600, seed=3)
    bad["vx"] = np.where(bad["x"] < 0.5, -3.0, 3.0)
    bad["cfg"]["cfl"] = 40.0
    b = R.Batch()
    g, f = b.add(good, max_steps=5), b.add(bad, max_steps=5)
    for _ in range(5):
        b.step()
    assert b.query(f)["state"] == "failed"
    assert b.query(f)["error"] in (-5, -6)
    assert b.query(g)["state"] == "done"
    ref = solo(R, good, 5)
    got = b.conserved(g)
    assert all(np.array_equal(got[k], ref[k]) for k in ref)
    b.close()


def test_batch_budget_rejects_overflow(R):
    b = R.Batch(max_cells=3000)
    b.add(W.sod(n_side=40, seed=1), max_steps=1)  # 1600 cells
    with pytest.raises(R.RichError) as e:
        b.add(W.sod(n_side=40, seed=2), max_steps=1)
    assert e.value.code == -7
    b.step()  # finishes and frees its cells
    b.add(W.sod(n_side=40, seed=2), max_steps=1)
    b.close()
