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


# launch mode 0 autotunes (staged and persistent trial steps); mode 1 runs
# every step staged, where the meshes of the next step are built on the host
# during each sweep from the points read back early
@pytest.mark.parametrize("mode", [0, 1])
def test_batch_admission_mid_run_and_uneven_budgets(R, mode):
    wls = mix(W.FP64)
    b = R.Batch()
    if mode:
        b.set_launch(mode, 256)
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


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_failure_is_isolated(R, mode):
    good = W.sod(n_side=20, seed=3)
    bad = W.random_mixed(n=600, seed=3)
    bad["vx"] = np.where(bad["x"] < 0.5, -3.0, 3.0)
    bad["cfg"]["cfl"] = 40.0
    b = R.Batch()
    if mode:
        b.set_launch(mode, 256)
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


class _Member:
    """A batch member seen as a simulation (conserved() only), for the
    element-by-element comparison with the oracle."""

    def __init__(self, b, sid):
        self.b, self.sid = b, sid

    def conserved(self):
        return self.b.conserved(self.sid)


def oracle_mix():
    # four kinds and sizes: walls and periodic boxes, Lagrangian rounding on
    return [W.sod(n_side=24, seed=11), W.sedov(n=2000, seed=12), W.gresho(n_side=20, seed=13),
            W.kelvin_helmholtz(n_side=32, seed=14)]


def test_batch_members_match_the_oracle_every_step(R, oracle):
    """FP64: each member of a packed batch equals the oracle run on the same
    inputs, element by element at the 1e-12 per-step tolerance, after each
    of four steps."""
    from tests.gpu_common import compare_conserved
    wls = oracle_mix()
    b = R.Batch(precision=W.FP64)
    ids = [b.add(wl, max_steps=4) for wl in wls]
    refs = [oracle.Sim(wl) for wl in wls]
    for step in range(4):
        b.step()
        for wl, sid, ref in zip(wls, ids, refs):
            ref.step()
            compare_conserved(_Member(b, sid), ref, wl["cfg"])
    b.close()


def test_batch_split_members_match_the_oracle_l1(R, oracle):
    """Split precision: after 30 steps every member's cell masses are within
    1e-5 of the FP64 oracle's in relative L1 (the batch returns conserved
    variables; mass is density times the cell's area), and mass and energy
    are conserved to 1e-10 over the last 29 steps (the Sod tube is left out: its limiter decisions
    behind the shock flip under FP32-size noise, see test_gpu_split.py)."""
    wls = oracle_mix()[1:]
    for wl in wls:
        wl["cfg"]["precision"] = W.FP32_SPLIT
    b = R.Batch(precision=W.FP32_SPLIT)
    ids = [b.add(wl, max_steps=30) for wl in wls]
    b.step()  # admission: the conserved variables exist from the first step on
    c0 = [b.conserved(sid) for sid in ids]
    for _ in range(29):
        b.step()
    for wl, sid, c in zip(wls, ids, c0):
        assert b.query(sid)["steps"] == 30
        ref = oracle.Sim(wl)
        for _ in range(30):
            ref.step()
        got, exp = b.conserved(sid), ref.conserved()
        l1 = float(np.sum(np.abs(got["m"] - exp["m"])) / np.sum(np.abs(exp["m"])))
        assert l1 <= 1e-5, (wl["name"], l1)
        for q in ("m", "E"):
            drift = abs(got[q].sum() - c[q].sum()) / np.abs(c[q]).sum()
            assert drift <= 1e-10, (wl["name"], q, drift)
    b.close()


def test_persistent_barrier_timeout_falls_back_to_staged(R):
    """Failure detection of the persistent sweep: its grid barrier is made
    to wait for one block more than the launch has, every wait runs out
    after a few thousand polls, the kernel returns, the batch sees the
    timeout flag, redoes the step with staged launches and keeps them; the
    results still equal the solo runs."""
    wls = mix(W.FP64)[:4]
    b = R.Batch()
    b.set_launch(2, 256)
    ids = [b.add(wl, max_steps=4) for wl in wls]
    b.step()
    assert b.launch_info()["persistent"] == 1
    assert b.inject_barrier_timeout() == 0
    b.inject_barrier_timeout(4096)
    b.step()  # the persistent sweep gives up; the step is redone stage by stage
    info = b.launch_info()
    assert b.inject_barrier_timeout() == 1
    assert info["persistent"] == 0 and info["staged_steps"] >= 1
    b.step()
    b.step()
    for wl, sid in zip(wls, ids):
        q = b.query(sid)
        assert q["state"] == "done" and q["steps"] == 4
        ref = solo(R, wl, 4)
        got = b.conserved(sid)
        assert all(np.array_equal(got[k], ref[k]) for k in ref), wl["name"]
    b.close()
