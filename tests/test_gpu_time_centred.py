"""GPU parity of the time-centred-fluxes scheme (Section 2.3; two sweeps and
two tessellations per step) against the oracle, through the C ABI:
per-step FP64 parity at 1e-12 of each field's scale (the per-cell fields
describe the step's second sweep, on the half-step mesh), several steps,
a whole Sod run, split precision, the two-round pieces API, and the
rejection of the scheme by batches."""
import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W
from tests.gpu_common import TOL, compare_conserved, grad_scale, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_3219_gb300 import rich
    return rich


def tc(wl):
    wl["cfg"]["scheme"] = W.SCHEME_TIME_CENTRED
    return wl


CASES = {
    "sod_32": lambda: W.sod(n_side=32),
    "sod_ragged_37": lambda: W.sod(n_side=37),
    "random_smooth_periodic": lambda: W.random_smooth(n=1500, seed=3),
    "random_mixed_reflective": lambda: W.random_mixed(n=2000, seed=8),
    "kh_48": lambda: W.kelvin_helmholtz(n_side=48, amp=0.1),
    "gresho_40": lambda: W.gresho(n_side=40),
    "sedov_8192": lambda: W.sedov(n=8192),
    "advection_lattice_16": lambda: W.advection(n_side=16),
    "uniform_eulerian": lambda: W.uniform(n_side=20, motion=W.MESH_EULERIAN),
}


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_matches_oracle(R, oracle, name):
    wl = tc(CASES[name]())
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    info = gpu.step(1)
    dt = ref.step()
    assert info["steps_done"] == 1
    assert abs(info["dt_last"] - dt) <= TOL * dt
    for f in ("area", "cx", "cy", "cs", "rho", "vx", "vy", "p"):
        assert rel_err(gpu.field(f), ref.field(f)) <= TOL, f
    assert np.array_equal(gpu.field("tess"), ref.field("tess"))
    for c in range(8):
        gr = ref.field("grad", c)
        scale = grad_scale(ref, c)
        assert rel_err(gpu.field("grad", c), gr, scale) <= 1e-11, ("grad", c)
        assert rel_err(gpu.field("lgrad", c), ref.field("lgrad", c), scale) <= 1e-11, ("lgrad", c)
    for f in ("wx", "wy"):
        sc = max(np.max(np.abs(ref.field(f))), np.max(ref.field("cs")))
        assert rel_err(gpu.field(f), ref.field(f), sc) <= TOL, f
    compare_conserved(gpu, ref, wl["cfg"])
    gpu.close()


@pytest.mark.parametrize("name", ["sod_32", "random_smooth_periodic", "gresho_40", "kh_48"])
def test_several_steps_match_oracle(R, oracle, name):
    wl = tc(CASES[name]())
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    for k in range(5):
        info = gpu.step(1)
        dt = ref.step()
        assert abs(info["dt_last"] - dt) <= 10 * TOL * dt, k
    compare_conserved(gpu, ref, wl["cfg"], tol=1e-11)
    gpu.close()


def test_sod_run_matches_oracle(R, oracle):
    wl = tc(W.sod(n_side=64))
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    k = 0
    while ref.t < 0.2 - 1e-14:
        ref.step(0.2)
        k += 1
    info = gpu.step(100000, 0.2)
    assert info["steps_done"] == k
    a, b = gpu.state(), ref.primitives()
    l1 = float(np.sum(np.abs(a["rho"] - b["rho"])) / np.sum(np.abs(b["rho"])))
    print(f"time-centred Sod 64^2 t=0.2: {k} steps, L1(rho) GPU vs oracle {l1:.2e}")
    assert l1 <= 1e-10
    gpu.close()


def test_split_precision_run(R, oracle):
    wl = tc(W.gresho(n_side=32))
    ref = oracle.Sim(wl)
    ws = tc(W.gresho(n_side=32))
    ws["cfg"]["precision"] = W.FP32_SPLIT
    gpu = R.Sim(ws)
    c0 = gpu.conserved()
    k = 0
    while ref.t < 0.1 - 1e-14:
        ref.step(0.1)
        k += 1
    info = gpu.step(100000, 0.1)
    assert info["steps_done"] == k
    a, b = gpu.state(), ref.primitives()
    l1 = float(np.sum(np.abs(a["rho"] - b["rho"])) / np.sum(np.abs(b["rho"])))
    print(f"time-centred split Gresho 32^2 t=0.1: L1(rho) vs oracle {l1:.2e}")
    assert l1 <= 1e-5
    c1 = gpu.conserved()
    for q in ("m", "E", "px", "py"):
        drift = abs(c1[q].sum() - c0[q].sum()) / np.abs(c0[q]).sum()
        assert drift <= 1e-10, (q, drift)
    gpu.close()


def test_pieces_api_takes_two_rounds(R, oracle):
    wl = tc(W.random_smooth(n=700, seed=5))
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    c0 = gpu.conserved()
    gpu.tessellate()
    gpu.sweep()
    i1 = gpu.sync()
    assert i1["steps_done"] == 0 and i1["t"] == 0.0
    half = gpu.conserved()  # the half-step state and points
    assert not np.array_equal(half["x"], c0["x"])
    gpu.tessellate()
    gpu.sweep()
    i2 = gpu.sync()
    dt = ref.step()
    assert i2["steps_done"] == 1 and abs(i2["t"] - dt) <= TOL * dt
    compare_conserved(gpu, ref, wl["cfg"])
    gpu.close()


def test_batches_and_server_reject_the_scheme(R):
    wl = tc(W.sod(n_side=16))
    b = R.Batch()
    with pytest.raises(R.RichError):
        b.add(wl)
    b.close()
    s = R.Server()
    with pytest.raises(R.RichError):
        s.submit(wl)
    s.close()


def test_area_inconsistency_orders_on_gpu(R, oracle):
    """Section 5 on the GPU: a fluid at rest on a rounding mesh, one step in
    each scheme at Courant numbers 0.4, 0.2, 0.1.  The density error (the
    area inconsistency) matches the oracle's cell by cell, and its median
    over the cells falls as dt^2 (extrapolated fluxes) and dt^3
    (time-centred fluxes)."""
    err = {}
    for scheme in (W.SCHEME_EXTRAPOLATED, W.SCHEME_TIME_CENTRED):
        err[scheme] = []
        for cfl in (0.4, 0.2, 0.1):
            wl = W.uniform(n_side=24, jitter=0.3, boundary=W.BC_REFLECTIVE, vx=0.0, vy=0.0)
            wl["cfg"] = dict(wl["cfg"], cfl=cfl, scheme=scheme)
            gpu, ref = R.Sim(wl), oracle.Sim(wl)
            gpu.step(1)
            ref.step()
            rg, rr = gpu.state()["rho"], ref.primitives()["rho"]
            assert np.max(np.abs(rg - rr)) <= TOL * np.max(np.abs(rr))
            eg = rg / 1.3 - 1.0
            err[scheme].append(float(np.median(np.abs(eg))))
            gpu.close()
    ex, tcs = err[W.SCHEME_EXTRAPOLATED], err[W.SCHEME_TIME_CENTRED]
    for k in range(2):
        assert 3.5 < ex[k] / ex[k + 1] < 4.5, ex
        assert 7.0 < tcs[k] / tcs[k + 1] < 9.5, tcs
    assert ex[0] > 2.0 * tcs[0]
