"""GPU parity: the CUDA FP64 sweep against the CPU oracle, element by
element, on the same seeded inputs (tolerance 1e-12 relative to each field's
scale, per step).  Calls go through the C ABI (librich.so)."""
import math

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


CASES = {
    "sod_32": lambda: W.sod(n_side=32),
    "sod_ragged_37": lambda: W.sod(n_side=37),
    "random_smooth_periodic": lambda: W.random_smooth(n=1500, seed=3),
    "random_smooth_reflective": lambda: W.random_smooth(n=1337, seed=4, boundary=W.BC_REFLECTIVE),
    "random_mixed_reflective": lambda: W.random_mixed(n=2000, seed=8),
    "random_mixed_periodic": lambda: W.random_mixed(n=999, seed=9, boundary=W.BC_PERIODIC),
    "kh_48": lambda: W.kelvin_helmholtz(n_side=48, amp=0.1),
    "gresho_40": lambda: W.gresho(n_side=40),
    "sedov_8192": lambda: W.sedov(n=8192),
    "advection_lattice_16": lambda: W.advection(n_side=16),
    "uniform_eulerian": lambda: W.uniform(n_side=20, motion=W.MESH_EULERIAN),
    "tess_only": lambda: W.random_smooth(n=800, seed=11, limiter=W.LIM_TESS),
    "arepo_only": lambda: W.random_mixed(n=800, seed=12),
}


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_matches_oracle(R, oracle, name):
    wl = CASES[name]()
    if name == "arepo_only":
        wl["cfg"]["limiter"] = W.LIM_AREPO
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    info = gpu.step(1)
    dt = ref.step()
    assert abs(info["dt_last"] - dt) <= TOL * dt
    n = gpu.n
    # intermediate per-cell quantities of the step
    checks = {"area": ("area", 0), "cx": ("cx", 0), "cy": ("cy", 0), "cs": ("cs", 0)}
    for k, (f, c) in checks.items():
        assert rel_err(gpu.field(f, c), ref.field(f, c)) <= TOL, k
    for v in range(4):
        assert rel_err(gpu.field("rho" if v == 0 else ["vx", "vy", "p"][v - 1]),
                       ref.field("rho" if v == 0 else ["vx", "vy", "p"][v - 1])) <= TOL, v
    tess_g, tess_r = gpu.field("tess"), ref.field("tess")
    assert np.array_equal(tess_g, tess_r)
    for c in range(8):
        gg, gr = gpu.field("grad", c), ref.field("grad", c)
        scale = grad_scale(ref, c)
        assert rel_err(gg, gr, scale) <= 1e-11, ("grad", c)
        lg, lr = gpu.field("lgrad", c), ref.field("lgrad", c)
        assert rel_err(lg, lr, scale) <= 1e-11, ("lgrad", c)
    for f in ("wx", "wy"):
        sc = max(np.max(np.abs(ref.field(f))), np.max(ref.field("cs")))
        assert rel_err(gpu.field(f), ref.field(f), sc) <= TOL, f
    compare_conserved(gpu, ref, wl["cfg"])
    gpu.close()


@pytest.mark.parametrize("name", ["sod_32", "random_smooth_periodic", "gresho_40", "kh_48"])
def test_several_steps_match_oracle(R, oracle, name):
    wl = CASES[name]()
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    for k in range(5):
        info = gpu.step(1)
        dt = ref.step()
        assert abs(info["dt_last"] - dt) <= 10 * TOL * dt, k
    compare_conserved(gpu, ref, wl["cfg"], tol=1e-11)
    gpu.close()


def test_run_to_t_end_lands_exactly(R, oracle):
    wl = W.sod(n_side=24)
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    info = gpu.step(1000, t_end=0.02)
    while ref.t < 0.02 - 1e-15:
        ref.step(0.02)
    assert info["t"] == 0.02
    compare_conserved(gpu, ref, wl["cfg"], tol=1e-11)


def test_primitives_on_moved_mesh_match_oracle(R, oracle):
    wl = W.random_smooth(n=1200, seed=5)
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    for _ in range(3):
        gpu.step(1)
        ref.step()
    a, b = gpu.state(), ref.primitives()
    for k in ("rho", "vx", "vy", "p", "area"):
        assert rel_err(a[k], b[k]) <= 1e-11, k


@pytest.mark.parametrize("n", [3, 4, 5, 7, 31, 255, 256, 257, 1025])
def test_ragged_and_tiny_sizes(R, oracle, n):
    rng = np.random.default_rng(n)
    for boundary in (W.BC_REFLECTIVE, W.BC_PERIODIC):
        cfg = W.default_cfg(boundary=boundary)
        wl = dict(cfg=cfg, x=rng.uniform(0.01, 0.99, n), y=rng.uniform(0.01, 0.99, n),
                  rho=rng.uniform(0.5, 2, n), vx=rng.uniform(-0.3, 0.3, n), vy=rng.uniform(-0.3, 0.3, n),
                  p=rng.uniform(0.5, 2, n))
        try:
            ref = oracle.Sim(wl)
        except oracle.OracleError:
            with pytest.raises(R.RichError):
                R.Sim(wl)
            continue
        gpu = R.Sim(wl)
        info = gpu.step(1)
        dt = ref.step()
        assert abs(info["dt_last"] - dt) <= TOL * dt
        compare_conserved(gpu, ref, cfg)
        gpu.close()


def test_invalid_inputs_are_rejected(R):
    wl = W.sod(n_side=8)
    bad = []
    for mod in ("empty", "two", "outside", "rho", "pressure", "nan", "dup", "gamma"):
        w = {k: (v.copy() if isinstance(v, np.ndarray) else dict(v) if isinstance(v, dict) else v)
             for k, v in wl.items()}
        if mod == "empty":
            for k in ("x", "y", "rho", "vx", "vy", "p"):
                w[k] = w[k][:0]
        elif mod == "two":
            for k in ("x", "y", "rho", "vx", "vy", "p"):
                w[k] = w[k][:2]
        elif mod == "outside":
            w["x"][3] = 1.5
        elif mod == "rho":
            w["rho"][2] = 0.0
        elif mod == "pressure":
            w["p"][5] = -1.0
        elif mod == "nan":
            w["vx"][1] = np.nan
        elif mod == "dup":
            w["x"][7], w["y"][7] = w["x"][6], w["y"][6]
        elif mod == "gamma":
            w["cfg"]["gamma"] = 1.0
        with pytest.raises(R.RichError) as e:
            R.Sim(w)
        bad.append((mod, e.value.code))
    codes = dict(bad)
    assert codes["dup"] == -2
    assert all(c == -1 for m, c in bad if m != "dup")


def test_failed_step_keeps_last_good_state(R):
    """A step that would make the thermal energy negative (here forced by a
    Courant number far above the stable range on a strong rarefaction) is
    reported on the host and leaves the state at the previous step."""
    wl = W.random_mixed(n=600, seed=3)
    wl["vx"] = np.where(wl["x"] < 0.5, -3.0, 3.0)
    wl["cfg"]["cfl"] = 40.0
    gpu = R.Sim(wl)
    before = gpu.conserved()
    with pytest.raises(R.RichError) as e:
        for _ in range(5):
            gpu.step(1)
            before = gpu.conserved()
    assert e.value.code in (-5, -6)
    after = gpu.conserved()
    for k in before:
        assert np.array_equal(before[k], after[k]), k


def test_conservation_on_gpu(R):
    wl = W.kelvin_helmholtz(n_side=64)
    gpu = R.Sim(wl)
    c0 = gpu.conserved()
    T0 = np.array([c0[k].sum() for k in ("m", "px", "py", "E")])
    S0 = np.array([np.abs(c0[k]).sum() for k in ("m", "px", "py", "E")])
    gpu.step(20)
    c1 = gpu.conserved()
    T1 = np.array([c1[k].sum() for k in ("m", "px", "py", "E")])
    assert np.all(np.abs(T1 - T0) <= 1e-13 * 20 * S0)
