"""rich_step overlaps the host tessellation of the moved points with the
end of the sweep: the points are read back as soon as the point motion
(a9) is done, and the next mesh is built on the host while the device
computes the gradients, fluxes and update.  Its results must equal, bit for
bit, those of the pieces API (rich_tessellate, rich_sweep, rich_sync), which
does each part of a step in turn, and the step's diagnostics must still
describe the sweep that was run."""
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


def _pieces_step(R, sim, scheme):
    for _ in range(2 if scheme == W.SCHEME_TIME_CENTRED else 1):
        R.rich_tessellate(sim.h)
        R.rich_sweep(sim.h, float("inf"))
        R.rich_sync(sim.h)


@pytest.mark.parametrize("scheme", [W.SCHEME_EXTRAPOLATED, W.SCHEME_TIME_CENTRED])
@pytest.mark.parametrize("precision", [W.FP64, W.FP32_SPLIT])
@pytest.mark.parametrize("name,make", [
    ("kh_64", lambda: W.kelvin_helmholtz(n_side=64, amp=0.1)),
    ("sod_reflective_40", lambda: W.sod(n_side=40)),
])
def test_pipelined_steps_equal_the_pieces_api(R, name, make, scheme, precision):
    wl = make()
    wl["cfg"]["scheme"] = scheme
    wl["cfg"]["precision"] = precision
    a, b = R.Sim(wl), R.Sim(wl)
    for k in range(6):
        # one call of several steps, then single steps (the mesh built at
        # the end of a call serves the next call)
        a.step(3 if k == 0 else 1)
        for _ in range(3 if k == 0 else 1):
            _pieces_step(R, b, scheme)
        ca, cb = a.conserved(), b.conserved()
        for f in ("x", "y", "m", "px", "py", "E"):
            assert np.array_equal(ca[f], cb[f]), (k, f)
        assert R.rich_time(a.h) == R.rich_time(b.h)
    # the step's diagnostics (areas, centres of mass, gradients, mesh
    # velocity) describe the sweep just run, although the next mesh is built
    for f, c in (("area", 0), ("cx", 0), ("cy", 0), ("grad", 3), ("lgrad", 6), ("wx", 0), ("wy", 0)):
        assert np.array_equal(a.field(f, c), b.field(f, c)), f
    # and a read of the current state sees the same mesh and geometry
    sa, sb = a.state(), b.state()
    for f in ("rho", "vx", "vy", "p", "area"):
        assert np.array_equal(sa[f], sb[f]), f
    a.close()
    b.close()


@pytest.mark.parametrize("scheme", [W.SCHEME_EXTRAPOLATED, W.SCHEME_TIME_CENTRED])
def test_pipelined_run_lands_on_t_end_and_continues(R, scheme):
    """A run to t_end: the step that lands on it builds no mesh ahead and
    leaves the time at t_end exactly; a later call to a further t_end then
    meshes the points itself, and a read of the state between the two calls
    (which meshes them too) changes nothing that follows."""
    wl = W.sod(n_side=24)
    wl["cfg"]["scheme"] = scheme
    a, c = R.Sim(wl), R.Sim(wl)
    ia = a.step(1000, 0.01)
    assert ia["t"] == 0.01 and R.rich_time(a.h) == 0.01
    a.step(1000, 0.02)
    assert R.rich_time(a.h) == 0.02
    c.step(1000, 0.01)
    c.state()
    c.step(1000, 0.02)
    ca, cc = a.conserved(), c.conserved()
    for f in ("x", "y", "m", "px", "py", "E"):
        assert np.array_equal(ca[f], cc[f]), f
    a.close()
    c.close()


def test_pipelined_steps_on_a_caller_stream(R):
    """The early read of the moved points waits on the caller's stream when
    the handle runs on one (rich_set_stream)."""
    torch = pytest.importorskip("torch")
    wl = W.kelvin_helmholtz(n_side=48, amp=0.1)
    a, b = R.Sim(wl), R.Sim(wl)
    st = torch.cuda.Stream()
    a.set_stream(st.cuda_stream)
    a.step(4)
    for _ in range(4):
        _pieces_step(R, b, W.SCHEME_EXTRAPOLATED)
    ca, cb = a.conserved(), b.conserved()
    for f in ("x", "y", "m", "px", "py", "E"):
        assert np.array_equal(ca[f], cb[f]), f
    a.set_stream(None)
    a.close()
    b.close()
