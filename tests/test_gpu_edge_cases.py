"""GPU edge cases through the C ABI, against the oracle where a step is
defined: the fewest points a box takes, collinear generating points (the
mirror images make the set two-dimensional), coincident points (rejected),
and a step that must land exactly on t_end."""
import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W
from tests.gpu_common import TOL, compare_conserved

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_3219_gb300 import rich
    return rich


def _wl(x, y, boundary, seed=0):
    rng = np.random.default_rng(seed)
    n = len(x)
    cfg = W.default_cfg(boundary=boundary, gamma=1.4)
    return dict(name="edge", seed=seed, cfg=cfg, x=np.asarray(x, np.float64), y=np.asarray(y, np.float64),
                rho=1.0 + 0.2 * rng.random(n), vx=0.1 * rng.standard_normal(n), vy=0.1 * rng.standard_normal(n),
                p=1.0 + 0.2 * rng.random(n))


@pytest.mark.parametrize("boundary", [W.BC_PERIODIC, W.BC_REFLECTIVE])
@pytest.mark.parametrize("n", [3, 4, 7])
def test_fewest_points_match_oracle(R, oracle, n, boundary):
    rng = np.random.default_rng(100 + n)
    wl = _wl(0.1 + 0.8 * rng.random(n), 0.1 + 0.8 * rng.random(n), boundary, seed=n)
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    for _ in range(3):
        info = gpu.step(1)
        dt = ref.step()
        assert abs(info["dt_last"] - dt) <= 10 * TOL * dt
    compare_conserved(gpu, ref, wl["cfg"], tol=1e-11)
    gpu.close()


def test_collinear_points_match_oracle(R, oracle):
    """Generating points on one line: the Voronoi cells are strips between
    the walls, and every quadruple of two neighbours and their mirror images
    is co-circular.  One step is compared: the line is not a stable state of
    the scheme (in the oracle too, a point's distance from the line grows by
    ~10^4 per step from round-off, and with random velocities a strip
    empties in the second step), so later steps amplify each side's own
    round-off.  The tolerance is 1e-10: a strip of width w between walls a
    distance 1 apart gets its area from cross products of vectors ~1/(2 w)
    times longer than the strip is wide, so its geometry carries that much
    more round-off than a round cell's."""
    rng = np.random.default_rng(7)
    x = np.sort(rng.uniform(0.05, 0.95, 40))
    wl = _wl(x, np.full(40, 0.5), W.BC_REFLECTIVE, seed=7)
    wl["vx"] = np.zeros(40)
    wl["vy"] = np.zeros(40)
    wl["p"] = np.ones(40)
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    info = gpu.step(1)
    dt = ref.step()
    assert abs(info["dt_last"] - dt) <= 1e-10 * dt
    compare_conserved(gpu, ref, wl["cfg"], tol=1e-10)
    gpu.close()


def test_coincident_points_are_rejected(R):
    wl = W.sod(n_side=8)
    wl["x"], wl["y"] = wl["x"].copy(), wl["y"].copy()
    wl["x"][5], wl["y"][5] = wl["x"][9], wl["y"][9]
    with pytest.raises(R.RichError) as e:
        R.Sim(wl)
    assert e.value.code == R.RICH_EDUPLICATE


def test_last_step_lands_on_t_end(R, oracle):
    wl = W.sod(n_side=16)
    gpu, ref = R.Sim(wl), oracle.Sim(wl)
    dt0 = ref.step()  # one full step, then aim a little past it
    t_end = 1.5 * dt0
    ref.step(t_end)
    info = gpu.step(10, t_end)
    assert info["steps_done"] == 2
    assert info["t"] == t_end and R.rich_time(gpu.h) == t_end
    compare_conserved(gpu, ref, wl["cfg"])
    gpu.close()


@pytest.mark.parametrize("name", ["sod_reflective", "kh_periodic", "random_reflective", "tiny_periodic",
                                  "lattice_periodic"])
def test_device_edge_list_equals_host_list(R, name):
    """The edge list the sweep uses is built on the device from the rings;
    it must equal, entry by entry, the list the host builder makes for the
    same mesh: a reflective box, a periodic box, random points, a periodic
    box so small that cells neighbour their own images, and a co-circular
    lattice."""
    if name == "sod_reflective":
        wl = W.sod(n_side=40, seed=31)
    elif name == "kh_periodic":
        wl = W.kelvin_helmholtz(n_side=48, seed=32)
    elif name == "random_reflective":
        wl = W.random_mixed(n=3000, seed=33)
    elif name == "tiny_periodic":
        wl = W.uniform(n_side=2, jitter=0.2, seed=34)
    else:
        wl = W.uniform(n_side=12, jitter=0.0, seed=35)
    edges, bad = R.rich_edge_list_check(wl["cfg"], wl["x"], wl["y"])
    assert edges > 0 and bad == 0, (name, edges, bad)
