"""Oracle pins for Section 2.2 (Eq. 1 gradient, Eqs. 3-6 limiters) and the
cell-rounding velocity of Section 6."""
import math
import os

import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _wl(x, y, cfg, rho, vx, vy, p):
    n = len(x)
    f = lambda a: np.broadcast_to(np.asarray(a, float), (n,)).copy()
    return dict(cfg=cfg, x=f(x), y=f(y), rho=f(rho), vx=f(vx), vy=f(vy), p=f(p))


def test_gradient_exact_for_linear_fields(oracle):
    """Eq. 1 (with r_ij pointing from i to j) reproduces the gradient of a
    linear field exactly on every closed cell: sum_j L_ij c_ij.t_ij = 0 and
    sum_j L_ij n_ij = 0 make the correction terms vanish."""
    rng = np.random.default_rng(3)
    n = 400
    x, y = rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    g = {"rho": (0.3, -0.2), "vx": (0.05, 0.07), "vy": (-0.04, 0.02), "p": (0.4, 0.1)}
    base = {"rho": 2.0, "vx": 0.1, "vy": -0.1, "p": 3.0}
    f = {k: base[k] + g[k][0] * x + g[k][1] * y for k in g}
    cfg = W.default_cfg(boundary=W.BC_REFLECTIVE, limiter=W.LIM_AREPO)
    s = oracle.Sim(_wl(x, y, cfg, f["rho"], f["vx"], f["vy"], f["p"]))
    ptr, nb = s.rings()
    interior = np.array([np.all(nb[ptr[i]:ptr[i + 1]] < n) for i in range(n)])
    assert interior.sum() > 250
    s.sweep()
    for v, k in enumerate(("rho", "vx", "vy", "p")):
        gx, gy = s.field("grad", 2 * v)[interior], s.field("grad", 2 * v + 1)[interior]
        np.testing.assert_allclose(gx, g[k][0], atol=1e-11)
        np.testing.assert_allclose(gy, g[k][1], atol=1e-11)


def test_gradient_of_constant_is_zero(oracle):
    wl = W.uniform(n_side=12, jitter=0.3)
    s = oracle.Sim(wl)
    s.sweep()
    for c in range(8):
        assert np.max(np.abs(s.field("grad", c))) < 1e-12


def test_gradient_square_lattice_central_difference(oracle):
    nx, ny = 8, 4
    x = (np.tile(np.arange(nx), ny) + 0.5)
    y = (np.repeat(np.arange(ny), nx) + 0.5)
    col = np.tile(np.arange(nx), ny)
    rho = 10.0 + col ** 2 * 0.5
    cfg = W.default_cfg(boundary=W.BC_PERIODIC, x0=0, x1=nx, y0=0, y1=ny, limiter=W.LIM_AREPO)
    s = oracle.Sim(_wl(x, y, cfg, rho, 0, 0, 1.0))
    s.sweep()
    gx = s.field("grad", 0)
    east = 10.0 + ((col + 1) % nx) ** 2 * 0.5
    west = 10.0 + ((col - 1) % nx) ** 2 * 0.5
    np.testing.assert_allclose(gx, (east - west) / 2.0, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(s.field("grad", 1), 0.0, atol=1e-14)


def _read_golden():
    out = {}
    with open(os.path.join(GOLDEN, "limiter_tvd_example.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            out[tok[0]] = tok[1:]
    return out


@pytest.mark.parametrize("mode", ["arepo", "tess_theta_0.5"])
def test_limiter_worked_example(oracle, mode):
    """Section 2.2's four cells 0, 1, 3, 7 laid out as lattice columns."""
    gold = _read_golden()
    vals = [float(v) for v in gold["values"]]
    exp = gold[mode]
    right2, left3 = float(exp[1]), float(exp[3])
    nx, ny = 8, 4
    col = np.tile(np.arange(nx), ny)
    x = col + 0.5
    y = np.repeat(np.arange(ny), nx) + 0.5
    colvals = np.array(vals + vals[::-1])  # 0 1 3 7 7 3 1 0
    off = 10.0
    rho = off + colvals[col]
    lim = W.LIM_AREPO if mode == "arepo" else W.LIM_TESS
    cfg = W.default_cfg(boundary=W.BC_PERIODIC, x0=0, x1=nx, y0=0, y1=ny, limiter=lim, theta=0.5)
    s = oracle.Sim(_wl(x, y, cfg, rho, 0, 0, 1.0))
    s.sweep()
    gx = s.field("lgrad", 0)
    c2 = (col == 1)  # holds the value 1 ("cell #2")
    c3 = (col == 2)  # holds the value 3 ("cell #3")
    face_r2 = colvals[1] + gx[c2] * 0.5
    face_l3 = colvals[2] - gx[c3] * 0.5
    np.testing.assert_allclose(face_r2, right2, rtol=1e-13)
    np.testing.assert_allclose(face_l3, left3, rtol=1e-13)
    if mode == "arepo":
        assert np.all(face_r2 > face_l3)  # the TVD violation
    else:
        assert np.all(face_r2 <= face_l3)


def test_limiter_alpha_in_unit_interval_and_bounds(oracle):
    wl = W.random_mixed(n=600, seed=21)
    wl["cfg"]["limiter"] = W.LIM_AREPO
    s = oracle.Sim(wl)
    s.sweep()
    for v in range(4):
        a = s.field("alpha", v)
        assert np.all(a >= 0) and np.all(a <= 1)
    assert np.any(s.field("alpha", 0) < 1)


def test_shock_switch_fires_on_pressure_jump(oracle):
    wl = W.sod(n_side=16)
    s = oracle.Sim(wl)
    s.sweep()
    tess = s.field("tess").astype(bool)
    x = wl["x"]
    assert tess[np.abs(x - 0.5) < 0.05].all()      # ratio 0.1 < delta_p at the jump
    assert not tess[np.abs(x - 0.5) > 0.2].any()   # smooth, at rest elsewhere


def test_lloyd_velocity_closed_form(oracle):
    """Section 6: a generator displaced by more than eta*R from its centre of
    mass gets the extra velocity chi*c_s towards it; below the threshold w = v."""
    n_side = 8
    h = 1.0 / n_side
    ii, jj = np.meshgrid(np.arange(n_side), np.arange(n_side))
    x = ((ii + 0.5) * h).ravel()
    y = ((jj + 0.5) * h).ravel()
    k = 3 * n_side + 4
    gamma, rho, p, v = 1.4, 1.3, 0.8, (0.2, -0.1)
    cs = math.sqrt(gamma * p / rho)
    R = math.sqrt(h * h / math.pi)
    for disp, fires in ((0.1 * h, True), (0.005 * h, False)):
        xd = x.copy()
        xd[k] += disp
        cfg = W.default_cfg(gamma=gamma, boundary=W.BC_PERIODIC, chi=0.15, eta=0.02)
        s = oracle.Sim(_wl(xd, y, cfg, rho, v[0], v[1], p))
        s.sweep()
        wx, wy = s.field("wx"), s.field("wy")
        if fires:
            assert disp > 0.02 * R
            np.testing.assert_allclose(wx[k], v[0] - 0.15 * cs, rtol=1e-13)
            np.testing.assert_allclose(wy[k], v[1], atol=1e-14)
        else:
            assert disp < 0.02 * R
            assert wx[k] == v[0] and wy[k] == v[1]
        others = np.ones(len(x), bool)
        others[k] = False
        # neighbours of the displaced cell see their centres move too; far cells stay at w = v
        far = (np.abs(xd - xd[k]) > 2.5 * h) & (np.abs(y - y[k]) > 2.5 * h)
        np.testing.assert_allclose(wx[far], v[0], atol=1e-14)
