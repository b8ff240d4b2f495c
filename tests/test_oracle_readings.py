"""Pins of two readings the oracle takes where the paper is silent.

Courant time step (Section 2.3 prints only the Courant number): read as
dt = cfl * min_i R_i / (c_i + |v_i - w_i|) with R_i = sqrt(A_i / pi).  On an
unjittered square lattice every cell is a square of side h whose centre of
mass is its generator, so R = h / sqrt(pi), the rounding velocity is off
(w = v with a moving mesh, w = 0 with a static one), and the time step has
a closed form in the fields of the slowest cell.

Limiter neighbours (Eqs. 3-8): the cells sharing a Voronoi edge of positive
length.  On a square lattice every four generators are co-circular; the
Delaunay triangulation picks one diagonal per square (by the symbolic
tie-break), the Voronoi diagram has none.  Mirroring a field across the
lattice's symmetry axis keeps the points and so the diagonals, but mirrors
the cells around each generator: a limiter that looked at the diagonal
(zero-length edge) neighbours would give results that are not the mirror
images of each other.

Each reading also comes with planted mistakes that must fail its pin.
"""
import math

import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W
from planted import build_planted


def lattice(n, box=1.0):
    h = box / n
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    return ((ii + 0.5) * h).ravel(), ((jj + 0.5) * h).ravel(), h


def _wl(x, y, cfg, rho, vx, vy, p):
    n = len(x)
    f = lambda a: np.broadcast_to(np.asarray(a, float), (n,)).copy()
    return dict(cfg=cfg, x=f(x), y=f(y), rho=f(rho), vx=f(vx), vy=f(vy), p=f(p))


def courant_cases():
    """(workload, expected dt, t_end) cases with closed-form time steps."""
    n, gamma, cfl = 8, 1.4, 0.3
    x, y, h = lattice(n)
    R = h / math.sqrt(math.pi)
    hot = 3 * n + 5
    rho = np.full(n * n, 1.2)
    p = np.full(n * n, 0.7)
    p[hot] = 4.0  # the slowest cell
    v = (0.35, -0.6)
    c_hot = math.sqrt(gamma * p[hot] / rho[hot])
    out = []
    for motion, speed in ((W.MESH_EULERIAN, c_hot + math.hypot(*v)), (W.MESH_LAGRANGIAN, c_hot)):
        cfg = W.default_cfg(gamma=gamma, cfl=cfl, boundary=W.BC_PERIODIC, motion=motion)
        dt = cfl * R / speed
        out.append((_wl(x, y, cfg, rho, v[0], v[1], p), dt, np.inf))
        # a step that would overshoot t_end lands on it
        out.append((_wl(x, y, cfg, rho, v[0], v[1], p), 0.25 * dt, 0.25 * dt))
    return out


def pin_courant(O, L=None):
    for wl, dt, t_end in courant_cases():
        s = O.Sim(wl) if L is None else PlantedSim(O, L, wl)
        got = s.sweep(t_end)
        s.close()
        if not abs(got - dt) <= 1e-14 * dt:
            return False
    return True


def mirrored_limiter_fields(O, L=None):
    """Limited gradients of a random field and of its mirror image x -> n - x
    on an n x n lattice of unit spacing (points at half-integers, so the
    mirror maps the point set onto itself exactly)."""
    n = 10
    x, y, _ = lattice(n, box=float(n))
    rng = np.random.default_rng(17)
    f = {k: rng.uniform(lo, hi, n * n) for k, lo, hi in
         (("rho", 0.5, 2.0), ("vx", -0.5, 0.5), ("vy", -0.5, 0.5), ("p", 0.6, 1.0))}
    col, row = (x - 0.5).astype(int), (y - 0.5).astype(int)
    mirror = row * n + (n - 1 - col)  # cell holding the mirror image of each cell
    res = []
    for lim in (W.LIM_AREPO, W.LIM_SWITCHED):
        cfg = W.default_cfg(boundary=W.BC_PERIODIC, x0=0, x1=n, y0=0, y1=n, limiter=lim, motion=W.MESH_EULERIAN)
        a = _wl(x, y, cfg, f["rho"], f["vx"], f["vy"], f["p"])
        b = _wl(x, y, cfg, f["rho"][mirror], -f["vx"][mirror], f["vy"][mirror], f["p"][mirror])
        out = []
        for wl in (a, b):
            s = O.Sim(wl) if L is None else PlantedSim(O, L, wl)
            s.sweep()
            out.append(np.stack([s.field("lgrad", c) for c in range(8)]))
            s.close()
        res.append((out[0], out[1], mirror))
    return res


def pin_point_contacts(O, L=None):
    """The mirrored field's limited gradient is the mirror image of the
    original's: d/dx flips sign for rho, vy and p, d/dy for vx."""
    sign = np.array([-1, 1, 1, -1, -1, 1, -1, 1])[:, None]
    for ga, gb, mirror in mirrored_limiter_fields(O, L):
        scale = np.max(np.abs(ga))
        if not np.max(np.abs(gb[:, mirror] - sign * ga)) <= 1e-12 * scale:
            return False
    return True


class PlantedSim:
    """Minimal stand-in for oracle.Sim on a planted copy of the library."""

    def __init__(self, O, L, wl):
        import ctypes as C
        self.O, self.L, self.n = O, L, len(wl["x"])
        self.cfg = O.Config.from_dict(wl["cfg"])
        arrs = [np.ascontiguousarray(wl[k], dtype=np.float64) for k in ("x", "y", "rho", "vx", "vy", "p")]
        self.h = C.c_void_p()
        rc = L.orc_create(C.byref(self.cfg), self.n, *[a.ctypes.data_as(O._D) for a in arrs], C.byref(self.h))
        assert rc == 0

    def sweep(self, t_end=np.inf):
        import ctypes as C
        dt = C.c_double()
        assert self.L.orc_sweep(self.h, t_end, C.byref(dt)) == 0
        return dt.value

    def field(self, name, comp=0):
        out = np.zeros(self.n)
        assert self.L.orc_get_cells(self.h, self.O.FIELDS[name] + comp, out.ctypes.data_as(self.O._D)) == 0
        return out

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None


def test_courant_closed_form(oracle):
    assert pin_courant(oracle)


def test_point_contacts_do_not_enter_the_limiter(oracle):
    assert pin_point_contacts(oracle)
    # the case is not vacuous: limiting is active and the diagonals carry
    # zero-length edges
    ga = mirrored_limiter_fields(oracle)[0][0]
    s = oracle.Sim(_wl(*lattice(10, 10.0)[:2], W.default_cfg(boundary=W.BC_PERIODIC, x0=0, x1=10, y0=0, y1=10),
                       1.0, 0.0, 0.0, 1.0))
    ptr, nb = s.rings()
    assert np.all(np.diff(ptr) > 4)  # every cell has more Delaunay neighbours than Voronoi edges
    s.close()
    assert np.any(np.abs(ga) > 0)


COURANT_MISTAKES = [
    ("R = sqrt(A)", "double R = sqrt(s->A[i] / M_PI);\n            double rel",
     "double R = sqrt(s->A[i]);\n            double rel"),
    ("|v| instead of |v - w|", "hypot(s->W[4 * i + 1] - s->wx[i], s->W[4 * i + 2] - s->wy[i])",
     "hypot(s->W[4 * i + 1], s->W[4 * i + 2])"),
    ("sound speed dropped", "double d = R / (s->cs[i] + rel);", "double d = R / (rel + 1e-300);"),
    ("Courant number dropped", "dt *= c->cfl;", "dt *= 1.0;"),
    ("no landing on t_end", "if (s->t + dt > t_end) dt = t_end - s->t;", ""),
]


@pytest.mark.parametrize("name,old,new", COURANT_MISTAKES, ids=[m[0] for m in COURANT_MISTAKES])
def test_courant_planted_mistake_fails(oracle, tmp_path, name, old, new):
    L = oracle.load(build_planted(tmp_path, old, new, within="static int sweep_pass("))
    assert not pin_courant(oracle, L), name


def test_point_contact_cut_removed_fails(oracle, tmp_path):
    L = oracle.load(build_planted(tmp_path, "double Lmin = 1e-9 * sqrt(s->A[i]);", "double Lmin = -1.0;",
                                  within="static int sweep_pass("))
    assert not pin_point_contacts(oracle, L)
