"""Oracle pins for the Voronoi geometry named under Eq. 1 (areas, centres of
mass) and for the ghost construction at reflecting and periodic boundaries."""
import math

import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W
from tests import clip_ref


def _sim(oracle, x, y, cfg, rho=1.0, p=1.0):
    n = len(x)
    wl = dict(cfg=cfg, x=np.asarray(x, float), y=np.asarray(y, float), rho=np.full(n, rho),
              vx=np.zeros(n), vy=np.zeros(n), p=np.full(n, p))
    return oracle.Sim(wl)


@pytest.mark.parametrize("boundary", [W.BC_REFLECTIVE, W.BC_PERIODIC])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cells_match_half_plane_clipping(oracle, boundary, seed):
    rng = np.random.default_rng(100 + seed)
    n = 40
    x, y = rng.random(n), rng.random(n)
    cfg = W.default_cfg(boundary=boundary)
    s = _sim(oracle, x, y, cfg)
    pr = s.primitives()
    ref = clip_ref.voronoi_cells(x, y, (0, 1, 0, 1), boundary == W.BC_PERIODIC)
    np.testing.assert_allclose(pr["area"], ref[:, 0], rtol=1e-11, atol=0)
    cx, cy = s.field("cx"), s.field("cy")
    if boundary == W.BC_PERIODIC:  # centres of mass compare modulo the period
        cx = ref[:, 1] + ((cx - ref[:, 1] + 0.5) % 1.0 - 0.5)
        cy = ref[:, 2] + ((cy - ref[:, 2] + 0.5) % 1.0 - 0.5)
    np.testing.assert_allclose(cx, ref[:, 1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(cy, ref[:, 2], rtol=0, atol=1e-12)


@pytest.mark.parametrize("boundary", [W.BC_REFLECTIVE, W.BC_PERIODIC])
def test_areas_sum_to_domain(oracle, boundary):
    rng = np.random.default_rng(7)
    n = 3000
    cfg = W.default_cfg(boundary=boundary, x0=-0.5, x1=0.5, y0=-1.0, y1=0.25)
    x = rng.uniform(-0.5, 0.5, n)
    y = rng.uniform(-1.0, 0.25, n)
    s = _sim(oracle, x, y, cfg)
    A = s.primitives()["area"]
    assert np.all(A > 0)
    assert abs(A.sum() - 1.25) < 1e-13 * 1.25 * 10


def test_square_lattice_closed_form(oracle):
    # unjittered lattice: every cell is an h x h square centred on its generator
    wl = W.advection(n_side=8)
    s = oracle.Sim(wl)
    pr = s.primitives()
    h = 1.0 / 8
    np.testing.assert_allclose(pr["area"], h * h, rtol=1e-14)
    np.testing.assert_allclose(s.field("cx"), wl["x"], atol=1e-15)
    np.testing.assert_allclose(s.field("cy"), wl["y"], atol=1e-15)


def test_hexagonal_lattice_closed_form(oracle):
    nx, ny = 8, 10
    h = 0.125
    Lx, Ly = nx * h, ny * h * math.sqrt(3) / 2
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    x = (ii + 0.25 + 0.5 * (jj % 2)) * h
    y = (jj + 0.5) * h * math.sqrt(3) / 2
    cfg = W.default_cfg(boundary=W.BC_PERIODIC, x0=0, x1=Lx, y0=0, y1=Ly)
    s = _sim(oracle, x.ravel(), y.ravel(), cfg)
    A = s.primitives()["area"]
    np.testing.assert_allclose(A, math.sqrt(3) / 2 * h * h, rtol=1e-13)


def test_reflective_cell_at_wall_is_clipped_by_wall(oracle):
    # three points: every cell is the box clipped by the bisectors
    x = np.array([0.2, 0.7, 0.45])
    y = np.array([0.3, 0.25, 0.8])
    cfg = W.default_cfg(boundary=W.BC_REFLECTIVE)
    s = _sim(oracle, x, y, cfg)
    A = s.primitives()["area"]
    ref = clip_ref.voronoi_cells(x, y, (0, 1, 0, 1), False)
    np.testing.assert_allclose(A, ref[:, 0], rtol=1e-12)
