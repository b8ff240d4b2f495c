"""CPU tests of the C-ABI library: it loads without a GPU, exports every
entry point of include/rich.h, and its host tessellation (Section 2.1: exact,
tie-broken Delaunay, ghost images, Voronoi rings) agrees with the oracle's
independent construction.  No device call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1410_3219_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1410_3219_gb300 import rich
    rich.lib()
    return rich


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rich.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rich_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(R):
    lib = ctypes.CDLL(R.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(R.EXPORTS) == names


def test_strerror_and_defaults(R):
    L = R.lib()
    assert L.rich_strerror(0) == b"ok"
    assert b"duplicate" in L.rich_strerror(-2) or b"coincident" in L.rich_strerror(-2)
    c = R.rich_config()
    L.rich_default_config(ctypes.byref(c))
    assert c.cfl == 0.3 and c.theta == 0.5 and c.delta_v == 0.2 and c.delta_p == 0.7
    assert c.chi == 0.15 and c.eta == 0.02


def _canon(tris, n):
    return {frozenset(t) for t in np.asarray(tris).tolist() if max(t) < n}


@pytest.mark.parametrize("kind", ["random", "lattice", "near_lattice", "mirrored"])
def test_host_delaunay_matches_oracle(R, oracle, kind):
    rng = np.random.default_rng(4)
    if kind == "random":
        x, y = rng.random(3000), rng.random(3000)
    elif kind == "lattice":
        x, y = [a.ravel() * 0.125 for a in np.meshgrid(np.arange(20), np.arange(17))]
    elif kind == "mirrored":
        # points beside a wall at x = 0.3 and their mirror images (w + w) - x,
        # as the ghosts of a walled box are made: every point, a neighbour
        # along the wall and their two images are co-circular up to the
        # rounding of the images, so the exact in-circle path and the
        # tie-break decide the triangulation along the wall
        w = 0.3
        px, py = w + rng.random(1500) * 0.05, rng.random(1500)
        x, y = np.concatenate([px, (w + w) - px]), np.concatenate([py, py])
    else:
        x, y = [a.ravel() * 0.125 + rng.uniform(-1, 1, a.size) * 1e-14 for a in np.meshgrid(np.arange(20), np.arange(17))]
    n = len(x)
    mine = R.rich_delaunay_host(x, y)
    ref = oracle.delaunay(x, y)
    a, b = _canon(mine, n), _canon(ref, n)
    # both enclose the points with different auxiliary triangles, so only hull
    # triangles may differ; every interior point has the same star
    assert len(a & b) >= len(b) - 4 * int(np.sqrt(n)) - 10
    touched = {v for t in a ^ b for v in t}
    interior_same = [v for v in range(n) if v not in touched]
    assert len(interior_same) > 0.8 * n
    if kind == "mirrored":
        # away from the hull, along the wall, the two agree triangle for triangle
        near = lambda t: all(abs(x[v] - 0.3) < 0.02 and 0.05 < y[v] < 0.95 for v in t)
        assert {t for t in a if near(t)} == {t for t in b if near(t)}


def test_host_delaunay_duplicate(R):
    with pytest.raises(R.RichError) as e:
        R.rich_delaunay_host(np.array([0.1, 0.5, 0.9, 0.1]), np.array([0.2, 0.6, 0.2, 0.2]))
    assert e.value.code == -2


def _canonical_rings(ptr, ids):
    """Rings as one array of neighbour ids, each ring rotated to start at its
    smallest id (the cyclic counter-clockwise order is kept)."""
    ptr = np.asarray(ptr, np.int64)
    deg = np.diff(ptr)
    cell = np.repeat(np.arange(len(deg)), deg)
    pos = np.arange(ptr[-1]) - ptr[cell]
    mins = np.minimum.reduceat(ids, ptr[:-1])
    # position of the minimum in each ring
    first = np.full(len(deg), np.iinfo(np.int64).min, np.int64)
    hit = ids == mins[cell]
    np.maximum.at(first, cell[hit], -pos[hit])
    start = -first
    return ids[ptr[cell] + (pos + start[cell]) % deg[cell]]


WORKLOADS = {
    "sod": lambda: W.sod(n_side=24),
    "sedov": lambda: W.sedov(n=3000),
    "kh": lambda: W.kelvin_helmholtz(n_side=24),
    "gresho": lambda: W.gresho(n_side=20),
    "lattice": lambda: W.advection(n_side=12),
    "random_reflective": lambda: W.random_mixed(n=700),
    # large enough for the slab-parallel builder to cut the points into
    # several slabs (one per host thread, at least 16384 points each); the
    # unjittered lattice is fully co-circular, so every slab must break the
    # ties exactly as the whole set does
    "sedov_slabs": lambda: W.sedov(n=70000),
    "kh_slabs": lambda: W.kelvin_helmholtz(n_side=260),
    "lattice_slabs": lambda: W.advection(n_side=260),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_rings_match_oracle(R, oracle, name):
    """Every real cell has the same counter-clockwise neighbour ring (as
    positions, ghosts included) in the library and in the oracle."""
    wl = WORKLOADS[name]()
    ptr, nbx, nby, src = R.rich_rings_host(wl["cfg"], wl["x"], wl["y"])
    s = oracle.Sim(wl)
    X, Y, S = s.points()
    optr, onb = s.rings()
    # neighbours named by their position (ghost images are computed the same
    # way on both sides, so equal points are bit-identical)
    pts = np.concatenate([np.stack([nbx, nby], 1), np.stack([X[onb], Y[onb]], 1)])
    _, ids = np.unique(pts, axis=0, return_inverse=True)
    ids = ids.ravel()
    mine = _canonical_rings(ptr, ids[: len(nbx)])
    theirs = _canonical_rings(optr, ids[len(nbx):])
    assert np.array_equal(np.asarray(ptr), np.asarray(optr))
    assert np.array_equal(mine, theirs)
    # neighbour source cells agree too
    assert np.array_equal(np.sort(src), np.sort(S[onb]))


def test_rings_reject_bad_input(R):
    cfg = W.default_cfg(boundary=W.BC_REFLECTIVE)
    with pytest.raises(R.RichError):
        R.rich_rings_host(cfg, np.array([0.1, 0.5, 1.5]), np.array([0.1, 0.5, 0.5]))
    with pytest.raises(R.RichError) as e:
        R.rich_rings_host(cfg, np.array([0.1, 0.5, 0.5, 0.8]), np.array([0.1, 0.5, 0.5, 0.2]))
    assert e.value.code == -2


def test_init_without_gpu_fails_loudly(R):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    wl = W.sod(n_side=8)
    with pytest.raises(R.RichError) as e:
        R.Sim(wl)
    assert e.value.code in (-9, -8)


def _init(R, wl, **over):
    """rich_init_mesh on a workload with fields replaced; returns the code."""
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in wl.items()}
    d["cfg"] = dict(wl["cfg"])
    cfg_fields = {name for name, _ in R.rich_config._fields_}
    for k, v in over.items():
        if k in cfg_fields:
            d["cfg"][k] = v
        else:
            d[k] = v
    try:
        R.Sim(d).close()
        return 0
    except R.RichError as e:
        return e.code


@pytest.mark.parametrize("case", ["too_few", "nan_point", "outside_box", "on_wall", "zero_density",
                                  "negative_pressure", "nan_velocity", "gamma_one", "bad_scheme",
                                  "bad_precision", "bad_limiter", "negative_eta"])
def test_init_rejects_bad_input_before_any_device_call(R, case):
    """Argument checks come first (RICH_EINVAL), so they hold with or without
    a GPU; a valid input then reaches the device check."""
    wl = W.sod(n_side=8)
    x, y = wl["x"].copy(), wl["y"].copy()
    over = {
        "too_few": dict(x=x[:2], y=y[:2], rho=wl["rho"][:2], vx=wl["vx"][:2], vy=wl["vy"][:2], p=wl["p"][:2]),
        "nan_point": dict(x=np.where(np.arange(len(x)) == 5, np.nan, x)),
        "outside_box": dict(x=np.where(np.arange(len(x)) == 5, 1.5, x)),
        "on_wall": dict(x=np.where(np.arange(len(x)) == 5, 0.0, x)),  # rigid walls: strictly inside
        "zero_density": dict(rho=np.where(np.arange(len(x)) == 3, 0.0, wl["rho"])),
        "negative_pressure": dict(p=np.where(np.arange(len(x)) == 3, -1.0, wl["p"])),
        "nan_velocity": dict(vx=np.where(np.arange(len(x)) == 3, np.nan, wl["vx"])),
        "gamma_one": dict(gamma=1.0),
        "bad_scheme": dict(scheme=7),
        "bad_precision": dict(precision=5),
        "bad_limiter": dict(limiter=9),
        "negative_eta": dict(eta=-0.1),
    }[case]
    assert _init(R, wl, **over) == R.RICH_EINVAL


def test_restart_rejects_a_non_permutation_order_on_the_host(R):
    wl = W.sod(n_side=8)
    n = len(wl["x"])
    m = np.full(n, 1.0 / n)
    E = np.full(n, 2.5 / n)
    z = np.zeros(n)
    with pytest.raises(R.RichError) as e:
        R.rich_init_conserved(wl["cfg"], wl["x"], wl["y"], m, z, z, E, 0.0, np.zeros(n, np.int64))
    # the order is checked once a device exists; without one the device check fails first
    assert e.value.code in (R.RICH_EINVAL, R.RICH_ENODEV)


def _positions(oracle, wl, steps, skip=0):
    s = oracle.Sim(wl)
    n = len(wl["x"])
    for _ in range(skip):
        s.step()
    xs, ys = [], []
    for _ in range(steps):
        X, Y, _ = s.points()
        xs.append(X[:n].copy())
        ys.append(Y[:n].copy())
        s.step()
    return np.array(xs), np.array(ys)


@pytest.mark.parametrize("step_cells", [0.02, 0.3, 2.0])
def test_mesh_updates_follow_points_across_grid_buckets(R, step_cells):
    """The host builder keeps its bucketing of the points from build to
    build while they have moved less than half a bucket and rebuilds it
    after: in a periodic shear flow moving every point by up to step_cells
    cell widths a step (buckets are about six cells wide at this size, so
    points cross buckets, and the bucketing is kept for tens of steps, a few
    or none), the sweep's inputs still equal those of fresh builds."""
    # 65,536 points: four tiles on four threads, so that tiles gather
    # their points from the buckets (one tile takes every point)
    wl = W.kelvin_helmholtz(n_side=256, amp=0.1)
    x, y = wl["x"].copy(), wl["y"].copy()
    d = step_cells / 256.0
    xs, ys = [], []
    for k in range(10):
        xs.append(x.copy())
        ys.append(y.copy())
        x = np.mod(x + d * np.sin(2.0 * np.pi * y), 1.0)
        y = np.mod(y + 0.5 * d * np.cos(2.0 * np.pi * x), 1.0)
    mismatched, updated, rebuilt, _ = R.rich_mesh_update_check(wl["cfg"], np.array(xs), np.array(ys), threads=4)
    assert mismatched == 0, (updated, rebuilt)
    assert updated + rebuilt >= 4 * 10


@pytest.mark.parametrize("name,make,steps,skip,turned", [
    ("sod_64", lambda: W.sod(n_side=64), 40, 0, True),
    ("kh_64", lambda: W.kelvin_helmholtz(n_side=64, amp=0.1), 30, 0, True),
    ("gresho_32", lambda: W.gresho(n_side=32), 30, 0, False),
    ("advection_lattice_16", lambda: W.advection(n_side=16), 20, 0, False),
    ("random_mixed_reflective", lambda: W.random_mixed(n=3000, seed=8), 20, 0, False),
    ("sedov_20000", lambda: W.sedov(n=20000, seed=2), 6, 2, False),
    ("kh_200", lambda: W.kelvin_helmholtz(n_side=200, amp=0.1), 4, 0, True),
])
def test_mesh_updated_in_place_equals_fresh(R, oracle, name, make, steps, skip, turned):
    """The host builder keeps each tile's triangulation between steps and
    updates it: moves the vertices (taking out and inserting again those of
    triangles that would turn over), flips to Delaunay, inserts new points.
    Over successive steps of oracle runs (co-circular lattices, mirrored and
    periodic ghosts, one and several tiles) the sweep's inputs equal those
    of fresh builds exactly, and after the first build nearly every tile is
    updated rather than rebuilt."""
    wl = make()
    xs, ys = _positions(oracle, wl, steps, skip)
    for threads in (1, 4):
        mismatched, updated, rebuilt, reinserted = R.rich_mesh_update_check(wl["cfg"], xs, ys, threads=threads)
        assert mismatched == 0, (threads, updated, rebuilt, reinserted)
        tiles = updated + rebuilt
        assert tiles >= steps
        assert updated >= 0.75 * tiles - (tiles // steps), (threads, updated, rebuilt)
        if turned:
            # the runs where triangles would turn over exercise the
            # take-out-and-re-insert path
            assert reinserted > 0, (threads, updated, rebuilt)
