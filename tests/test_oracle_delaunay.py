"""Oracle pins for the tessellation of Section 2.1: the point-insertion
Delaunay triangulation against an O(n^4) exact brute force, Euler's formula,
degenerate lattices and duplicate detection."""
import itertools

import numpy as np
import pytest

from tests import exact_ref as X


def hull_points(pts):
    """Input points on the convex hull boundary (collinear ones included)."""
    pts = sorted(set(pts))
    def half(seq):
        h = []
        for p in seq:
            while len(h) >= 2 and X.orient(h[-2], h[-1], p) < 0:
                h.pop()
            h.append(p)
        return h
    lower, upper = half(pts), half(reversed(pts))
    return set(lower[:-1] + upper[:-1])


def brute_delaunay(pts):
    """All counter-clockwise triangles whose tie-broken circumcircle is empty."""
    out = set()
    n = len(pts)
    for a, b, c in itertools.combinations(range(n), 3):
        if X.orient(pts[a], pts[b], pts[c]) == 0:
            continue
        if X.orient(pts[a], pts[b], pts[c]) < 0:
            b, c = c, b
        if all(X.incircle_perturbed(pts[a], pts[b], pts[c], pts[d]) < 0 for d in range(n) if d not in (a, b, c)):
            out.add(frozenset((a, b, c)))
    return out


CASES = {
    "random": lambda rng: [tuple(v) for v in rng.integers(0, 256, (11, 2)) / 64.0],
    "lattice": lambda rng: [(i * 0.5, j * 0.5) for i in range(4) for j in range(3)],
    "cocircular": lambda rng: [(1 + np.cos(t), 1 + np.sin(t)) for t in np.linspace(0, 2 * np.pi, 9)[:-1]]
                              + [(0.25, 0.25), (1.0, 1.0)],
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_delaunay_matches_brute_force(oracle, case, seed):
    rng = np.random.default_rng(seed)
    pts = CASES[case](rng)
    pts = list(dict.fromkeys(pts))  # distinct
    n = len(pts)
    x = np.array([p[0] for p in pts])
    y = np.array([p[1] for p in pts])
    tris = oracle.delaunay(x, y)
    real = {frozenset(t) for t in tris.tolist() if max(t) < n}
    brute = brute_delaunay(pts)
    # every triangle among input points is a Delaunay triangle
    assert real <= brute
    # Euler: a triangulation of n points with h on the hull has 2n - h - 2 triangles
    hull = hull_points(pts)
    assert len(brute) == 2 * n - len(hull) - 2
    # triangles the finite enclosing construction may hide have an edge on the hull
    for t in brute - real:
        assert sum(pts[k] in hull for k in t) >= 2
    # every output triangle is counter-clockwise
    for t in tris.tolist():
        if max(t) < n:
            assert X.orient(pts[t[0]], pts[t[1]], pts[t[2]]) > 0


def test_insertion_order_independent(oracle):
    rng = np.random.default_rng(5)
    x = np.repeat(np.arange(6) * 0.25, 5)
    y = np.tile(np.arange(5) * 0.25, 6)
    base = {frozenset(t) for t in oracle.delaunay(x, y).tolist() if max(t) < len(x)}
    for _ in range(4):
        perm = rng.permutation(len(x))
        tr = oracle.delaunay(x[perm], y[perm])
        got = {frozenset(perm[list(t)]) for t in tr.tolist() if max(t) < len(x)}
        assert got == base


def test_duplicate_rejected(oracle):
    x = np.array([0.1, 0.5, 0.9, 0.5])
    y = np.array([0.1, 0.8, 0.2, 0.8])
    with pytest.raises(ValueError):
        oracle.delaunay(x, y)


def test_euler_large_random(oracle):
    rng = np.random.default_rng(9)
    n = 2000
    x, y = rng.random(n), rng.random(n)
    tris = oracle.delaunay(x, y)
    real = [t for t in tris.tolist() if max(t) < n]
    # the enclosing triangle is far away, so only hull triangles can be hidden:
    # interior count is bounded by Euler and close to 2n
    assert len(real) <= 2 * n - 3 - 2
    assert len(real) > 2 * n - 5 * int(np.sqrt(n))
