"""Exact rational reference arithmetic used by the CPU pin tests (Python
Fractions; every double converts to a Fraction exactly).  Independent of both
the oracle and the CUDA library."""
from fractions import Fraction as Fr


def orient(a, b, c):
    ax, ay, bx, by, cx, cy = map(Fr, (*a, *b, *c))
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


def det4_lifted(pts, delta=None):
    """4x4 lifting determinant |x y x^2+y^2+delta_p 1| for the points a,b,c,d."""
    rows = []
    for k, p in enumerate(pts):
        x, y = Fr(p[0]), Fr(p[1])
        z = x * x + y * y + (delta[k] if delta is not None else 0)
        rows.append([x, y, z, Fr(1)])

    def det(m):
        if len(m) == 1:
            return m[0][0]
        s = 0
        for j in range(len(m)):
            if m[0][j] == 0:
                continue
            minor = [r[:j] + r[j + 1:] for r in m[1:]]
            s += (-1) ** j * m[0][j] * det(minor)
        return s

    return det(rows)


def incircle_raw(a, b, c, d):
    v = det4_lifted([a, b, c, d])
    return (v > 0) - (v < 0)


def incircle_perturbed(a, b, c, d, eps=Fr(1, 10 ** 40)):
    """Sign with explicit lifted-height perturbations delta_p = eps**(rank+1),
    rank = lexicographic order of the four points (smallest first)."""
    pts = [a, b, c, d]
    order = sorted(range(4), key=lambda k: (pts[k][0], pts[k][1]))
    delta = [0] * 4
    for r, k in enumerate(order):
        delta[k] = eps ** (r + 1)
    v = det4_lifted(pts, delta)
    return (v > 0) - (v < 0)
