// Exact geometric predicates for the host tessellation (paper Section 2.1:
// the in-circle test must return the exact sign whenever round-off could flip
// it).  A double-precision evaluation is accepted when its magnitude exceeds a
// forward error bound; otherwise the determinant is recomputed exactly with
// floating-point expansion arithmetic (Priest 1991; Shewchuk 1997).
//
// Four exactly co-circular points are resolved by symbolic perturbation of
// the lifted heights |p|^2 (Edelsbrunner & Muecke 1990): point p is lifted by
// an infinitesimal d_p > 0 and the lexicographically smallest point (x, then
// y) carries the dominant perturbation.  The triangulation is then unique for
// any set of distinct points, independent of insertion order.
#pragma once

#include <cmath>

namespace rich {

// The fast paths are inline so that the loops over triangles and edges
// evaluate them without a call; like the exact paths they must be compiled
// without floating-point contraction (every translation unit of the host
// library is).  The bounds are a few times looser than the tight ones of
// Shewchuk (1997), which only sends more near-degenerate cases to the exact
// path.
constexpr double kOrientBound = 1e-15;    // >= (3 + 16 eps) eps
constexpr double kIncircleBound = 1e-14;  // >= (10 + 96 eps) eps

// the exact evaluations (out of line), for when the bound is not met
int orient2d_exact(double ax, double ay, double bx, double by, double cx, double cy);
int incircle_exact(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy);
// the symbolic tie-break of four exactly co-circular points
int incircle_tiebreak(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy);

// > 0 if a, b, c turn counter-clockwise, < 0 clockwise, 0 collinear.
inline int orient2d(double ax, double ay, double bx, double by, double cx, double cy)
{
    const double l = (bx - ax) * (cy - ay);
    const double r = (by - ay) * (cx - ax);
    const double det = l - r;
    const double bound = kOrientBound * (std::fabs(l) + std::fabs(r));
    if (det > bound) return 1;
    if (-det > bound) return -1;
    return orient2d_exact(ax, ay, bx, by, cx, cy);
}

// Sign of the in-circle determinant for counter-clockwise a, b, c:
// > 0 when d is strictly inside their circumcircle, 0 when co-circular.
inline int incircle_exact_sign(double ax, double ay, double bx, double by, double cx, double cy, double dx,
                               double dy)
{
    const double adx = ax - dx, ady = ay - dy, bdx = bx - dx, bdy = by - dy, cdx = cx - dx, cdy = cy - dy;
    const double p1 = bdx * cdy, p2 = cdx * bdy, p3 = cdx * ady, p4 = adx * cdy, p5 = adx * bdy, p6 = bdx * ady;
    const double la = adx * adx + ady * ady, lb = bdx * bdx + bdy * bdy, lc = cdx * cdx + cdy * cdy;
    const double det = la * (p1 - p2) + lb * (p3 - p4) + lc * (p5 - p6);
    const double perm = la * (std::fabs(p1) + std::fabs(p2)) + lb * (std::fabs(p3) + std::fabs(p4)) +
                        lc * (std::fabs(p5) + std::fabs(p6));
    const double bound = kIncircleBound * perm;
    if (std::isfinite(det) && std::isfinite(bound)) {
        if (det > bound) return 1;
        if (-det > bound) return -1;
    }
    return incircle_exact(ax, ay, bx, by, cx, cy, dx, dy);
}

// Same, with the symbolic tie-break: never 0 for distinct points.
inline int incircle_sos(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy)
{
    const int s = incircle_exact_sign(ax, ay, bx, by, cx, cy, dx, dy);
    return s != 0 ? s : incircle_tiebreak(ax, ay, bx, by, cx, cy, dx, dy);
}

}  // namespace rich
