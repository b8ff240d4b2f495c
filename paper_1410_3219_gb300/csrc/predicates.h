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

namespace rich {

// > 0 if a, b, c turn counter-clockwise, < 0 clockwise, 0 collinear.
int orient2d(double ax, double ay, double bx, double by, double cx, double cy);

// Sign of the in-circle determinant for counter-clockwise a, b, c:
// > 0 when d is strictly inside their circumcircle, 0 when co-circular.
int incircle_exact_sign(double ax, double ay, double bx, double by, double cx, double cy,
                        double dx, double dy);

// Same, with the symbolic tie-break: never 0 for distinct points.
int incircle_sos(double ax, double ay, double bx, double by, double cx, double cy,
                 double dx, double dy);

}  // namespace rich
