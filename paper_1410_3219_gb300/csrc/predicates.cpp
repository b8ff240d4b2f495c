// Exact orientation / in-circle predicates (see predicates.h).
//
// Fast path (inline, in the header): the determinant in plain double
// arithmetic with a forward error bound proportional to its "permanent" (the
// same sum with absolute values).
//
// Exact path: non-overlapping floating-point expansions.  TwoSum (Knuth) and
// an FMA-based TwoProduct give exact sums and products of two doubles as
// two-component expansions; GrowExpansion adds a double to an expansion
// exactly, keeping the components non-overlapping and increasing in
// magnitude, so the sign of an expansion is the sign of its last non-zero
// component.  Expansions live in fixed arrays on the stack (nothing is
// allocated on the exact path, which the mirror images of a walled box reach
// at every wall-side edge: a point, its neighbour along the wall and their
// two images are co-circular up to the rounding of the images).  This file
// must be compiled without floating-point contraction.
#include "predicates.h"

#include <cmath>

namespace rich {
namespace {

// An expansion in a caller-provided array: components non-overlapping and
// increasing in magnitude, zero components dropped (the value zero is the
// single component 0).  Every routine writes into storage of its own; the
// bounds on the lengths below follow from the operations of the in-circle
// determinant, whose inputs are the two-component coordinate differences.

inline void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    double bv = s - a;
    double av = s - bv;
    e = (a - av) + (b - bv);
}

inline void two_prod(double a, double b, double &p, double &e)
{
    p = a * b;
    e = std::fma(a, b, -p);
}

// h[0, n) += b exactly, in place (room for n + 1); returns the new length.
// Component i is read before anything is written at or beyond it.
inline int grow(double *h, int n, double b)
{
    double q = b;
    int k = 0;
    for (int i = 0; i < n; i++) {
        double s, err;
        two_sum(q, h[i], s, err);
        if (err != 0.0) h[k++] = err;
        q = s;
    }
    if (q != 0.0 || k == 0) h[k++] = q;
    return k;
}

// h = e + f (room for ne + nf)
inline int add(const double *e, int ne, const double *f, int nf, double *h)
{
    for (int i = 0; i < ne; i++) h[i] = e[i];
    int n = ne;
    for (int j = 0; j < nf; j++) n = grow(h, n, f[j]);
    return n;
}

// h = e * b (room for 2 ne + 1)
inline int scale(const double *e, int ne, double b, double *h)
{
    h[0] = 0.0;
    int n = 1;
    for (int i = 0; i < ne; i++) {
        double p, err;
        two_prod(e[i], b, p, err);
        n = grow(h, n, err);
        n = grow(h, n, p);
    }
    return n;
}

// h = e * f (room for 2 ne nf + 1; t: scratch of 2 ne + 1)
inline int mul(const double *e, int ne, const double *f, int nf, double *h, double *t)
{
    h[0] = 0.0;
    int n = 1;
    for (int j = 0; j < nf; j++) {
        const int nt = scale(e, ne, f[j], t);
        for (int i = 0; i < nt; i++) n = grow(h, n, t[i]);
    }
    return n;
}

inline int negate(double *e, int n)
{
    for (int i = 0; i < n; i++) e[i] = -e[i];
    return n;
}

// a - b as one component when the difference is exact, else two
inline int diff(double a, double b, double *h)
{
    double s, e;
    two_sum(a, -b, s, e);
    if (e == 0.0) {
        h[0] = s;
        return 1;
    }
    h[0] = e;
    h[1] = s;
    return 2;
}

inline int sign_of(const double *e, int n)
{
    for (int i = n - 1; i >= 0; i--)
        if (e[i] != 0.0) return e[i] > 0.0 ? 1 : -1;
    return 0;
}

// A coordinate difference: one or two components.
struct Diff {
    double v[2];
    int n;
    Diff(double a, double b) { n = diff(a, b, v); }
};

// x*y - z*w (room for 2 * 8)
inline int cross(const Diff &x, const Diff &y, const Diff &z, const Diff &w, double *h)
{
    double a[9], b[9], t[5];
    const int na = mul(x.v, x.n, y.v, y.n, a, t);
    const int nb = negate(b, mul(z.v, z.n, w.v, w.n, b, t));
    return add(a, na, b, nb, h);
}

// x*x + y*y (room for 2 * 8)
inline int norm2(const Diff &x, const Diff &y, double *h)
{
    double a[9], b[9], t[5];
    const int na = mul(x.v, x.n, x.v, x.n, a, t);
    const int nb = mul(y.v, y.n, y.v, y.n, b, t);
    return add(a, na, b, nb, h);
}

}  // namespace

int orient2d_exact(double ax, double ay, double bx, double by, double cx, double cy)
{
    const Diff bax(bx, ax), cay(cy, ay), bay(by, ay), cax(cx, ax);
    double h[18];
    return sign_of(h, cross(bax, cay, bay, cax, h));
}

int incircle_exact(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy)
{
    const Diff adx(ax, dx), ady(ay, dy), bdx(bx, dx), bdy(by, dy), cdx(cx, dx), cdy(cy, dy);
    // lifted heights (up to 18 components) times the 2x2 minors (up to 18)
    double la[18], lb[18], lc[18], ma[18], mb[18], mc[18];
    const int nla = norm2(adx, ady, la), nlb = norm2(bdx, bdy, lb), nlc = norm2(cdx, cdy, lc);
    const int nma = cross(bdx, cdy, cdx, bdy, ma);
    const int nmb = cross(cdx, ady, adx, cdy, mb);
    const int nmc = cross(adx, bdy, bdx, ady, mc);
    // products up to 2 * 18 * 18 + 1 = 649 components, their sum up to 1947
    double t[37], pa[649], pb[649], pc[649], det[1947];
    const int npa = mul(la, nla, ma, nma, pa, t);
    const int npb = mul(lb, nlb, mb, nmb, pb, t);
    const int npc = mul(lc, nlc, mc, nmc, pc, t);
    int n = add(pa, npa, pb, npb, det);
    for (int i = 0; i < npc; i++) n = grow(det, n, pc[i]);
    return sign_of(det, n);
}

namespace {

inline bool lex_less(double px, double py, double qx, double qy)
{
    return px < qx || (px == qx && py < qy);
}

}  // namespace

int incircle_tiebreak(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy)
{
    // First-order change of the lifting determinant when each height |p|^2
    // grows by d_p:  d_a*orient(b,c,d) - d_b*orient(a,c,d) + d_c*orient(a,b,d)
    // - d_d*orient(a,b,c).  The lexicographically smallest point dominates.
    int k = 0;
    double mx = ax, my = ay;
    if (lex_less(bx, by, mx, my)) { k = 1; mx = bx; my = by; }
    if (lex_less(cx, cy, mx, my)) { k = 2; mx = cx; my = cy; }
    if (lex_less(dx, dy, mx, my)) { k = 3; }
    switch (k) {
    case 0: return orient2d(bx, by, cx, cy, dx, dy);
    case 1: return -orient2d(ax, ay, cx, cy, dx, dy);
    case 2: return orient2d(ax, ay, bx, by, dx, dy);
    default: return -orient2d(ax, ay, bx, by, cx, cy);
    }
}

}  // namespace rich
