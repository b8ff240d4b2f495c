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
// component.  This file must be compiled without floating-point contraction.
#include "predicates.h"

#include <cmath>
#include <vector>

namespace rich {
namespace {

using Exp = std::vector<double>;

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

// h = e + b exactly
Exp grow(const Exp &e, double b)
{
    Exp h;
    h.reserve(e.size() + 1);
    double q = b;
    for (double ei : e) {
        double s, err;
        two_sum(q, ei, s, err);
        if (err != 0.0) h.push_back(err);
        q = s;
    }
    if (q != 0.0 || h.empty()) h.push_back(q);
    return h;
}

Exp add(const Exp &e, const Exp &f)
{
    Exp h = e;
    for (double fi : f) h = grow(h, fi);
    return h;
}

Exp neg(Exp e)
{
    for (double &v : e) v = -v;
    return e;
}

Exp scale(const Exp &e, double b)
{
    Exp h{0.0};
    for (double ei : e) {
        double p, err;
        two_prod(ei, b, p, err);
        h = grow(h, err);
        h = grow(h, p);
    }
    return h;
}

Exp mul(const Exp &e, const Exp &f)
{
    Exp h{0.0};
    for (double fi : f) h = add(h, scale(e, fi));
    return h;
}

Exp diff(double a, double b)
{
    double s, e;
    two_sum(a, -b, s, e);
    return Exp{e, s};
}

int sign_of(const Exp &e)
{
    for (auto it = e.rbegin(); it != e.rend(); ++it)
        if (*it != 0.0) return *it > 0.0 ? 1 : -1;
    return 0;
}

}  // namespace

int orient2d_exact(double ax, double ay, double bx, double by, double cx, double cy)
{
    Exp l = mul(diff(bx, ax), diff(cy, ay));
    Exp r = mul(diff(by, ay), diff(cx, ax));
    return sign_of(add(l, neg(r)));
}

int incircle_exact(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy)
{
    Exp adx = diff(ax, dx), ady = diff(ay, dy);
    Exp bdx = diff(bx, dx), bdy = diff(by, dy);
    Exp cdx = diff(cx, dx), cdy = diff(cy, dy);
    Exp la = add(mul(adx, adx), mul(ady, ady));
    Exp lb = add(mul(bdx, bdx), mul(bdy, bdy));
    Exp lc = add(mul(cdx, cdx), mul(cdy, cdy));
    Exp ma = add(mul(bdx, cdy), neg(mul(cdx, bdy)));
    Exp mb = add(mul(cdx, ady), neg(mul(adx, cdy)));
    Exp mc = add(mul(adx, bdy), neg(mul(bdx, ady)));
    Exp det = add(add(mul(la, ma), mul(lb, mb)), mul(lc, mc));
    return sign_of(det);
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
