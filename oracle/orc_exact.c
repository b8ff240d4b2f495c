/*
 * ORACLE (test infrastructure only; never linked into the CUDA library).
 *
 * Exact orientation and in-circle predicates for the tessellation step of
 * Section 2.1 of the paper, which asks for the exact sign whenever round-off
 * could flip it.  The paper uses adaptive floating-point arithmetic; this
 * oracle takes a deliberately different, slow and obviously exact route:
 *
 *   1. evaluate the determinant in double precision together with its
 *      "permanent" (the same expression with every term made non-negative);
 *      if |det| exceeds 1e-10 * permanent (about 1e5 times the worst-case
 *      rounding error of the evaluation), its sign is certain;
 *   2. otherwise write every coordinate as an integer times a common power
 *      of two (every double is m * 2^e with a 53-bit integer m) and evaluate
 *      the determinant polynomial in exact big-integer arithmetic.
 *
 * Ties (four exactly co-circular points) are broken by symbolic perturbation
 * of the lifted heights |p|^2: every point p gets |p|^2 + d_p with d_p > 0
 * infinitesimal, and the lexicographically smallest point (x first, then y)
 * carries the dominant perturbation.  This defines one triangulation for any
 * set of distinct points, whatever the insertion order, so two independent
 * builders agree exactly even on lattices.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "orc.h"

#define BN_LIMBS 128 /* 4096 bits: enough for an exponent spread of ~950 bits */

typedef struct {
    int sign; /* -1, 0, +1 */
    int len;  /* limbs in use */
    uint32_t d[BN_LIMBS];
} bn;

static void bn_fail(const char *what)
{
    fprintf(stderr, "oracle bignum overflow in %s (coordinate exponent spread too large)\n", what);
    abort();
}

static void bn_norm(bn *a)
{
    while (a->len > 0 && a->d[a->len - 1] == 0) a->len--;
    if (a->len == 0) a->sign = 0;
}

/* a = v * 2^(-emin), exact (v is m * 2^e with e >= emin). */
static void bn_from_double(bn *a, double v, int emin)
{
    memset(a, 0, sizeof(*a));
    if (v == 0.0) return;
    int e;
    double f = frexp(fabs(v), &e);           /* |v| = f * 2^e, f in [0.5, 1) */
    uint64_t m = (uint64_t)ldexp(f, 53);     /* exact 53-bit integer */
    int shift = (e - 53) - emin;             /* >= 0 by choice of emin */
    int limb = shift / 32, bit = shift % 32;
    if (limb + 3 > BN_LIMBS) bn_fail("from_double");
    /* place m << bit into limbs starting at 'limb' */
    uint32_t lo = (uint32_t)(m & 0xffffffffu), hi = (uint32_t)(m >> 32);
    uint64_t w0 = (uint64_t)lo << bit;
    uint64_t w1 = ((uint64_t)hi << bit) + (w0 >> 32);
    a->d[limb] = (uint32_t)w0;
    a->d[limb + 1] = (uint32_t)w1;
    a->d[limb + 2] = (uint32_t)(w1 >> 32);
    a->len = limb + 3;
    a->sign = v > 0 ? 1 : -1;
    bn_norm(a);
}

static int mag_cmp(const bn *a, const bn *b)
{
    if (a->len != b->len) return a->len > b->len ? 1 : -1;
    for (int i = a->len - 1; i >= 0; i--)
        if (a->d[i] != b->d[i]) return a->d[i] > b->d[i] ? 1 : -1;
    return 0;
}

static void mag_add(bn *r, const bn *a, const bn *b)
{
    int n = a->len > b->len ? a->len : b->len;
    if (n + 1 > BN_LIMBS) bn_fail("add");
    uint64_t carry = 0;
    bn t;
    memset(&t, 0, sizeof(t));
    for (int i = 0; i < n; i++) {
        uint64_t s = carry + (i < a->len ? a->d[i] : 0) + (i < b->len ? b->d[i] : 0);
        t.d[i] = (uint32_t)s;
        carry = s >> 32;
    }
    t.d[n] = (uint32_t)carry;
    t.len = n + 1;
    t.sign = 1;
    *r = t;
}

/* |a| >= |b| required */
static void mag_sub(bn *r, const bn *a, const bn *b)
{
    bn t;
    memset(&t, 0, sizeof(t));
    int64_t borrow = 0;
    for (int i = 0; i < a->len; i++) {
        int64_t s = (int64_t)a->d[i] - (i < b->len ? b->d[i] : 0) - borrow;
        borrow = s < 0;
        if (s < 0) s += ((int64_t)1 << 32);
        t.d[i] = (uint32_t)s;
    }
    t.len = a->len;
    t.sign = 1;
    *r = t;
}

static void bn_add(bn *r, const bn *a, const bn *b)
{
    if (a->sign == 0) { *r = *b; return; }
    if (b->sign == 0) { *r = *a; return; }
    if (a->sign == b->sign) {
        int s = a->sign;
        mag_add(r, a, b);
        r->sign = s;
    } else {
        int c = mag_cmp(a, b);
        if (c == 0) { memset(r, 0, sizeof(*r)); return; }
        if (c > 0) { int s = a->sign; mag_sub(r, a, b); r->sign = s; }
        else { int s = b->sign; mag_sub(r, b, a); r->sign = s; }
    }
    bn_norm(r);
}

static void bn_neg(bn *a) { a->sign = -a->sign; }

static void bn_sub(bn *r, const bn *a, const bn *b)
{
    bn nb = *b;
    bn_neg(&nb);
    bn_add(r, a, &nb);
}

static void bn_mul(bn *r, const bn *a, const bn *b)
{
    if (a->sign == 0 || b->sign == 0) { memset(r, 0, sizeof(*r)); return; }
    if (a->len + b->len > BN_LIMBS) bn_fail("mul");
    bn t;
    memset(&t, 0, sizeof(t));
    for (int i = 0; i < a->len; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < b->len; j++) {
            uint64_t cur = (uint64_t)t.d[i + j] + (uint64_t)a->d[i] * b->d[j] + carry;
            t.d[i + j] = (uint32_t)cur;
            carry = cur >> 32;
        }
        t.d[i + b->len] = (uint32_t)carry;
    }
    t.len = a->len + b->len;
    t.sign = a->sign * b->sign;
    bn_norm(&t);
    *r = t;
}

static int min_exponent(const double *v, int k)
{
    int emin = 1 << 30;
    for (int i = 0; i < k; i++) {
        if (v[i] == 0.0) continue;
        int e;
        frexp(v[i], &e);
        if (e - 53 < emin) emin = e - 53;
    }
    return emin == (1 << 30) ? 0 : emin;
}

/* ---- orientation ---------------------------------------------------------- */

static int orient_exact(double ax, double ay, double bx, double by, double cx, double cy)
{
    double v[6] = {ax, ay, bx, by, cx, cy};
    int emin = min_exponent(v, 6);
    bn A[6];
    for (int i = 0; i < 6; i++) bn_from_double(&A[i], v[i], emin);
    bn bxa, bya, cxa, cya, t1, t2, det;
    bn_sub(&bxa, &A[2], &A[0]);
    bn_sub(&bya, &A[3], &A[1]);
    bn_sub(&cxa, &A[4], &A[0]);
    bn_sub(&cya, &A[5], &A[1]);
    bn_mul(&t1, &bxa, &cya);
    bn_mul(&t2, &bya, &cxa);
    bn_sub(&det, &t1, &t2);
    return det.sign;
}

int orc_orient(double ax, double ay, double bx, double by, double cx, double cy)
{
    double l = (bx - ax) * (cy - ay), r = (by - ay) * (cx - ax);
    double det = l - r, perm = fabs(l) + fabs(r);
    if (isfinite(det) && isfinite(perm) && fabs(det) > 1e-10 * perm) return det > 0 ? 1 : -1;
    return orient_exact(ax, ay, bx, by, cx, cy);
}

/* ---- in-circle ------------------------------------------------------------ */

static int incircle_exact(const double *v /* ax ay bx by cx cy dx dy */)
{
    int emin = min_exponent(v, 8);
    bn P[8];
    for (int i = 0; i < 8; i++) bn_from_double(&P[i], v[i], emin);
    bn adx, ady, bdx, bdy, cdx, cdy;
    bn_sub(&adx, &P[0], &P[6]);
    bn_sub(&ady, &P[1], &P[7]);
    bn_sub(&bdx, &P[2], &P[6]);
    bn_sub(&bdy, &P[3], &P[7]);
    bn_sub(&cdx, &P[4], &P[6]);
    bn_sub(&cdy, &P[5], &P[7]);
    bn t1, t2, la, lb, lc, ca, cb, cc, u, det;
    /* lifted heights of a, b, c relative to d */
    bn_mul(&t1, &adx, &adx); bn_mul(&t2, &ady, &ady); bn_add(&la, &t1, &t2);
    bn_mul(&t1, &bdx, &bdx); bn_mul(&t2, &bdy, &bdy); bn_add(&lb, &t1, &t2);
    bn_mul(&t1, &cdx, &cdx); bn_mul(&t2, &cdy, &cdy); bn_add(&lc, &t1, &t2);
    /* 2x2 minors */
    bn_mul(&t1, &bdx, &cdy); bn_mul(&t2, &cdx, &bdy); bn_sub(&ca, &t1, &t2);
    bn_mul(&t1, &cdx, &ady); bn_mul(&t2, &adx, &cdy); bn_sub(&cb, &t1, &t2);
    bn_mul(&t1, &adx, &bdy); bn_mul(&t2, &bdx, &ady); bn_sub(&cc, &t1, &t2);
    bn_mul(&det, &la, &ca);
    bn_mul(&u, &lb, &cb); bn_add(&det, &det, &u);
    bn_mul(&u, &lc, &cc); bn_add(&det, &det, &u);
    return det.sign;
}

/* Unperturbed sign: > 0 when d lies strictly inside the circle through the
   counter-clockwise triangle a, b, c. */
int orc_incircle_raw(double ax, double ay, double bx, double by, double cx, double cy,
                     double dx, double dy)
{
    double adx = ax - dx, ady = ay - dy, bdx = bx - dx, bdy = by - dy, cdx = cx - dx, cdy = cy - dy;
    double la = adx * adx + ady * ady, lb = bdx * bdx + bdy * bdy, lc = cdx * cdx + cdy * cdy;
    double m1 = bdx * cdy, m2 = cdx * bdy, m3 = cdx * ady, m4 = adx * cdy, m5 = adx * bdy, m6 = bdx * ady;
    double det = la * (m1 - m2) + lb * (m3 - m4) + lc * (m5 - m6);
    double perm = la * (fabs(m1) + fabs(m2)) + lb * (fabs(m3) + fabs(m4)) + lc * (fabs(m5) + fabs(m6));
    if (isfinite(det) && isfinite(perm) && fabs(det) > 1e-10 * perm) return det > 0 ? 1 : -1;
    double v[8] = {ax, ay, bx, by, cx, cy, dx, dy};
    return incircle_exact(v);
}

static int lex_less(double px, double py, double qx, double qy)
{
    return px < qx || (px == qx && py < qy);
}

/* Perturbed in-circle sign (never 0 for distinct points with a, b, c
   counter-clockwise).  With lifted heights |p|^2 + d_p the 4x4 lifting
   determinant changes, to first order, by d_a*orient(b,c,d) - d_b*orient(a,c,d)
   + d_c*orient(a,b,d) - d_d*orient(a,b,c); the term of the lexicographically
   smallest point dominates. */
int orc_incircle_sos(double ax, double ay, double bx, double by, double cx, double cy,
                     double dx, double dy)
{
    int s = orc_incircle_raw(ax, ay, bx, by, cx, cy, dx, dy);
    if (s != 0) return s;
    int which = 0;
    double mx = ax, my = ay;
    if (lex_less(bx, by, mx, my)) { which = 1; mx = bx; my = by; }
    if (lex_less(cx, cy, mx, my)) { which = 2; mx = cx; my = cy; }
    if (lex_less(dx, dy, mx, my)) { which = 3; mx = dx; my = dy; }
    switch (which) {
    case 0: return orc_orient(bx, by, cx, cy, dx, dy);
    case 1: return -orc_orient(ax, ay, cx, cy, dx, dy);
    case 2: return orc_orient(ax, ay, bx, by, dx, dy);
    default: return -orc_orient(ax, ay, bx, by, cx, cy);
    }
}
