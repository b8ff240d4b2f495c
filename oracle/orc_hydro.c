/*
 * ORACLE (test infrastructure only; never linked into the CUDA library).
 *
 * One step of the moving-mesh scheme of the paper, written as plainly as
 * possible, in FP64, one cell and one edge at a time:
 *
 *   tessellation  Section 2.1: Delaunay of the generating points plus ghost
 *                 images (mirror images at reflecting walls, shifted copies
 *                 for periodic boxes); Voronoi vertices are the circumcentres.
 *   geometry      cell area A_i, centre of mass s_i, edge length L_ij, edge
 *                 midpoint, r_ij, c_ij (the quantities named under Eq. 1).
 *   primitives    rho = m/A, v = P/m, p = (gamma-1)(E - |P|^2/(2m))/A.
 *   gradient      Eq. 1 (Green-Gauss), read with r_ij the generator separation
 *                 pointing from i to j and the denominators |r_ij|.
 *   limiter       Eqs. 3-5 (AREPO) and Eq. 6 (TESS, theta), switched per cell
 *                 by Eqs. 7-8 (delta_v, delta_p), Section 2.2.
 *   mesh motion   Section 6: w_i = v_i, plus chi*c_s towards the centre of mass
 *                 when the generator is more than eta*R_i away from it.
 *   time step     Courant condition of Section 2.3 (number 0.3 by default).
 *   fluxes        Section 2.3 "extrapolated fluxes": edge states are the
 *                 linear extrapolation of Eq. 2 advanced half a step with the
 *                 primitive Euler equations; Section 2.4 HLLC solver in the
 *                 frame of the moving edge (Section 1); Galilean transform back.
 *   update        U_i <- U_i - dt sum_j L_ij F_ij (conservative, Section 5).
 *
 * The second time advancement of Section 2.3, "time centred fluxes" (the
 * paper's own), runs the same sweep twice per step with no time prediction
 * of the edge states (spatial extrapolation only):
 *   half step     on the mesh of r^n: dt from the Courant condition;
 *                 U^{n+1/2} = U^n - (dt/2) sum L F(W^n),
 *                 r^{n+1/2} = r^n + (dt/2) w^n;
 *   full step     mesh rebuilt at r^{n+1/2}, W^{n+1/2} from U^{n+1/2} and the
 *                 new areas, w^{n+1/2} from them; the same dt;
 *                 U^{n+1} = U^n - dt sum L F(W^{n+1/2}) over the edges of the
 *                 half-step mesh, r^{n+1} = r^n + dt w^{n+1/2}.
 *
 * Points the paper leaves open and the reading taken here:
 *   - the limiter's max/min include the cell's own value (so alpha is in [0,1])
 *     and alpha is the minimum over all edges of the cell; the neighbours of
 *     Eqs. 3-8 are the cells sharing an edge longer than 1e-9 sqrt(A_i);
 *   - Eq. 7 reads -div(v) > delta_v c_s/R_i with R_i = sqrt(A_i/pi) and div(v)
 *     from the unlimited gradient; Eq. 8 reads "some neighbour has
 *     min(P_i,P_j)/max(P_i,P_j) < delta_p"; the switch applies to all four
 *     primitive variables of the cell;
 *   - the half-step prediction uses cell-centre primitives and the limited
 *     gradients in the primitive Euler equations written in the frame moving
 *     with the edge velocity w_f;
 *   - the edge velocity is that of the perpendicular bisector at the edge
 *     midpoint: w_f = (w_i+w_j)/2 - ((w_j-w_i).c_ij/|r_ij|) n_ij;
 *   - HLLC wave speeds are the direct (Davis) estimates;
 *   - dt = cfl * min_i R_i/(c_i + |v_i - w_i|), clipped to reach t_end;
 *   - the rounding velocity switches on as a step at d = eta*R_i;
 *   - a generating point that crosses a rigid wall is reflected back across it.
 * Every edge flux is evaluated from each of its two cells separately, which
 * is the literal per-cell sum above; the two evaluations agree to round-off.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "orc.h"

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_EDUP -2
#define ORC_ETESS -3
#define ORC_ETOOFEW -4
#define ORC_EBAD -5

struct orc_sim {
    orc_config c;
    int n;
    double *x, *y;              /* generating points */
    double *m, *px, *py, *E;    /* extensive conserved quantities */
    double t;
    int tess_ok;
    double band;
    /* tessellation */
    int np;
    double *X, *Y;              /* real points then ghost images */
    int *src, *fx, *fy;         /* source cell; mirror flags (+-1 walls, 0 none) */
    int *sx, *sy;               /* periodic shifts (-1, 0, 1) */
    int *rptr, *rnb;            /* counter-clockwise neighbour ring of each real cell */
    double *rvx, *rvy;          /* Voronoi vertex after ring slot k (absolute coords) */
    /* per-cell results of the last sweep */
    double *A, *ox, *oy;        /* area; centre of mass minus generator */
    double *W;                  /* 4 per cell: rho, vx, vy, p */
    double *cs;
    double *g, *gl;             /* 8 per cell: d/dx, d/dy of rho, vx, vy, p */
    double *alpha;              /* 4 per cell */
    double *wx, *wy;
    int *tess;
    double dt;
    double *x_prev, *y_prev;    /* generating points at the start of the last sweep */
    /* time-centred scheme: state and points at the start of the step */
    double *m0, *px0, *py0, *E0, *x0, *y0;
};

static void *xmalloc(size_t n) { void *p = calloc(1, n > 0 ? n : 1); if (!p) abort(); return p; }

/* ------------------------------------------------------------------------ */
/* ghost images                                                              */

static int add_point(orc_sim *s, int *cap, double X, double Y, int src, int fx, int fy, int sx, int sy)
{
    if (s->np == *cap) {
        *cap = *cap * 2 + 64;
        s->X = realloc(s->X, sizeof(double) * *cap);
        s->Y = realloc(s->Y, sizeof(double) * *cap);
        s->src = realloc(s->src, sizeof(int) * *cap);
        s->fx = realloc(s->fx, sizeof(int) * *cap);
        s->fy = realloc(s->fy, sizeof(int) * *cap);
        s->sx = realloc(s->sx, sizeof(int) * *cap);
        s->sy = realloc(s->sy, sizeof(int) * *cap);
    }
    int q = s->np++;
    s->X[q] = X; s->Y[q] = Y; s->src[q] = src;
    s->fx[q] = fx; s->fy[q] = fy; s->sx[q] = sx; s->sy[q] = sy;
    return q;
}

/* image coordinate: mirror about x0 is (x0+x0)-x, about x1 is (x1+x1)-x;
   a periodic copy is x+L or x-L with L = x1-x0. */
static double image_coord(double v, double lo, double hi, int flip, int shift)
{
    if (flip < 0) return (lo + lo) - v;
    if (flip > 0) return (hi + hi) - v;
    if (shift > 0) return v + (hi - lo);
    if (shift < 0) return v - (hi - lo);
    return v;
}

static void build_points(orc_sim *s, double w)
{
    const orc_config *c = &s->c;
    int cap = 0;
    s->np = 0;
    for (int i = 0; i < s->n; i++) add_point(s, &cap, s->x[i], s->y[i], i, 0, 0, 0, 0);
    for (int i = 0; i < s->n; i++) {
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++) {
                if (a == 0 && b == 0) continue;
                int fx = 0, fy = 0, sx = 0, sy = 0;
                if (c->boundary == 1) { sx = a; sy = b; }
                else { fx = a; fy = b; }
                double X = image_coord(s->x[i], c->x0, c->x1, fx, sx);
                double Y = image_coord(s->y[i], c->y0, c->y1, fy, sy);
                if (X >= c->x0 - w && X <= c->x1 + w && Y >= c->y0 - w && Y <= c->y1 + w)
                    add_point(s, &cap, X, Y, i, fx, fy, sx, sy);
            }
    }
}

/* ------------------------------------------------------------------------ */
/* circumcentre relative to the first vertex                                 */

static void circumcentre(double ax, double ay, double bx, double by, double cx, double cy,
                         double *ux, double *uy)
{
    double bxr = bx - ax, byr = by - ay, cxr = cx - ax, cyr = cy - ay;
    double d = 2.0 * (bxr * cyr - byr * cxr);
    double b2 = bxr * bxr + byr * byr, c2 = cxr * cxr + cyr * cyr;
    *ux = ax + (cyr * b2 - byr * c2) / d;
    *uy = ay + (bxr * c2 - cxr * b2) / d;
}

typedef struct { int i, a, b; double vx, vy; } ring_entry;

static int cmp_entry(const void *p, const void *q)
{
    const ring_entry *u = (const ring_entry *)p, *v = (const ring_entry *)q;
    if (u->i != v->i) return u->i - v->i;
    return u->a - v->a;
}

static void free_tess(orc_sim *s)
{
    free(s->X); free(s->Y); free(s->src); free(s->fx); free(s->fy); free(s->sx); free(s->sy);
    free(s->rptr); free(s->rnb); free(s->rvx); free(s->rvy);
    s->X = s->Y = NULL; s->src = s->fx = s->fy = s->sx = s->sy = NULL;
    s->rptr = s->rnb = NULL; s->rvx = s->rvy = NULL;
    s->np = 0;
}

int orc_tessellate(orc_sim *s)
{
    const orc_config *c = &s->c;
    double Lx = c->x1 - c->x0, Ly = c->y1 - c->y0;
    double h = sqrt(Lx * Ly / s->n);
    double w = 4.0 * h;
    double wmax = Lx < Ly ? Lx : Ly;
    if (w > wmax) w = wmax;
    for (;;) {
        free_tess(s);
        build_points(s, w);
        int ntri = 0, *tris = NULL;
        int rc = orc_delaunay(s->np, s->X, s->Y, &ntri, &tris);
        if (rc == -2) { free(tris); return ORC_EDUP; }
        if (rc != 0) { free(tris); return ORC_ETESS; }
        /* collect the triangles that touch a real cell; check the band */
        int ok = 1, nent = 0;
        ring_entry *ent = xmalloc(sizeof(ring_entry) * 3 * (size_t)ntri);
        for (int t = 0; t < ntri && ok; t++) {
            int *v = &tris[3 * t];
            int real = v[0] < s->n || v[1] < s->n || v[2] < s->n;
            if (!real) continue;
            if (v[0] >= s->np || v[1] >= s->np || v[2] >= s->np) { ok = 0; break; }
            double ux, uy;
            circumcentre(s->X[v[0]], s->Y[v[0]], s->X[v[1]], s->Y[v[1]], s->X[v[2]], s->Y[v[2]], &ux, &uy);
            double R = hypot(s->X[v[0]] - ux, s->Y[v[0]] - uy) * (1.0 + 1e-9) + 1e-12 * (Lx + Ly);
            if (!(ux - R >= c->x0 - w && ux + R <= c->x1 + w && uy - R >= c->y0 - w && uy + R <= c->y1 + w)) {
                ok = 0;
                break;
            }
            for (int k = 0; k < 3; k++) {
                if (v[k] >= s->n) continue;
                ent[nent].i = v[k];
                ent[nent].a = v[(k + 1) % 3];
                ent[nent].b = v[(k + 2) % 3];
                ent[nent].vx = ux;
                ent[nent].vy = uy;
                nent++;
            }
        }
        free(tris);
        if (!ok) {
            free(ent);
            if (w >= wmax) return ORC_ETOOFEW;
            w = 2.0 * w > wmax ? wmax : 2.0 * w;
            continue;
        }
        /* chain the triangles around every real cell into a ring */
        qsort(ent, nent, sizeof(ring_entry), cmp_entry);
        s->rptr = xmalloc(sizeof(int) * (s->n + 1));
        s->rnb = xmalloc(sizeof(int) * nent);
        s->rvx = xmalloc(sizeof(double) * nent);
        s->rvy = xmalloc(sizeof(double) * nent);
        int e = 0;
        for (int i = 0; i < s->n; i++) {
            s->rptr[i] = e;
            int lo = e, hi = e;
            while (hi < nent && ent[hi].i == i) hi++;
            int deg = hi - lo;
            if (deg < 3) { free(ent); return ORC_ETESS; }
            /* follow a -> b successors starting from the first entry */
            int cur = lo;
            for (int k = 0; k < deg; k++) {
                s->rnb[e + k] = ent[cur].a;
                s->rvx[e + k] = ent[cur].vx;
                s->rvy[e + k] = ent[cur].vy;
                int nxt = -1;
                for (int q = lo; q < hi; q++)
                    if (ent[q].a == ent[cur].b) { nxt = q; break; }
                if (nxt < 0) { free(ent); return ORC_ETESS; }
                cur = nxt;
            }
            if (cur != lo) { free(ent); return ORC_ETESS; }
            e = hi;
        }
        s->rptr[s->n] = e;
        free(ent);
        s->band = w;
        s->tess_ok = 1;
        return ORC_OK;
    }
}

/* ------------------------------------------------------------------------ */
/* ghost views of per-cell data                                              */

static void view_W(const orc_sim *s, int q, double W[4])
{
    int k = s->src[q];
    memcpy(W, &s->W[4 * k], sizeof(double) * 4);
    if (s->fx[q]) W[1] = -W[1];
    if (s->fy[q]) W[2] = -W[2];
}

/* gradient layout: (d/dx, d/dy) of rho, vx, vy, p */
static void view_grad(const orc_sim *s, const double *G, int q, double g[8])
{
    int k = s->src[q];
    memcpy(g, &G[8 * k], sizeof(double) * 8);
    double ax = s->fx[q] ? -1.0 : 1.0, ay = s->fy[q] ? -1.0 : 1.0;
    /* a mirrored scalar f'(x') = f(Tx'): each derivative picks up the flip of its axis;
       a mirrored velocity component also picks up the flip of its own axis */
    g[0] *= ax; g[1] *= ay;
    g[2] *= ax * ax; g[3] *= ax * ay;
    g[4] *= ay * ax; g[5] *= ay * ay;
    g[6] *= ax; g[7] *= ay;
}

static void view_w(const orc_sim *s, int q, double w[2])
{
    int k = s->src[q];
    w[0] = s->fx[q] ? -s->wx[k] : s->wx[k];
    w[1] = s->fy[q] ? -s->wy[k] : s->wy[k];
}

/* centre of mass minus generator */
static void view_off(const orc_sim *s, int q, double o[2])
{
    int k = s->src[q];
    o[0] = s->fx[q] ? -s->ox[k] : s->ox[k];
    o[1] = s->fy[q] ? -s->oy[k] : s->oy[k];
}

/* geometry of ring slot (i, k), all vectors relative to generator i */
typedef struct {
    int j;
    double L;        /* edge length */
    double mx, my;   /* edge midpoint - r_i */
    double rx, ry;   /* r_j - r_i */
    double rl;       /* |r_j - r_i| */
    double nx, ny;   /* unit normal from i to j */
    double cx, cy;   /* c_ij: edge midpoint - generator midpoint */
} slot_geom;

static void get_slot(const orc_sim *s, int i, int k, slot_geom *G)
{
    int lo = s->rptr[i], deg = s->rptr[i + 1] - lo;
    int kp = (k + deg - 1) % deg;
    double ax = s->rvx[lo + kp] - s->x[i], ay = s->rvy[lo + kp] - s->y[i];
    double bx = s->rvx[lo + k] - s->x[i], by = s->rvy[lo + k] - s->y[i];
    G->j = s->rnb[lo + k];
    G->L = hypot(bx - ax, by - ay);
    G->mx = 0.5 * (ax + bx);
    G->my = 0.5 * (ay + by);
    G->rx = s->X[G->j] - s->x[i];
    G->ry = s->Y[G->j] - s->y[i];
    G->rl = hypot(G->rx, G->ry);
    G->nx = G->rx / G->rl;
    G->ny = G->ry / G->rl;
    G->cx = G->mx - 0.5 * G->rx;
    G->cy = G->my - 0.5 * G->ry;
}

/* ------------------------------------------------------------------------ */
/* HLLC (Section 2.4) in the edge frame: W = (rho, u normal, u tangential, p) */

void orc_hllc(double gam, const double WL[4], const double WR[4], double F[4])
{
    double rL = WL[0], uL = WL[1], tL = WL[2], pL = WL[3];
    double rR = WR[0], uR = WR[1], tR = WR[2], pR = WR[3];
    double cL = sqrt(gam * pL / rL), cR = sqrt(gam * pR / rR);
    double EL = pL / (gam - 1.0) + 0.5 * rL * (uL * uL + tL * tL);
    double ER = pR / (gam - 1.0) + 0.5 * rR * (uR * uR + tR * tR);
    double SL = fmin(uL - cL, uR - cR);
    double SR = fmax(uL + cL, uR + cR);
    double FL[4] = {rL * uL, rL * uL * uL + pL, rL * uL * tL, uL * (EL + pL)};
    double FR[4] = {rR * uR, rR * uR * uR + pR, rR * uR * tR, uR * (ER + pR)};
    if (SL >= 0.0) { memcpy(F, FL, sizeof(FL)); return; }
    if (SR <= 0.0) { memcpy(F, FR, sizeof(FR)); return; }
    double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    if (Ss >= 0.0) {
        double f = rL * (SL - uL) / (SL - Ss);
        double Us[4] = {f, f * Ss, f * tL, f * (EL / rL + (Ss - uL) * (Ss + pL / (rL * (SL - uL))))};
        double U[4] = {rL, rL * uL, rL * tL, EL};
        for (int q = 0; q < 4; q++) F[q] = FL[q] + SL * (Us[q] - U[q]);
    } else {
        double f = rR * (SR - uR) / (SR - Ss);
        double Us[4] = {f, f * Ss, f * tR, f * (ER / rR + (Ss - uR) * (Ss + pR / (rR * (SR - uR))))};
        double U[4] = {rR, rR * uR, rR * tR, ER};
        for (int q = 0; q < 4; q++) F[q] = FR[q] + SR * (Us[q] - U[q]);
    }
}

/* Edge state of one side: Eq. 2 extrapolation to the edge midpoint, then half
   a step of the primitive Euler equations in the frame moving with wf. */
static void predict(double gam, double hdt, const double W[4], const double g[8], double offx, double offy,
                    const double wf[2], double out[4])
{
    double rho = W[0], vx = W[1], vy = W[2], p = W[3];
    double ux = vx - wf[0], uy = vy - wf[1];
    double div = g[2] + g[5];
    out[0] = rho + g[0] * offx + g[1] * offy;
    out[1] = vx + g[2] * offx + g[3] * offy;
    out[2] = vy + g[4] * offx + g[5] * offy;
    out[3] = p + g[6] * offx + g[7] * offy;
    out[0] -= hdt * (ux * g[0] + uy * g[1] + rho * div);
    out[1] -= hdt * (ux * g[2] + uy * g[3] + g[6] / rho);
    out[2] -= hdt * (ux * g[4] + uy * g[5] + g[7] / rho);
    out[3] -= hdt * (ux * g[6] + uy * g[7] + gam * p * div);
}

/* the edge-state prediction on its own, for the pins of Section 2.3's
   half-step prediction (velocity out in the lab frame) */
void orc_predict(double gam, double hdt, const double W[4], const double g[8], double offx, double offy,
                 const double wf[2], double out[4])
{
    predict(gam, hdt, W, g, offx, offy, wf, out);
}

/* ------------------------------------------------------------------------ */

int orc_create(const orc_config *cfg, int n, const double *x, const double *y, const double *rho,
               const double *vx, const double *vy, const double *p, orc_sim **out)
{
    *out = NULL;
    if (n < 3 || !(cfg->gamma > 1.0) || !(cfg->x1 > cfg->x0) || !(cfg->y1 > cfg->y0)) return ORC_EINVAL;
    if (cfg->scheme != 0 && cfg->scheme != 1) return ORC_EINVAL;
    for (int i = 0; i < n; i++) {
        if (!(x[i] > cfg->x0 && x[i] < cfg->x1 && y[i] > cfg->y0 && y[i] < cfg->y1)) {
            if (!(cfg->boundary == 1 && x[i] >= cfg->x0 && x[i] < cfg->x1 && y[i] >= cfg->y0 && y[i] < cfg->y1))
                return ORC_EINVAL;
        }
        if (!(rho[i] > 0) || !(p[i] > 0) || !isfinite(vx[i]) || !isfinite(vy[i])) return ORC_EINVAL;
    }
    orc_sim *s = xmalloc(sizeof(orc_sim));
    s->c = *cfg;
    s->n = n;
    s->x = xmalloc(sizeof(double) * n); s->y = xmalloc(sizeof(double) * n);
    memcpy(s->x, x, sizeof(double) * n); memcpy(s->y, y, sizeof(double) * n);
    s->m = xmalloc(sizeof(double) * n); s->px = xmalloc(sizeof(double) * n);
    s->py = xmalloc(sizeof(double) * n); s->E = xmalloc(sizeof(double) * n);
    s->A = xmalloc(sizeof(double) * n); s->ox = xmalloc(sizeof(double) * n); s->oy = xmalloc(sizeof(double) * n);
    s->W = xmalloc(sizeof(double) * 4 * n); s->cs = xmalloc(sizeof(double) * n);
    s->g = xmalloc(sizeof(double) * 8 * n); s->gl = xmalloc(sizeof(double) * 8 * n);
    s->alpha = xmalloc(sizeof(double) * 4 * n);
    s->wx = xmalloc(sizeof(double) * n); s->wy = xmalloc(sizeof(double) * n);
    s->tess = xmalloc(sizeof(int) * n);
    s->x_prev = xmalloc(sizeof(double) * n); s->y_prev = xmalloc(sizeof(double) * n);
    memcpy(s->x_prev, x, sizeof(double) * n); memcpy(s->y_prev, y, sizeof(double) * n);
    s->m0 = xmalloc(sizeof(double) * n); s->px0 = xmalloc(sizeof(double) * n);
    s->py0 = xmalloc(sizeof(double) * n); s->E0 = xmalloc(sizeof(double) * n);
    s->x0 = xmalloc(sizeof(double) * n); s->y0 = xmalloc(sizeof(double) * n);
    int rc = orc_tessellate(s);
    if (rc != ORC_OK) { orc_destroy(s); return rc; }
    /* areas of the initial cells turn the primitive fields into extensive ones */
    for (int i = 0; i < n; i++) {
        int lo = s->rptr[i], deg = s->rptr[i + 1] - lo;
        double A2 = 0;
        for (int k = 0; k < deg; k++) {
            int k1 = (k + 1) % deg;
            double ax = s->rvx[lo + k] - x[i], ay = s->rvy[lo + k] - y[i];
            double bx = s->rvx[lo + k1] - x[i], by = s->rvy[lo + k1] - y[i];
            A2 += ax * by - ay * bx;
        }
        double A = 0.5 * A2;
        s->m[i] = rho[i] * A;
        s->px[i] = rho[i] * vx[i] * A;
        s->py[i] = rho[i] * vy[i] * A;
        s->E[i] = (p[i] / (cfg->gamma - 1.0) + 0.5 * rho[i] * (vx[i] * vx[i] + vy[i] * vy[i])) * A;
    }
    *out = s;
    return ORC_OK;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free_tess(s);
    free(s->x); free(s->y); free(s->m); free(s->px); free(s->py); free(s->E);
    free(s->A); free(s->ox); free(s->oy); free(s->W); free(s->cs); free(s->g); free(s->gl);
    free(s->alpha); free(s->wx); free(s->wy); free(s->tess);
    free(s->x_prev); free(s->y_prev);
    free(s->m0); free(s->px0); free(s->py0); free(s->E0); free(s->x0); free(s->y0);
    free(s);
}

static int geometry_and_primitives(orc_sim *s)
{
    const double gam = s->c.gamma;
    const int n = s->n;
    /* geometry: area and centre of mass of every real cell (shoelace about r_i) */
    for (int i = 0; i < n; i++) {
        int lo = s->rptr[i], deg = s->rptr[i + 1] - lo;
        double A2 = 0, Sx = 0, Sy = 0;
        for (int k = 0; k < deg; k++) {
            int k1 = (k + 1) % deg;
            double ax = s->rvx[lo + k] - s->x[i], ay = s->rvy[lo + k] - s->y[i];
            double bx = s->rvx[lo + k1] - s->x[i], by = s->rvy[lo + k1] - s->y[i];
            double cr = ax * by - ay * bx;
            A2 += cr;
            Sx += (ax + bx) * cr;
            Sy += (ay + by) * cr;
        }
        s->A[i] = 0.5 * A2;
        s->ox[i] = Sx / (3.0 * A2);
        s->oy[i] = Sy / (3.0 * A2);
        if (!(s->A[i] > 0)) return ORC_ETESS;
    }
    /* primitive variables and sound speed */
    for (int i = 0; i < n; i++) {
        double rho = s->m[i] / s->A[i];
        double vx = s->px[i] / s->m[i], vy = s->py[i] / s->m[i];
        double p = (gam - 1.0) * (s->E[i] - 0.5 * (s->px[i] * vx + s->py[i] * vy)) / s->A[i];
        s->W[4 * i] = rho; s->W[4 * i + 1] = vx; s->W[4 * i + 2] = vy; s->W[4 * i + 3] = p;
        s->cs[i] = sqrt(gam * p / rho);
        if (!(rho > 0) || !(p > 0)) return ORC_EBAD;
    }
    return ORC_OK;
}

/* One sweep over the current tessellation.  pass 0: the extrapolated-fluxes
   step; pass 1: the half step of the time-centred scheme (saves U^n and r^n
   first); pass 2: its full step with the half step's dt, from the saved
   U^n and r^n. */
static int sweep_pass(orc_sim *s, double t_end, int pass, double *dt_out)
{
    if (!s->tess_ok) return ORC_ETESS;
    const orc_config *c = &s->c;
    const double gam = c->gamma;
    const int n = s->n;

    int rc = geometry_and_primitives(s);
    if (rc) return rc;
    memcpy(s->x_prev, s->x, sizeof(double) * n);
    memcpy(s->y_prev, s->y, sizeof(double) * n);
    /* Eq. 1: Green-Gauss gradient of each primitive */
    for (int i = 0; i < n; i++) {
        int lo = s->rptr[i], deg = s->rptr[i + 1] - lo;
        double acc[8] = {0};
        for (int k = 0; k < deg; k++) {
            slot_geom G;
            get_slot(s, i, k, &G);
            double Wj[4];
            view_W(s, G.j, Wj);
            for (int v = 0; v < 4; v++) {
                double fi = s->W[4 * i + v], fj = Wj[v];
                acc[2 * v] += G.L * ((fj - fi) * G.cx / G.rl + 0.5 * (fi + fj) * G.nx);
                acc[2 * v + 1] += G.L * ((fj - fi) * G.cy / G.rl + 0.5 * (fi + fj) * G.ny);
            }
        }
        for (int q = 0; q < 8; q++) s->g[8 * i + q] = acc[q] / s->A[i];
    }
    /* Eqs. 3-8: slope limiter with the shock switch.  Neighbours are the
       cells sharing a Voronoi edge of positive length: an edge shorter than
       1e-9 sqrt(A_i) is a point contact (the Delaunay triangulation of
       co-circular points is not unique, the Voronoi diagram is). */
    for (int i = 0; i < n; i++) {
        int lo = s->rptr[i], deg = s->rptr[i + 1] - lo;
        const double *Wi = &s->W[4 * i];
        const double *gi = &s->g[8 * i];
        double R = sqrt(s->A[i] / M_PI);
        double Lmin = 1e-9 * sqrt(s->A[i]);
        int shock = -(gi[2] + gi[5]) > c->delta_v * s->cs[i] / R;
        double fmaxv[4], fminv[4];
        for (int v = 0; v < 4; v++) fmaxv[v] = fminv[v] = Wi[v];
        for (int k = 0; k < deg; k++) {
            slot_geom G;
            get_slot(s, i, k, &G);
            if (G.L <= Lmin) continue;
            double Wj[4];
            view_W(s, G.j, Wj);
            for (int v = 0; v < 4; v++) {
                if (Wj[v] > fmaxv[v]) fmaxv[v] = Wj[v];
                if (Wj[v] < fminv[v]) fminv[v] = Wj[v];
            }
            double pr = fmin(Wi[3], Wj[3]) / fmax(Wi[3], Wj[3]);
            if (pr < c->delta_p) shock = 1;
        }
        int use_tess = c->limiter == 2 || (c->limiter == 0 && shock);
        s->tess[i] = use_tess;
        for (int v = 0; v < 4; v++) {
            double a = 1.0;
            for (int k = 0; k < deg; k++) {
                slot_geom G;
                get_slot(s, i, k, &G);
                if (G.L <= Lmin) continue;
                double Wj[4];
                view_W(s, G.j, Wj);
                double dphi = gi[2 * v] * (G.mx - s->ox[i]) + gi[2 * v + 1] * (G.my - s->oy[i]);
                double psi;
                if (dphi == 0.0) psi = 1.0;
                else if (use_tess) psi = fmax(c->theta * (Wj[v] - Wi[v]) / dphi, 0.0);
                else if (dphi > 0.0) psi = (fmaxv[v] - Wi[v]) / dphi;
                else psi = (fminv[v] - Wi[v]) / dphi;
                if (psi < a) a = psi;
            }
            s->alpha[4 * i + v] = a;
            s->gl[8 * i + 2 * v] = a * gi[2 * v];
            s->gl[8 * i + 2 * v + 1] = a * gi[2 * v + 1];
        }
    }
    /* Section 6: mesh-generating point velocities */
    for (int i = 0; i < n; i++) {
        double vx = s->W[4 * i + 1], vy = s->W[4 * i + 2];
        if (c->motion == 1) { s->wx[i] = 0; s->wy[i] = 0; continue; }
        double d = hypot(s->ox[i], s->oy[i]);
        double R = sqrt(s->A[i] / M_PI);
        if (d > c->eta * R) {
            s->wx[i] = vx + c->chi * s->cs[i] * s->ox[i] / d;
            s->wy[i] = vy + c->chi * s->cs[i] * s->oy[i] / d;
        } else {
            s->wx[i] = vx;
            s->wy[i] = vy;
        }
    }
    /* Courant condition (the full step of the time-centred scheme keeps the
       half step's dt) */
    double dt = INFINITY;
    if (pass == 2) {
        dt = s->dt;
    } else {
        for (int i = 0; i < n; i++) {
            double R = sqrt(s->A[i] / M_PI);
            double rel = hypot(s->W[4 * i + 1] - s->wx[i], s->W[4 * i + 2] - s->wy[i]);
            double d = R / (s->cs[i] + rel);
            if (d < dt) dt = d;
        }
        dt *= c->cfl;
        if (s->t + dt > t_end) dt = t_end - s->t;
        if (!(dt >= 0)) return ORC_EBAD;
        s->dt = dt;
    }
    /* edge states: advanced half a step in time by the extrapolated-fluxes
       scheme, spatial extrapolation only in the time-centred one */
    const double hdt = pass == 0 ? 0.5 * dt : 0.0;
    if (pass == 1) {
        memcpy(s->m0, s->m, sizeof(double) * n); memcpy(s->px0, s->px, sizeof(double) * n);
        memcpy(s->py0, s->py, sizeof(double) * n); memcpy(s->E0, s->E, sizeof(double) * n);
        memcpy(s->x0, s->x, sizeof(double) * n); memcpy(s->y0, s->y, sizeof(double) * n);
    }
    /* fluxes through every edge of every cell, and the conservative update */
    double *dU = xmalloc(sizeof(double) * 4 * n);
    for (int i = 0; i < n; i++) {
        int lo = s->rptr[i], deg = s->rptr[i + 1] - lo;
        double Wi[4], gi[8], wi[2] = {s->wx[i], s->wy[i]}, oi[2] = {s->ox[i], s->oy[i]};
        memcpy(Wi, &s->W[4 * i], sizeof(Wi));
        memcpy(gi, &s->gl[8 * i], sizeof(gi));
        for (int k = 0; k < deg; k++) {
            slot_geom G;
            get_slot(s, i, k, &G);
            double Wj[4], gj[8], wj[2], oj[2];
            view_W(s, G.j, Wj);
            view_grad(s, s->gl, G.j, gj);
            view_w(s, G.j, wj);
            view_off(s, G.j, oj);
            /* velocity of the edge: the perpendicular bisector at its midpoint */
            double dwc = ((wj[0] - wi[0]) * G.cx + (wj[1] - wi[1]) * G.cy) / G.rl;
            double wf[2] = {0.5 * (wi[0] + wj[0]) - dwc * G.nx, 0.5 * (wi[1] + wj[1]) - dwc * G.ny};
            /* edge midpoint relative to each side's centre of mass */
            double offi_x = G.mx - oi[0], offi_y = G.my - oi[1];
            double offj_x = G.mx - (G.rx + oj[0]), offj_y = G.my - (G.ry + oj[1]);
            double Si[4], Sj[4];
            predict(gam, hdt, Wi, gi, offi_x, offi_y, wf, Si);
            predict(gam, hdt, Wj, gj, offj_x, offj_y, wf, Sj);
            /* boost into the edge frame and rotate to (normal, tangential) */
            double tx = -G.ny, ty = G.nx;
            double WL[4] = {Si[0], (Si[1] - wf[0]) * G.nx + (Si[2] - wf[1]) * G.ny,
                            (Si[1] - wf[0]) * tx + (Si[2] - wf[1]) * ty, Si[3]};
            double WR[4] = {Sj[0], (Sj[1] - wf[0]) * G.nx + (Sj[2] - wf[1]) * G.ny,
                            (Sj[1] - wf[0]) * tx + (Sj[2] - wf[1]) * ty, Sj[3]};
            double Fe[4];
            orc_hllc(gam, WL, WR, Fe);
            /* rotate back and transform to the lab frame */
            double Fmx = Fe[1] * G.nx + Fe[2] * tx, Fmy = Fe[1] * G.ny + Fe[2] * ty;
            double F0 = Fe[0];
            double F1 = Fmx + F0 * wf[0];
            double F2 = Fmy + F0 * wf[1];
            double F3 = Fe[3] + Fmx * wf[0] + Fmy * wf[1] + 0.5 * (wf[0] * wf[0] + wf[1] * wf[1]) * F0;
            dU[4 * i] -= dt * G.L * F0;
            dU[4 * i + 1] -= dt * G.L * F1;
            dU[4 * i + 2] -= dt * G.L * F2;
            dU[4 * i + 3] -= dt * G.L * F3;
        }
    }
    /* new state and points from those at the start of the step: half the
       change in the half step of the time-centred scheme */
    const double f = pass == 1 ? 0.5 : 1.0;
    const double *bm = pass == 0 ? s->m : s->m0, *bpx = pass == 0 ? s->px : s->px0;
    const double *bpy = pass == 0 ? s->py : s->py0, *bE = pass == 0 ? s->E : s->E0;
    const double *bx = pass == 0 ? s->x : s->x0, *by = pass == 0 ? s->y : s->y0;
    int bad = 0;
    for (int i = 0; i < n; i++) {
        s->m[i] = bm[i] + f * dU[4 * i];
        s->px[i] = bpx[i] + f * dU[4 * i + 1];
        s->py[i] = bpy[i] + f * dU[4 * i + 2];
        s->E[i] = bE[i] + f * dU[4 * i + 3];
        if (!(s->m[i] > 0) || !(s->E[i] - 0.5 * (s->px[i] * s->px[i] + s->py[i] * s->py[i]) / s->m[i] > 0)) bad = 1;
        /* move the generating points; wrap into a periodic box, and reflect a
           point that crossed a rigid wall back across it (as its mirror image) */
        double nx = bx[i] + f * dt * s->wx[i], ny = by[i] + f * dt * s->wy[i];
        if (c->boundary == 1) {
            double Lx = c->x1 - c->x0, Ly = c->y1 - c->y0;
            if (nx < c->x0) nx += Lx;
            else if (nx >= c->x1) nx -= Lx;
            if (ny < c->y0) ny += Ly;
            else if (ny >= c->y1) ny -= Ly;
        } else {
            if (nx <= c->x0) nx = (c->x0 + c->x0) - nx;
            else if (nx >= c->x1) nx = (c->x1 + c->x1) - nx;
            if (ny <= c->y0) ny = (c->y0 + c->y0) - ny;
            else if (ny >= c->y1) ny = (c->y1 + c->y1) - ny;
            if (!(nx > c->x0 && nx < c->x1 && ny > c->y0 && ny < c->y1)) bad = 1;
        }
        s->x[i] = nx;
        s->y[i] = ny;
    }
    free(dU);
    if (pass != 1) s->t += dt;
    s->tess_ok = 0;
    if (dt_out) *dt_out = dt;
    return bad ? ORC_EBAD : ORC_OK;
}

/* primitives and areas on the current positions (tessellates if they moved) */
int orc_get_primitives(orc_sim *s, double *rho, double *vx, double *vy, double *p, double *area)
{
    if (!s->tess_ok) {
        int rc = orc_tessellate(s);
        if (rc) return rc;
    }
    int rc = geometry_and_primitives(s);
    if (rc) return rc;
    memcpy(s->x_prev, s->x, sizeof(double) * s->n);
    memcpy(s->y_prev, s->y, sizeof(double) * s->n);
    for (int i = 0; i < s->n; i++) {
        if (rho) rho[i] = s->W[4 * i];
        if (vx) vx[i] = s->W[4 * i + 1];
        if (vy) vy[i] = s->W[4 * i + 2];
        if (p) p[i] = s->W[4 * i + 3];
        if (area) area[i] = s->A[i];
    }
    return ORC_OK;
}

/* one step over the current tessellation: one sweep (extrapolated fluxes),
   or half step, re-tessellation and full step (time-centred fluxes) */
int orc_sweep(orc_sim *s, double t_end, double *dt_out)
{
    if (s->c.scheme == 0) return sweep_pass(s, t_end, 0, dt_out);
    int rc = sweep_pass(s, t_end, 1, NULL);
    if (rc) return rc;
    rc = orc_tessellate(s);
    if (rc) return rc;
    return sweep_pass(s, t_end, 2, dt_out);
}

int orc_step(orc_sim *s, double t_end, double *dt_out)
{
    if (!s->tess_ok) {
        int rc = orc_tessellate(s);
        if (rc) return rc;
    }
    return orc_sweep(s, t_end, dt_out);
}

double orc_time(const orc_sim *s) { return s->t; }
double orc_band(const orc_sim *s) { return s->band; }
int orc_num_points(const orc_sim *s) { return s->np; }

int orc_get_points(const orc_sim *s, double *X, double *Y, int *src)
{
    for (int q = 0; q < s->np; q++) {
        if (X) X[q] = s->X[q];
        if (Y) Y[q] = s->Y[q];
        if (src) src[q] = s->src[q];
    }
    return s->np;
}

int orc_ring_total(const orc_sim *s) { return s->tess_ok ? s->rptr[s->n] : -1; }

int orc_get_ring(const orc_sim *s, int *ptr, int *nb)
{
    if (!s->tess_ok) return ORC_ETESS;
    memcpy(ptr, s->rptr, sizeof(int) * (s->n + 1));
    memcpy(nb, s->rnb, sizeof(int) * s->rptr[s->n]);
    return ORC_OK;
}

int orc_get_conserved(const orc_sim *s, double *x, double *y, double *m, double *px, double *py, double *E)
{
    size_t b = sizeof(double) * s->n;
    if (x) memcpy(x, s->x, b);
    if (y) memcpy(y, s->y, b);
    if (m) memcpy(m, s->m, b);
    if (px) memcpy(px, s->px, b);
    if (py) memcpy(py, s->py, b);
    if (E) memcpy(E, s->E, b);
    return ORC_OK;
}

/* fields: 0 area, 1-2 centre of mass, 3-6 rho vx vy p, 7 c_s, 8-15 gradient,
   16-23 limited gradient, 24-25 w, 26 TESS flag, 27-30 alpha, 31 dt */
int orc_get_cells(const orc_sim *s, int f, double *out)
{
    for (int i = 0; i < s->n; i++) {
        double v;
        if (f == 0) v = s->A[i];
        else if (f == 1) v = s->x_prev[i] + s->ox[i];
        else if (f == 2) v = s->y_prev[i] + s->oy[i];
        else if (f >= 3 && f <= 6) v = s->W[4 * i + f - 3];
        else if (f == 7) v = s->cs[i];
        else if (f >= 8 && f <= 15) v = s->g[8 * i + f - 8];
        else if (f >= 16 && f <= 23) v = s->gl[8 * i + f - 16];
        else if (f == 24) v = s->wx[i];
        else if (f == 25) v = s->wy[i];
        else if (f == 26) v = s->tess[i];
        else if (f >= 27 && f <= 30) v = s->alpha[4 * i + f - 27];
        else if (f == 31) v = s->dt;
        else return ORC_EINVAL;
        out[i] = v;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact solution of the 1D Riemann problem for an ideal gas (used only to pin
   the shock-tube runs).  The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0,
   where f_K is the velocity jump across a shock (Rankine-Hugoniot) or a
   rarefaction (isentropic, Riemann invariant) connecting state K to pressure p. */

static double wave_f(double gam, double p, double rK, double pK)
{
    double cK = sqrt(gam * pK / rK);
    if (p > pK) {
        double A = 2.0 / ((gam + 1.0) * rK), B = (gam - 1.0) / (gam + 1.0) * pK;
        return (p - pK) * sqrt(A / (p + B));
    }
    return 2.0 * cK / (gam - 1.0) * (pow(p / pK, (gam - 1.0) / (2.0 * gam)) - 1.0);
}

int orc_riemann_exact(double gam, double rl, double ul, double pl, double rr, double ur, double pr,
                      double *ps, double *us)
{
    double cl = sqrt(gam * pl / rl), cr = sqrt(gam * pr / rr);
    if (2.0 / (gam - 1.0) * (cl + cr) <= ur - ul) return -1; /* vacuum forms */
    double lo = 0.0, hi = fmax(pl, pr);
    while (wave_f(gam, hi, rl, pl) + wave_f(gam, hi, rr, pr) + ur - ul < 0.0) hi *= 2.0;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = wave_f(gam, mid, rl, pl) + wave_f(gam, mid, rr, pr) + ur - ul;
        if (f < 0.0) lo = mid; else hi = mid;
    }
    *ps = 0.5 * (lo + hi);
    *us = 0.5 * (ul + ur) + 0.5 * (wave_f(gam, *ps, rr, pr) - wave_f(gam, *ps, rl, pl));
    return 0;
}

void orc_riemann_sample(double gam, double rl, double ul, double pl, double rr, double ur, double pr,
                        double ps, double us, double xi, double out[3])
{
    double g1 = gam - 1.0, gp = gam + 1.0;
    double cl = sqrt(gam * pl / rl), cr = sqrt(gam * pr / rr);
    if (xi <= us) {
        if (ps > pl) {
            double S = ul - cl * sqrt(gp / (2 * gam) * ps / pl + g1 / (2 * gam));
            if (xi <= S) { out[0] = rl; out[1] = ul; out[2] = pl; return; }
            out[0] = rl * (ps / pl + g1 / gp) / (g1 / gp * ps / pl + 1.0);
            out[1] = us; out[2] = ps;
        } else {
            double head = ul - cl, cs_ = cl * pow(ps / pl, g1 / (2 * gam)), tail = us - cs_;
            if (xi <= head) { out[0] = rl; out[1] = ul; out[2] = pl; return; }
            if (xi >= tail) { out[0] = rl * pow(ps / pl, 1.0 / gam); out[1] = us; out[2] = ps; return; }
            double c = 2.0 / gp * (cl + 0.5 * g1 * (ul - xi));
            out[1] = 2.0 / gp * (cl + 0.5 * g1 * ul + xi);
            out[0] = rl * pow(c / cl, 2.0 / g1);
            out[2] = pl * pow(c / cl, 2.0 * gam / g1);
        }
    } else {
        if (ps > pr) {
            double S = ur + cr * sqrt(gp / (2 * gam) * ps / pr + g1 / (2 * gam));
            if (xi >= S) { out[0] = rr; out[1] = ur; out[2] = pr; return; }
            out[0] = rr * (ps / pr + g1 / gp) / (g1 / gp * ps / pr + 1.0);
            out[1] = us; out[2] = ps;
        } else {
            double head = ur + cr, cs_ = cr * pow(ps / pr, g1 / (2 * gam)), tail = us + cs_;
            if (xi >= head) { out[0] = rr; out[1] = ur; out[2] = pr; return; }
            if (xi <= tail) { out[0] = rr * pow(ps / pr, 1.0 / gam); out[1] = us; out[2] = ps; return; }
            double c = 2.0 / gp * (cr - 0.5 * g1 * (ur - xi));
            out[1] = 2.0 / gp * (-cr + 0.5 * g1 * ur + xi);
            out[0] = rr * pow(c / cr, 2.0 / g1);
            out[2] = pr * pow(c / cr, 2.0 * gam / g1);
        }
    }
}
