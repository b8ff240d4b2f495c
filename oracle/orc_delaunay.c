/*
 * ORACLE (test infrastructure only; never linked into the CUDA library).
 *
 * Delaunay triangulation by point insertion (Section 2.1): points are added
 * one after another; the triangles whose circumscribed circle contains the
 * new point (exact, tie-broken in-circle test from orc_exact.c) are removed
 * and the hole is re-triangulated by joining its boundary to the new point
 * (Bowyer-Watson form of the insertion).  A large enclosing triangle of three
 * auxiliary vertices starts the construction; its vertices are numbered
 * n, n+1, n+2 in the output.
 *
 * Plain O(n log n)-ish code: points are inserted in a serpentine grid order
 * and located by walking from the last created triangle.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "orc.h"

typedef struct {
    int v[3];  /* counter-clockwise vertices */
    int nb[3]; /* nb[k]: triangle across the edge opposite v[k] (-1: none) */
    int alive;
} otri;

typedef struct {
    int n;
    const double *x, *y;
    otri *t;
    int nt, cap;
    int *freel;
    int nfree;
} odt;

static int new_tri(odt *d)
{
    if (d->nfree > 0) return d->freel[--d->nfree];
    if (d->nt == d->cap) {
        d->cap = d->cap * 2 + 16;
        d->t = (otri *)realloc(d->t, sizeof(otri) * d->cap);
        d->freel = (int *)realloc(d->freel, sizeof(int) * d->cap);
    }
    return d->nt++;
}

static double PX(const odt *d, int i) { return d->x[i]; }
static double PY(const odt *d, int i) { return d->y[i]; }

typedef struct { long key; int idx; } okey;

static int cmp_key(const void *a, const void *b)
{
    const okey *p = (const okey *)a, *q = (const okey *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx - q->idx;
}

/* Triangulate n distinct points.  On success returns 0 and sets *tris to a
   malloc'ed array of 3*(*ntri) vertex ids (ids >= n are the auxiliary
   vertices).  Returns -2 if two points coincide. */
int orc_delaunay(int n, const double *xin, const double *yin, int *ntri, int **tris)
{
    *ntri = 0;
    *tris = NULL;
    if (n < 1) return -1;
    double xmin = xin[0], xmax = xin[0], ymin = yin[0], ymax = yin[0];
    for (int i = 1; i < n; i++) {
        if (xin[i] < xmin) xmin = xin[i];
        if (xin[i] > xmax) xmax = xin[i];
        if (yin[i] < ymin) ymin = yin[i];
        if (yin[i] > ymax) ymax = yin[i];
    }
    double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
    double M = fmax(xmax - xmin, ymax - ymin);
    if (M <= 0) M = 1.0;
    double *x = (double *)malloc(sizeof(double) * (n + 3));
    double *y = (double *)malloc(sizeof(double) * (n + 3));
    memcpy(x, xin, sizeof(double) * n);
    memcpy(y, yin, sizeof(double) * n);
    /* enclosing triangle, far outside the bounding box */
    x[n] = cx - 40.0 * M; y[n] = cy - 20.0 * M;
    x[n + 1] = cx + 40.0 * M; y[n + 1] = cy - 20.0 * M;
    x[n + 2] = cx; y[n + 2] = cy + 40.0 * M;

    odt d;
    memset(&d, 0, sizeof(d));
    d.n = n;
    d.x = x;
    d.y = y;
    int t0 = new_tri(&d);
    d.t[t0].v[0] = n; d.t[t0].v[1] = n + 1; d.t[t0].v[2] = n + 2;
    d.t[t0].nb[0] = d.t[t0].nb[1] = d.t[t0].nb[2] = -1;
    d.t[t0].alive = 1;

    /* serpentine grid order */
    int g = (int)ceil(sqrt((double)n / 4.0));
    if (g < 1) g = 1;
    okey *ord = (okey *)malloc(sizeof(okey) * n);
    for (int i = 0; i < n; i++) {
        double fx = (xin[i] - xmin) / (xmax - xmin > 0 ? xmax - xmin : 1.0);
        double fy = (yin[i] - ymin) / (ymax - ymin > 0 ? ymax - ymin : 1.0);
        int gx = (int)(fx * g), gy = (int)(fy * g);
        if (gx >= g) gx = g - 1;
        if (gy >= g) gy = g - 1;
        if (gy & 1) gx = g - 1 - gx;
        ord[i].key = (long)gy * g + gx;
        ord[i].idx = i;
    }
    qsort(ord, n, sizeof(okey), cmp_key);

    int *mark = (int *)calloc(1, sizeof(int));
    int markcap = 0;
    int *by_a = (int *)malloc(sizeof(int) * (n + 3));
    int *by_b = (int *)malloc(sizeof(int) * (n + 3));
    int *stack = NULL, *cav = NULL, *bnd_t = NULL, *bnd_k = NULL;
    int scap = 0;
    int last = t0;
    int stamp = 0;
    int err = 0;

    for (int oi = 0; oi < n && !err; oi++) {
        int p = ord[oi].idx;
        double px = x[p], py = y[p];
        /* --- locate by a visibility walk --- */
        int t = last;
        long steps = 0;
        for (;;) {
            otri *T = &d.t[t];
            int moved = 0;
            for (int k = 0; k < 3; k++) {
                int a = T->v[(k + 1) % 3], b = T->v[(k + 2) % 3];
                if (orc_orient(PX(&d, a), PY(&d, a), PX(&d, b), PY(&d, b), px, py) < 0) {
                    t = T->nb[k];
                    moved = 1;
                    break;
                }
            }
            if (!moved) break;
            if (t < 0 || ++steps > 4L * (d.nt + 10)) { err = -3; break; }
        }
        if (err) break;
        for (int k = 0; k < 3; k++) {
            int q = d.t[t].v[k];
            if (x[q] == px && y[q] == py) { err = -2; break; }
        }
        if (err) break;
        /* --- cavity: triangles whose circle contains p --- */
        if (d.nt + 8 > markcap) {
            int nc = 2 * (d.nt + 8);
            mark = (int *)realloc(mark, sizeof(int) * nc);
            for (int i = markcap; i < nc; i++) mark[i] = 0;
            markcap = nc;
        }
        if (scap < d.nt + 8) {
            scap = 2 * (d.nt + 8);
            stack = (int *)realloc(stack, sizeof(int) * scap);
            cav = (int *)realloc(cav, sizeof(int) * scap);
            bnd_t = (int *)realloc(bnd_t, sizeof(int) * scap);
            bnd_k = (int *)realloc(bnd_k, sizeof(int) * scap);
        }
        stamp += 2; /* mark == stamp: in cavity; stamp+1: tested, outside */
        int ns = 0, nc = 0, nbnd = 0;
        stack[ns++] = t;
        mark[t] = stamp;
        while (ns > 0) {
            int c = stack[--ns];
            cav[nc++] = c;
            for (int k = 0; k < 3; k++) {
                int o = d.t[c].nb[k];
                if (o < 0 || mark[o] == stamp || mark[o] == stamp + 1) continue;
                otri *O = &d.t[o];
                if (orc_incircle_sos(x[O->v[0]], y[O->v[0]], x[O->v[1]], y[O->v[1]], x[O->v[2]],
                                     y[O->v[2]], px, py) > 0) {
                    mark[o] = stamp;
                    stack[ns++] = o;
                } else {
                    mark[o] = stamp + 1;
                }
            }
        }
        for (int ci = 0; ci < nc; ci++) {
            int c = cav[ci];
            for (int k = 0; k < 3; k++) {
                int o = d.t[c].nb[k];
                if (o >= 0 && mark[o] == stamp) continue;
                bnd_t[nbnd] = c;
                bnd_k[nbnd] = k;
                nbnd++;
            }
        }
        /* --- new triangles (p, a, b) on every boundary edge --- */
        int *newt = stack; /* reuse */
        /* copy the boundary edges out, then free the cavity so its slots can be reused */
        int *ea = (int *)malloc(sizeof(int) * 3 * (nbnd + 1));
        for (int bi = 0; bi < nbnd; bi++) {
            int c = bnd_t[bi], k = bnd_k[bi];
            ea[3 * bi] = d.t[c].v[(k + 1) % 3];
            ea[3 * bi + 1] = d.t[c].v[(k + 2) % 3];
            ea[3 * bi + 2] = d.t[c].nb[k];
        }
        for (int ci = 0; ci < nc; ci++) {
            d.t[cav[ci]].alive = 0;
            d.freel[d.nfree++] = cav[ci];
        }
        for (int bi = 0; bi < nbnd; bi++) {
            int nt_ = new_tri(&d);
            newt[bi] = nt_;
            otri *N = &d.t[nt_];
            N->v[0] = p; N->v[1] = ea[3 * bi]; N->v[2] = ea[3 * bi + 1];
            N->nb[0] = ea[3 * bi + 2];
            N->nb[1] = N->nb[2] = -1;
            N->alive = 1;
            by_a[N->v[1]] = nt_;
            by_b[N->v[2]] = nt_;
        }
        for (int bi = 0; bi < nbnd; bi++) {
            int nt_ = newt[bi];
            otri *N = &d.t[nt_];
            int a = N->v[1], b = N->v[2];
            N->nb[2] = by_b[a]; /* edge p-a is shared with the triangle ending at a */
            N->nb[1] = by_a[b]; /* edge b-p is shared with the triangle starting at b */
            int o = N->nb[0];
            if (o >= 0) {
                otri *O = &d.t[o];
                for (int k = 0; k < 3; k++)
                    if (O->v[(k + 1) % 3] == b && O->v[(k + 2) % 3] == a) O->nb[k] = nt_;
            }
        }
        free(ea);
        last = newt[0];
        if (d.nt + 8 > markcap) {
            int ncap = 2 * (d.nt + 8);
            mark = (int *)realloc(mark, sizeof(int) * ncap);
            for (int i = markcap; i < ncap; i++) mark[i] = 0;
            markcap = ncap;
        }
    }

    if (!err) {
        int cnt = 0;
        for (int i = 0; i < d.nt; i++) cnt += d.t[i].alive;
        int *out = (int *)malloc(sizeof(int) * 3 * (cnt > 0 ? cnt : 1));
        int j = 0;
        for (int i = 0; i < d.nt; i++) {
            if (!d.t[i].alive) continue;
            out[3 * j] = d.t[i].v[0];
            out[3 * j + 1] = d.t[i].v[1];
            out[3 * j + 2] = d.t[i].v[2];
            j++;
        }
        *ntri = cnt;
        *tris = out;
    }
    free(ord); free(mark); free(by_a); free(by_b); free(stack); free(cav); free(bnd_t); free(bnd_k);
    free(d.t); free(d.freel); free(x); free(y);
    return err;
}

void orc_free(void *p) { free(p); }
