// Host tessellation: ghost images, Delaunay by point insertion with Lawson
// flips, band check, rings and the de-duplicated Voronoi edge list.
// See mesh.h.
#include "mesh.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "predicates.h"

namespace rich {

// ---------------------------------------------------------------------------
// Hilbert order

static uint32_t hilbert_index(uint32_t x, uint32_t y)
{
    // position along the Hilbert curve of a 2^16 x 2^16 grid: at each level the
    // quadrant contributes (3*rx)^ry and the remaining coordinates are rotated
    // into that quadrant's frame
    const uint32_t n = 1u << 16;
    uint32_t d = 0;
    for (uint32_t s = n >> 1; s > 0; s >>= 1) {
        uint32_t rx = (x & s) ? 1u : 0u;
        uint32_t ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = n - 1 - x;
                y = n - 1 - y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

static void radix_sort(std::vector<uint32_t> &keys, std::vector<int32_t> &idx, std::vector<uint32_t> &tk,
                       std::vector<int32_t> &ti)
{
    size_t n = keys.size();
    tk.resize(n);
    ti.resize(n);
    for (int pass = 0; pass < 2; pass++) {
        int shift = 16 * pass;
        std::vector<uint32_t> cnt(65537, 0);
        for (size_t i = 0; i < n; i++) cnt[((keys[i] >> shift) & 0xffffu) + 1]++;
        for (int b = 0; b < 65536; b++) cnt[b + 1] += cnt[b];
        for (size_t i = 0; i < n; i++) {
            uint32_t b = (keys[i] >> shift) & 0xffffu;
            uint32_t pos = cnt[b]++;
            tk[pos] = keys[i];
            ti[pos] = idx[i];
        }
        keys.swap(tk);
        idx.swap(ti);
    }
}

void hilbert_order(int32_t n, const double *x, const double *y, std::vector<int32_t> &order)
{
    std::vector<uint32_t> keys(n), tk;
    std::vector<int32_t> ti;
    order.resize(n);
    if (n == 0) return;
    double xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0];
    for (int32_t i = 1; i < n; i++) {
        xmin = std::min(xmin, x[i]); xmax = std::max(xmax, x[i]);
        ymin = std::min(ymin, y[i]); ymax = std::max(ymax, y[i]);
    }
    double sx = xmax > xmin ? 65535.0 / (xmax - xmin) : 0.0;
    double sy = ymax > ymin ? 65535.0 / (ymax - ymin) : 0.0;
    for (int32_t i = 0; i < n; i++) {
        uint32_t gx = (uint32_t)std::min(65535.0, std::max(0.0, (x[i] - xmin) * sx));
        uint32_t gy = (uint32_t)std::min(65535.0, std::max(0.0, (y[i] - ymin) * sy));
        keys[i] = hilbert_index(gx, gy);
        order[i] = i;
    }
    radix_sort(keys, order, tk, ti);
}

// ---------------------------------------------------------------------------
// Delaunay by point insertion + Lawson flips

int Delaunay::incircle(int32_t t, int32_t d) const
{
    const Tri &T = tris[t];
    return incircle_sos(px_[T.v[0]], py_[T.v[0]], px_[T.v[1]], py_[T.v[1]], px_[T.v[2]], py_[T.v[2]], px_[d],
                        py_[d]);
}

void Delaunay::set_nb(int32_t t, int32_t old_nb, int32_t new_nb)
{
    if (t < 0) return;
    Tri &T = tris[t];
    for (int k = 0; k < 3; k++)
        if (T.nb[k] == old_nb) {
            T.nb[k] = new_nb;
            return;
        }
}

// Walk from the hint towards p.  Returns 0 (p strictly inside t), 1 (p on the
// edge opposite vertex 'edge' of t), -2 (p coincides with a vertex), -3 (lost).
int Delaunay::locate(int32_t p, int32_t &t_out, int &edge)
{
    int32_t t = hint_;
    const double qx = px_[p], qy = py_[p];
    size_t limit = 4 * tris.size() + 64;
    for (size_t it = 0; it < limit; it++) {
        const Tri &T = tris[t];
        int o[3];
        rng_ = rng_ * 1664525u + 1013904223u;
        int start = (int)((rng_ >> 16) % 3u);
        bool moved = false;
        for (int q = 0; q < 3; q++) {
            int k = (start + q) % 3;
            int32_t a = T.v[(k + 1) % 3], b = T.v[(k + 2) % 3];
            o[k] = orient2d(px_[a], py_[a], px_[b], py_[b], qx, qy);
            if (o[k] < 0) {
                t = T.nb[k];
                moved = true;
                break;
            }
        }
        if (!moved) {
            int zeros = (o[0] == 0) + (o[1] == 0) + (o[2] == 0);
            t_out = t;
            if (zeros == 0) return 0;
            if (zeros == 1) {
                edge = o[0] == 0 ? 0 : (o[1] == 0 ? 1 : 2);
                return 1;
            }
            return -2;
        }
        if (t < 0) return -3;
    }
    return -3;
}

void Delaunay::insert_inside(int32_t t, int32_t p)
{
    Tri old = tris[t];
    int32_t a = old.v[0], b = old.v[1], c = old.v[2];
    int32_t na = old.nb[0], nbb = old.nb[1], nc = old.nb[2];
    int32_t t1 = (int32_t)tris.size(), t2 = t1 + 1;
    tris.resize(tris.size() + 2);
    tris[t] = Tri{{p, b, c}, {na, t1, t2}};
    tris[t1] = Tri{{p, c, a}, {nbb, t2, t}};
    tris[t2] = Tri{{p, a, b}, {nc, t, t1}};
    set_nb(nbb, t, t1);
    set_nb(nc, t, t2);
    stack_.push_back(t);
    stack_.push_back(t1);
    stack_.push_back(t2);
    legalize(p);
    hint_ = t;
}

void Delaunay::insert_on_edge(int32_t t, int k, int32_t p)
{
    Tri T = tris[t];
    int32_t a = T.v[k], b = T.v[(k + 1) % 3], c = T.v[(k + 2) % 3];
    int32_t t_ca = T.nb[(k + 1) % 3], t_ab = T.nb[(k + 2) % 3];
    int32_t u = T.nb[k];
    Tri U = tris[u];
    int m = 0;
    while (U.nb[m] != t) m++;
    int32_t d = U.v[m];
    int32_t u_bd = U.nb[(m + 1) % 3], u_dc = U.nb[(m + 2) % 3];
    int32_t A = t, Cc = u;
    int32_t B = (int32_t)tris.size(), D = B + 1;
    tris.resize(tris.size() + 2);
    tris[A] = Tri{{p, c, a}, {t_ca, B, Cc}};
    tris[B] = Tri{{p, a, b}, {t_ab, D, A}};
    tris[Cc] = Tri{{p, d, c}, {u_dc, A, D}};
    tris[D] = Tri{{p, b, d}, {u_bd, Cc, B}};
    set_nb(t_ab, t, B);
    set_nb(u_bd, u, D);
    stack_.push_back(A);
    stack_.push_back(B);
    stack_.push_back(Cc);
    stack_.push_back(D);
    legalize(p);
    hint_ = A;
}

// Every triangle on the stack has p as v[0]; test the edge opposite p.
void Delaunay::legalize(int32_t p)
{
    while (!stack_.empty()) {
        int32_t t = stack_.back();
        stack_.pop_back();
        Tri &T = tris[t];
        int32_t u = T.nb[0];
        if (u < 0) continue;
        Tri &U = tris[u];
        int m = 0;
        while (m < 3 && U.nb[m] != t) m++;
        if (m == 3) continue;
        int32_t d = U.v[m];
        if (incircle(t, d) <= 0) continue;
        // flip edge (b, c) of T = (p, b, c) and U = (d, c, b) into (b, d)
        int32_t b = T.v[1], c = T.v[2];
        int32_t T_cp = T.nb[1], T_pb = T.nb[2];
        int32_t u_bd = U.nb[(m + 1) % 3], u_dc = U.nb[(m + 2) % 3];
        tris[t] = Tri{{p, b, d}, {u_bd, u, T_pb}};
        tris[u] = Tri{{p, d, c}, {u_dc, T_cp, t}};
        set_nb(u_bd, u, t);
        set_nb(T_cp, t, u);
        stack_.push_back(t);
        stack_.push_back(u);
    }
}

int Delaunay::build(const double *x, const double *y, int32_t np)
{
    tris.clear();
    stack_.clear();
    if (np < 1) return -3;
    px_.assign(x, x + np);
    py_.assign(y, y + np);
    double xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0];
    for (int32_t i = 1; i < np; i++) {
        xmin = std::min(xmin, x[i]); xmax = std::max(xmax, x[i]);
        ymin = std::min(ymin, y[i]); ymax = std::max(ymax, y[i]);
    }
    double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
    double M = std::max(xmax - xmin, ymax - ymin);
    if (!(M > 0)) M = 1.0;
    // enclosing triangle far outside the bounding box
    px_.push_back(cx - 64.0 * M); py_.push_back(cy - 32.0 * M);
    px_.push_back(cx + 64.0 * M); py_.push_back(cy - 32.0 * M);
    px_.push_back(cx);            py_.push_back(cy + 64.0 * M);
    tris.reserve((size_t)2 * np + 16);
    tris.push_back(Tri{{np, np + 1, np + 2}, {-1, -1, -1}});
    hint_ = 0;
    hilbert_order(np, x, y, order_);
    for (int32_t oi = 0; oi < np; oi++) {
        int32_t p = order_[oi];
        int32_t t = -1;
        int edge = -1;
        int r = locate(p, t, edge);
        if (r == -2) return -2;
        if (r < 0) return -3;
        if (r == 0) insert_inside(t, p);
        else insert_on_edge(t, edge, p);
    }
    return 0;
}

// ---------------------------------------------------------------------------
// ghosts + rings + edges

static inline double image_coord(double v, double lo, double hi, int flip, int shift)
{
    if (flip < 0) return (lo + lo) - v;
    if (flip > 0) return (hi + hi) - v;
    if (shift > 0) return v + (hi - lo);
    if (shift < 0) return v - (hi - lo);
    return v;
}

static void make_ghosts(const BoxConfig &box, int32_t n, const double *x, const double *y, double w, HostMesh &m)
{
    m.gx.clear(); m.gy.clear(); m.ghost_src.clear(); m.ghost_xf.clear(); m.ghost_shift.clear();
    const double lox = box.x0 - w, hix = box.x1 + w, loy = box.y0 - w, hiy = box.y1 + w;
    for (int32_t i = 0; i < n; i++) {
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++) {
                if (a == 0 && b == 0) continue;
                int fx = 0, fy = 0, sx = 0, sy = 0;
                if (box.boundary == 1) { sx = a; sy = b; }
                else { fx = a; fy = b; }
                double X = image_coord(x[i], box.x0, box.x1, fx, sx);
                double Y = image_coord(y[i], box.y0, box.y1, fy, sy);
                if (X < lox || X > hix || Y < loy || Y > hiy) continue;
                m.gx.push_back(X);
                m.gy.push_back(Y);
                m.ghost_src.push_back(i);
                m.ghost_xf.push_back((fx ? XF_MIRROR_X : 0) | (fy ? XF_MIRROR_Y : 0));
                m.ghost_shift.push_back((sx + 1) + 3 * (sy + 1));
            }
    }
    m.g = (int32_t)m.gx.size();
}

int build_host_mesh(const BoxConfig &box, int32_t n, const double *x, const double *y, Delaunay &dt, HostMesh &m)
{
    const double Lx = box.x1 - box.x0, Ly = box.y1 - box.y0;
    const double h = std::sqrt(Lx * Ly / std::max(n, 1));
    const double wmax = std::min(Lx, Ly);
    double w = std::min(5.0 * h, wmax);
    std::vector<double> X, Y;
    std::vector<int32_t> vtri, tmap;
    m.n = n;
    m.attempts = 0;
    for (;;) {
        m.attempts++;
        make_ghosts(box, n, x, y, w, m);
        const int32_t np = n + m.g;
        X.resize(np);
        Y.resize(np);
        std::memcpy(X.data(), x, sizeof(double) * n);
        std::memcpy(Y.data(), y, sizeof(double) * n);
        std::memcpy(X.data() + n, m.gx.data(), sizeof(double) * m.g);
        std::memcpy(Y.data() + n, m.gy.data(), sizeof(double) * m.g);
        int rc = dt.build(X.data(), Y.data(), np);
        if (rc) return rc;
        const std::vector<Tri> &T = dt.tris;
        // compact the triangles touching a real point and check the band
        tmap.assign(T.size(), -1);
        m.tri.clear();
        bool ok = true;
        const double lox = box.x0 - w, hix = box.x1 + w, loy = box.y0 - w, hiy = box.y1 + w;
        for (size_t t = 0; t < T.size() && ok; t++) {
            const int32_t *v = T[t].v;
            if (v[0] >= n && v[1] >= n && v[2] >= n) continue;
            if (v[0] >= np || v[1] >= np || v[2] >= np) { ok = false; break; }
            double ax = X[v[0]], ay = Y[v[0]];
            double bx = X[v[1]] - ax, by = Y[v[1]] - ay, cx = X[v[2]] - ax, cy = Y[v[2]] - ay;
            double d = 2.0 * (bx * cy - by * cx);
            double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
            double ux = (cy * b2 - by * c2) / d, uy = (bx * c2 - cx * b2) / d;
            double R = std::sqrt(ux * ux + uy * uy) * (1.0 + 1e-9) + 1e-12 * (Lx + Ly);
            ux += ax;
            uy += ay;
            if (!(ux - R >= lox && ux + R <= hix && uy - R >= loy && uy + R <= hiy)) { ok = false; break; }
            tmap[t] = (int32_t)(m.tri.size() / 3);
            m.tri.push_back(v[0]);
            m.tri.push_back(v[1]);
            m.tri.push_back(v[2]);
        }
        if (!ok) {
            if (w >= wmax) return -4;
            w = std::min(2.0 * w, wmax);
            continue;
        }
        m.band = w;
        // one incident triangle per real point
        vtri.assign(n, -1);
        for (size_t t = 0; t < T.size(); t++) {
            if (tmap[t] < 0) continue;
            for (int k = 0; k < 3; k++)
                if (T[t].v[k] < n) vtri[T[t].v[k]] = (int32_t)t;
        }
        // rings: rotate counter-clockwise about each real point
        m.cell_ptr.assign(n + 1, 0);
        m.slot_nb.clear();
        m.slot_tri.clear();
        for (int32_t i = 0; i < n; i++) {
            m.cell_ptr[i] = (int32_t)m.slot_nb.size();
            int32_t t0 = vtri[i];
            if (t0 < 0) return -3;
            int32_t t = t0;
            int guard = 0;
            do {
                const Tri &tr = T[t];
                int k = tr.v[0] == i ? 0 : (tr.v[1] == i ? 1 : 2);
                m.slot_nb.push_back(tr.v[(k + 1) % 3]);
                m.slot_tri.push_back(tmap[t]);
                t = tr.nb[(k + 1) % 3];
                if (t < 0 || tmap[t] < 0 || ++guard > 4096) return -3;
            } while (t != t0);
        }
        m.cell_ptr[n] = (int32_t)m.slot_nb.size();
        // edges, each physical edge once
        const size_t S = m.slot_nb.size();
        m.slot_edge.assign(S, -1);
        m.edge_l.clear(); m.edge_r.clear(); m.edge_ta.clear(); m.edge_tb.clear();
        for (int32_t i = 0; i < n; i++) {
            const int32_t lo = m.cell_ptr[i], deg = m.cell_ptr[i + 1] - lo;
            for (int32_t k = 0; k < deg; k++) {
                const int32_t s = lo + k;
                if (m.slot_edge[s] >= 0) continue;
                const int32_t j = m.slot_nb[s];
                int32_t partner_cell = -1, partner_nb = -1;
                if (j < n) {
                    if (j < i) return -3;  // should have been assigned from j's ring
                    partner_cell = j;
                    partner_nb = i;
                } else {
                    const int32_t gq = j - n;
                    if (box.boundary == 1) {
                        const int32_t src = m.ghost_src[gq];
                        const int32_t sh = m.ghost_shift[gq];
                        const int32_t sx = sh % 3 - 1, sy = sh / 3 - 1;
                        if (src < i) return -3;
                        if (src == i && (sy < 0 || (sy == 0 && sx < 0))) continue;  // created by the +shift slot
                        partner_cell = src;
                        partner_nb = -((-sx + 1) + 3 * (-sy + 1)) - 1;  // ghost of i with the opposite shift
                    }
                }
                const int32_t e = (int32_t)m.edge_l.size();
                m.edge_l.push_back(i);
                m.edge_r.push_back(j);
                m.edge_ta.push_back(m.slot_tri[lo + (k + deg - 1) % deg]);
                m.edge_tb.push_back(m.slot_tri[s]);
                m.slot_edge[s] = 2 * e;
                if (partner_cell >= 0) {
                    const int32_t plo = m.cell_ptr[partner_cell], phi = m.cell_ptr[partner_cell + 1];
                    int32_t found = -1;
                    for (int32_t q = plo; q < phi; q++) {
                        const int32_t c = m.slot_nb[q];
                        if (partner_nb >= 0) {
                            if (c == partner_nb) { found = q; break; }
                        } else if (c >= n) {
                            const int32_t want = -partner_nb - 1;
                            if (m.ghost_src[c - n] == i && m.ghost_shift[c - n] == want && q != s) {
                                found = q;
                                break;
                            }
                        }
                    }
                    if (found < 0 || m.slot_edge[found] >= 0) return -3;
                    m.slot_edge[found] = 2 * e + 1;
                }
            }
        }
        for (size_t s = 0; s < S; s++)
            if (m.slot_edge[s] < 0) return -3;
        return 0;
    }
}

}  // namespace rich
