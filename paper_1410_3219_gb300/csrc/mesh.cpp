// Host tessellation: ghost images, Delaunay by point insertion with Lawson
// flips, band check, rings and the de-duplicated Voronoi edge list.
// See mesh.h.
#include "mesh.h"

#include <algorithm>
#include <chrono>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>

#include "predicates.h"
#include "threadpool.h"

namespace rich {

// ---------------------------------------------------------------------------
// Hilbert order

static uint32_t hilbert_index(uint32_t x, uint32_t y, int levels)
{
    // position along the Hilbert curve of a 2^levels x 2^levels grid: at each
    // level the quadrant contributes (3*rx)^ry and the remaining coordinates
    // are rotated into that quadrant's frame
    // (branch-free: the reflection n-1-v is v ^ (n-1) for v < n)
    const uint32_t top = (1u << levels) - 1u;
    uint32_t d = 0;
    for (int k = levels - 1; k >= 0; k--) {
        const uint32_t rx = (x >> k) & 1u, ry = (y >> k) & 1u;
        d += ((3u * rx) ^ ry) << (2 * k);
        const uint32_t flip = 0u - (rx & (ry ^ 1u));
        x ^= flip & top;
        y ^= flip & top;
        const uint32_t sw = (x ^ y) & (0u - (ry ^ 1u));
        x ^= sw;
        y ^= sw;
    }
    return d;
}

// LSD radix sort of (key, index) pairs on the low `bits` bits, 11 bits a pass
static void radix_sort(std::vector<uint32_t> &keys, std::vector<int32_t> &idx, int bits)
{
    const size_t n = keys.size();
    std::vector<uint32_t> tk(n);
    std::vector<int32_t> ti(n);
    constexpr int kDigit = 11;
    std::vector<uint32_t> cnt((1u << kDigit) + 1);
    for (int shift = 0; shift < bits; shift += kDigit) {
        std::fill(cnt.begin(), cnt.end(), 0u);
        const uint32_t mask = (1u << kDigit) - 1u;
        for (size_t i = 0; i < n; i++) cnt[((keys[i] >> shift) & mask) + 1]++;
        for (uint32_t b = 0; b < mask + 1; b++) cnt[b + 1] += cnt[b];
        for (size_t i = 0; i < n; i++) {
            const uint32_t pos = cnt[(keys[i] >> shift) & mask]++;
            tk[pos] = keys[i];
            ti[pos] = idx[i];
        }
        keys.swap(tk);
        idx.swap(ti);
    }
}

void hilbert_order(int32_t n, const double *x, const double *y, std::vector<int32_t> &order)
{
    order.resize(n);
    if (n == 0) return;
    // resolution: about 2^3 grid cells per point along each axis is plenty
    // for locality; the curve index then needs 2 * levels bits
    int levels = 4;
    while (levels < 16 && (int64_t)1 << (2 * (levels - 3)) < (int64_t)n) levels++;
    std::vector<uint32_t> keys(n);
    double xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0];
    for (int32_t i = 1; i < n; i++) {
        xmin = std::min(xmin, x[i]); xmax = std::max(xmax, x[i]);
        ymin = std::min(ymin, y[i]); ymax = std::max(ymax, y[i]);
    }
    const double top = (double)((1u << levels) - 1u);
    double sx = xmax > xmin ? top / (xmax - xmin) : 0.0;
    double sy = ymax > ymin ? top / (ymax - ymin) : 0.0;
    for (int32_t i = 0; i < n; i++) {
        uint32_t gx = (uint32_t)std::min(top, std::max(0.0, (x[i] - xmin) * sx));
        uint32_t gy = (uint32_t)std::min(top, std::max(0.0, (y[i] - ymin) * sy));
        keys[i] = hilbert_index(gx, gy, levels);
        order[i] = i;
    }
    radix_sort(keys, order, 2 * levels);
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

// two triangle slots: freed ones first (a vertex removal frees two)
void Delaunay::alloc2(int32_t &a, int32_t &b)
{
    if (free_.size() >= 2) {
        a = free_.back();
        free_.pop_back();
        b = free_.back();
        free_.pop_back();
        return;
    }
    a = (int32_t)tris.size();
    b = a + 1;
    tris.resize(tris.size() + 2);
}

void Delaunay::insert_inside(int32_t t, int32_t p)
{
    Tri old = tris[t];
    int32_t a = old.v[0], b = old.v[1], c = old.v[2];
    int32_t na = old.nb[0], nbb = old.nb[1], nc = old.nb[2];
    int32_t t1, t2;
    alloc2(t1, t2);
    tris[t] = Tri{{p, b, c}, {na, t1, t2}};
    tris[t1] = Tri{{p, c, a}, {nbb, t2, t}};
    tris[t2] = Tri{{p, a, b}, {nc, t, t1}};
    note(t);
    note(t1);
    note(t2);
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
    int32_t B, D;
    alloc2(B, D);
    tris[A] = Tri{{p, c, a}, {t_ca, B, Cc}};
    tris[B] = Tri{{p, a, b}, {t_ab, D, A}};
    tris[Cc] = Tri{{p, d, c}, {u_dc, A, D}};
    tris[D] = Tri{{p, b, d}, {u_bd, Cc, B}};
    note(A);
    note(B);
    note(Cc);
    note(D);
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
        note(t);
        note(u);
        set_nb(u_bd, u, t);
        set_nb(T_cp, t, u);
        stack_.push_back(t);
        stack_.push_back(u);
    }
}

int Delaunay::build(const double *x, const double *y, int32_t np)
{
    log_.clear();
    log_all_ = true;
    tris.clear();
    stack_.clear();
    free_.clear();
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
    corner_ = np;
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

// Flip the edge opposite vertex k of triangle t: (a, b, c) and (d, c, b)
// become (a, b, d) and (a, d, c), in the slots of t and of the neighbour.
void Delaunay::flip(int32_t t, int k)
{
    const Tri T = tris[t];
    const int32_t u = T.nb[k];
    const Tri U = tris[u];
    int m = 0;
    while (U.nb[m] != t) m++;
    const int32_t a = T.v[k], b = T.v[(k + 1) % 3], c = T.v[(k + 2) % 3], d = U.v[m];
    const int32_t t_ca = T.nb[(k + 1) % 3], t_ab = T.nb[(k + 2) % 3];
    const int32_t u_bd = U.nb[(m + 1) % 3], u_dc = U.nb[(m + 2) % 3];
    tris[t] = Tri{{a, b, d}, {u_bd, u, t_ab}};
    tris[u] = Tri{{a, d, c}, {u_dc, t_ca, t}};
    note(t);
    note(u);
    set_nb(u_bd, u, t);
    set_nb(t_ca, t, u);
}

// whether that flip leaves two counter-clockwise triangles
bool Delaunay::flip_ok(int32_t t, int k) const
{
    const Tri &T = tris[t];
    const int32_t u = T.nb[k];
    if (u < 0) return false;
    const Tri &U = tris[u];
    int m = 0;
    while (m < 3 && U.nb[m] != t) m++;
    if (m == 3) return false;
    const int32_t a = T.v[k], b = T.v[(k + 1) % 3], c = T.v[(k + 2) % 3], d = U.v[m];
    return orient2d(px_[a], py_[a], px_[b], py_[b], px_[d], py_[d]) > 0 &&
           orient2d(px_[a], py_[a], px_[d], py_[d], px_[c], py_[c]) > 0;
}

// Take interior vertex v (in live triangle t) out: flip its edges away while
// it has more than three, then merge its three triangles into the one of
// its neighbours.  Frees two triangle slots.
bool Delaunay::remove_vertex(int32_t v, int32_t t)
{
    std::vector<int32_t> st, lk;  // v's triangles and neighbours, counter-clockwise
    for (int guard = 0; guard < 256; guard++) {
        st.clear();
        lk.clear();
        int32_t cur = t;
        for (int step = 0; step < 64; step++) {
            const Tri &T = tris[cur];
            int j = 0;
            while (j < 3 && T.v[j] != v) j++;
            if (j == 3) return false;
            st.push_back(cur);
            lk.push_back(T.v[(j + 1) % 3]);
            cur = T.nb[(j + 1) % 3];  // across edge (v, T.v[j + 2])
            if (cur < 0) return false;  // v on the hull
            if (cur == t) break;
        }
        if (cur != t) return false;
        const int d = (int)st.size();
        if (d == 3) {
            const int32_t l0 = lk[0], l1 = lk[1], l2 = lk[2];
            if (orient2d(px_[l0], py_[l0], px_[l1], py_[l1], px_[l2], py_[l2]) <= 0) return false;
            int32_t o[3];
            for (int i = 0; i < 3; i++) {
                const Tri &T = tris[st[i]];
                int j = 0;
                while (T.v[j] != v) j++;
                o[i] = T.nb[j];  // across (l_i, l_i+1)
            }
            tris[st[0]] = Tri{{l0, l1, l2}, {o[1], o[2], o[0]}};
            note(st[0]);
            touched_.push_back(st[0]);
            set_nb(o[1], st[1], st[0]);
            set_nb(o[2], st[2], st[0]);
            for (int i = 1; i < 3; i++) {
                tris[st[i]] = Tri{{-1, -1, -1}, {-1, -1, -1}};
                free_.push_back(st[i]);
            }
            hint_ = st[0];
            return true;
        }
        // an edge (v, lk[i]) whose flip keeps both triangles counter-clockwise
        bool done = false;
        for (int i = 0; i < d && !done; i++) {
            const Tri &T = tris[st[i]];
            int j = 0;
            while (T.v[j] != v) j++;
            const int k = (j + 2) % 3;  // opposite lk[i + 1]: the edge (v, lk[i])
            if (flip_ok(st[i], k)) {
                touched_.push_back(st[i]);
                touched_.push_back(tris[st[i]].nb[k]);
                flip(st[i], k);
                t = st[i];  // still has v
                done = true;
            }
        }
        if (!done) return false;
    }
    return false;
}

int Delaunay::insert_at(int32_t v)
{
    int32_t t = -1;
    int edge = -1;
    const int r = locate(v, t, edge);
    if (r == -2) return -2;
    if (r < 0) return -3;
    if (r == 0) insert_inside(t, v);
    else insert_on_edge(t, edge, v);
    return 0;
}

bool Delaunay::move_all(const std::vector<double> &nx, const std::vector<double> &ny, int32_t max_back)
{
    const int32_t NV = size();
    old_x_.assign(px_.begin(), px_.end());
    old_y_.assign(py_.begin(), py_.end());
    const std::vector<double> &ox = old_x_, &oy = old_y_;
    for (int32_t v = 0; v < NV; v++)
        if (!is_corner(v)) {
            px_[v] = nx[v];
            py_[v] = ny[v];
        }
    std::vector<uint8_t> &back = back_;
    back.assign(NV, 0);
    std::vector<int32_t> &S = back_list_;
    S.clear();
    // where[v]: a triangle holding v, for the vertices put back
    std::vector<int32_t> &where = where_;
    where.assign(NV, -1);
    // The vertices of a triangle that the new positions turn over go back to
    // their old positions (they are taken out and inserted again below).  A
    // vertex put back can turn over only triangles of its own star, so after
    // one pass over all triangles only the stars of the vertices put back
    // are tested again (S doubles as the queue of stars to test).
    auto put_back = [&](int32_t t) -> bool {
        const Tri &T = tris[t];
        for (int k = 0; k < 3; k++) {
            const int32_t v = T.v[k];
            if (is_corner(v)) return false;
            if (back[v]) continue;
            back[v] = 1;
            S.push_back(v);
            where[v] = t;
            px_[v] = ox[v];
            py_[v] = oy[v];
        }
        return true;
    };
    auto turned = [&](int32_t t) {
        const Tri &T = tris[t];
        return orient2d(px_[T.v[0]], py_[T.v[0]], px_[T.v[1]], py_[T.v[1]], px_[T.v[2]], py_[T.v[2]]) <= 0;
    };
    for (int32_t t = 0; t < (int32_t)tris.size(); t++)
        if (tris[t].v[0] >= 0 && turned(t) && !put_back(t)) return false;
    for (size_t q = 0; q < S.size(); q++) {
        if ((int32_t)S.size() > max_back) return false;
        // the star of S[q], through the neighbour links
        const int32_t v = S[q], t0 = where[v];
        int32_t t = t0;
        for (int step = 0;; step++) {
            if (step == 64) return false;
            if (turned(t) && !put_back(t)) return false;
            const Tri &T = tris[t];
            const int k = T.v[0] == v ? 0 : (T.v[1] == v ? 1 : 2);
            t = T.nb[(k + 1) % 3];
            if (t < 0) return false;  // v on the hull
            if (t == t0) break;
        }
    }
    if ((int32_t)S.size() > max_back) return false;
    const size_t mark = log_.size();
    make_delaunay();
    if (S.empty()) return true;
    // out with them.  A triangle of each: the one it was put back from,
    // unless the flips rewrote it (then the vertex is in a rewritten slot,
    // which the log holds); one pass over all triangles if the log is off
    if (log_all_) {
        for (int32_t t = 0; t < (int32_t)tris.size(); t++)
            for (int k = 0; k < 3; k++)
                if (tris[t].v[k] >= 0 && back[tris[t].v[k]]) where[tris[t].v[k]] = t;
    } else {
        for (size_t i = mark; i < log_.size(); i++) {
            const int32_t t = log_[i];
            if (tris[t].v[0] >= 0)
                for (int k = 0; k < 3; k++)
                    if (back[tris[t].v[k]]) where[tris[t].v[k]] = t;
        }
    }
    rewritten_.clear();
    for (int32_t v : S) {
        const int32_t t = where[v];
        if (t < 0 || !(tris[t].v[0] == v || tris[t].v[1] == v || tris[t].v[2] == v)) return false;
        touched_.clear();
        if (!remove_vertex(v, t)) return false;
        // where the vertex was: a start for locating it again
        where[v] = hint_;
        rewritten_.insert(rewritten_.end(), touched_.begin(), touched_.end());
        // the triangles the removal rewrote are where the remaining
        // vertices of S around it now are
        for (int32_t u : touched_)
            if (tris[u].v[0] >= 0)
                for (int k = 0; k < 3; k++)
                    if (back[tris[u].v[k]] && tris[u].v[k] != v) where[tris[u].v[k]] = u;
    }
    // the triangulation was Delaunay before the removals, and they rewrote
    // only these triangles: Lawson from their edges
    make_delaunay(&rewritten_);
    for (int32_t v : S) {
        px_[v] = nx[v];
        py_[v] = ny[v];
        const int32_t h = where[v];
        if (h >= 0 && h < (int32_t)tris.size() && tris[h].v[0] >= 0) hint_ = h;
        if (insert_at(v) != 0) return false;
    }
    reinserted += (int64_t)S.size();
    return true;
}

// Lawson: test every edge once, flip the ones whose opposite vertex lies
// inside the circumcircle, and test again the four outer edges of each
// flipped quadrilateral.  An entry is (triangle, k): the edge opposite
// vertex k; entries left stale by later flips test whatever edge is there.
void Delaunay::make_delaunay(const std::vector<int32_t> *seed)
{
    edges_.clear();
    if (seed) {
        for (int32_t t : *seed)
            if (t >= 0 && t < (int32_t)tris.size() && tris[t].v[0] >= 0)
                for (int k = 0; k < 3; k++) edges_.push_back(((int64_t)t << 2) | k);
    } else {
        // one pass over the triangles tests each edge once where it lies in
        // memory; only the edges that fail start the flipping
        // (candidates are gathered a block of triangles at a time without
        // a branch on the neighbour's index, whose outcome is random, then
        // tested)
        const int32_t NT = (int32_t)tris.size();
        constexpr int32_t kBlock = 256;
        int32_t cand[3 * kBlock];
        for (int32_t t0 = 0; t0 < NT; t0 += kBlock) {
            const int32_t t1 = std::min(NT, t0 + kBlock);
            int nc = 0;
            for (int32_t t = t0; t < t1; t++) {
                const Tri &T = tris[t];
                const bool live = T.v[0] >= 0;
                for (int k = 0; k < 3; k++) {
                    cand[nc] = (t << 2) | k;
                    nc += live & (T.nb[k] > t);
                }
            }
            for (int q = 0; q < nc; q++) {
                if (q + 8 < nc) {
                    // the neighbour triangle of a candidate a few ahead
                    const int32_t t8 = cand[q + 8] >> 2;
                    __builtin_prefetch(&tris[tris[t8].nb[cand[q + 8] & 3]]);
                }
                const int32_t t = cand[q] >> 2;
                const int k = cand[q] & 3;
                const Tri &T = tris[t];
                // U shares the edge (b, c): its third vertex is the one that
                // is neither (no search of U's links, whose outcome the
                // branch predictor cannot learn either)
                const Tri &U = tris[T.nb[k]];
                const int32_t a = T.v[k], b = T.v[(k + 1) % 3], c = T.v[(k + 2) % 3];
                const int32_t d = U.v[0] ^ U.v[1] ^ U.v[2] ^ b ^ c;
                if (incircle_sos(px_[a], py_[a], px_[b], py_[b], px_[c], py_[c], px_[d], py_[d]) > 0)
                    edges_.push_back(((int64_t)t << 2) | k);
            }
        }
    }
    while (!edges_.empty()) {
        const int64_t ek = edges_.back();
        edges_.pop_back();
        const int32_t t = (int32_t)(ek >> 2);
        const int k = (int)(ek & 3);
        const Tri T = tris[t];
        const int32_t u = T.nb[k];
        if (u < 0) continue;
        const Tri &U = tris[u];
        const int32_t a = T.v[k], b = T.v[(k + 1) % 3], c = T.v[(k + 2) % 3];
        const int32_t d = U.v[0] ^ U.v[1] ^ U.v[2] ^ b ^ c;
        if (incircle_sos(px_[a], py_[a], px_[b], py_[b], px_[c], py_[c], px_[d], py_[d]) <= 0) continue;
        // flip edge (b, c) of (a, b, c) and (d, c, b) into (a, d)
        flip(t, k);
        edges_.push_back(((int64_t)t << 2) | 0);
        edges_.push_back(((int64_t)t << 2) | 2);
        edges_.push_back(((int64_t)u << 2) | 0);
        edges_.push_back(((int64_t)u << 2) | 1);
    }
}

int32_t Delaunay::insert_point(double x, double y)
{
    const int32_t p = (int32_t)px_.size();
    px_.push_back(x);
    py_.push_back(y);
    int32_t t = -1;
    int edge = -1;
    const int r = locate(p, t, edge);
    if (r == -2) return -2;
    if (r < 0) return -3;
    if (r == 0) insert_inside(t, p);
    else insert_on_edge(t, edge, p);
    return p;
}

void degree_order(int32_t n, const int32_t *cell_ptr, int32_t *order)
{
    constexpr int32_t kMaxDeg = 64;
    for (int32_t w0 = 0; w0 < n; w0 += kOrderWindow) {
        const int32_t w1 = std::min(n, w0 + kOrderWindow);
        int32_t count[kMaxDeg + 1] = {};
        for (int32_t i = w0; i < w1; i++) count[std::min(cell_ptr[i + 1] - cell_ptr[i], kMaxDeg)]++;
        // exclusive offsets, largest degree first
        int32_t pos[kMaxDeg + 1];
        int32_t acc = w0;
        for (int32_t d = kMaxDeg; d >= 0; d--) {
            pos[d] = acc;
            acc += count[d];
        }
        for (int32_t i = w0; i < w1; i++) order[pos[std::min(cell_ptr[i + 1] - cell_ptr[i], kMaxDeg)]++] = i;
    }
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

// Ghost images of the points in chunks of kChunk (in parallel with a pool):
// count per chunk, then fill at the prefix offsets, so the ghost order is
// the same as one pass over the points.
static void make_ghosts(const BoxConfig &box, int32_t n, const double *x, const double *y, double w, HostMesh &m,
                        ThreadPool *pool)
{
    const double lox = box.x0 - w, hix = box.x1 + w, loy = box.y0 - w, hiy = box.y1 + w;
    constexpr int32_t kChunk = 16384;
    const int64_t nc = (n + kChunk - 1) / kChunk;
    std::vector<int64_t> off(nc + 1, 0);
    // visit(i, emit): every image of point i inside the band.  An image's x
    // depends on a only and its y on b only, so each axis is tested once
    // (most points, away from the walls, have none).
    const bool per = box.boundary == 1;
    // an image (mirrored or shifted) reaches the band only from a point
    // within w of a wall: the points well inside, by a margin far above the
    // images' round-off, are skipped before any image is formed
    const double margin = 1e-9 * (std::fabs(box.x0) + std::fabs(box.x1) + std::fabs(box.y0) + std::fabs(box.y1) + w);
    const double in_x0 = box.x0 + w + margin, in_x1 = box.x1 - w - margin;
    const double in_y0 = box.y0 + w + margin, in_y1 = box.y1 - w - margin;
    auto visit = [&](int32_t i, auto &&emit) {
        if (x[i] > in_x0 && x[i] < in_x1 && y[i] > in_y0 && y[i] < in_y1) return;
        double X[3], Y[3];
        bool okx[3], oky[3];
        for (int a = -1; a <= 1; a += 2) {
            X[a + 1] = image_coord(x[i], box.x0, box.x1, per ? 0 : a, per ? a : 0);
            okx[a + 1] = !(X[a + 1] < lox || X[a + 1] > hix);
            Y[a + 1] = image_coord(y[i], box.y0, box.y1, per ? 0 : a, per ? a : 0);
            oky[a + 1] = !(Y[a + 1] < loy || Y[a + 1] > hiy);
        }
        if (!(okx[0] || okx[2] || oky[0] || oky[2])) return;
        X[1] = x[i];
        Y[1] = y[i];
        okx[1] = !(X[1] < lox || X[1] > hix);
        oky[1] = !(Y[1] < loy || Y[1] > hiy);
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++) {
                if (a == 0 && b == 0) continue;
                if (!okx[a + 1] || !oky[b + 1]) continue;
                const int fx = per ? 0 : a, fy = per ? 0 : b, sx = per ? a : 0, sy = per ? b : 0;
                emit(X[a + 1], Y[b + 1], (fx ? XF_MIRROR_X : 0) | (fy ? XF_MIRROR_Y : 0), (sx + 1) + 3 * (sy + 1),
                     (a + 1) + 3 * (b + 1));
            }
    };
    // the points with images, per chunk, found by the counting pass so that
    // the filling pass visits only them
    std::vector<std::vector<int32_t>> cand(nc);
    auto count = [&](int64_t c) {
        int64_t k = 0;
        const int32_t i0 = (int32_t)(c * kChunk), i1 = (int32_t)std::min<int64_t>(n, (c + 1) * kChunk);
        for (int32_t i = i0; i < i1; i++) {
            // (the test that skips most points, in the loop itself)
            if (x[i] > in_x0 && x[i] < in_x1 && y[i] > in_y0 && y[i] < in_y1) continue;
            const int64_t k0 = k;
            visit(i, [&](double, double, int32_t, int32_t, int32_t) { k++; });
            if (k != k0) cand[c].push_back(i);
        }
        off[c + 1] = k;
    };
    if (pool && nc > 1) pool->parallel_for(nc, count);
    else
        for (int64_t c = 0; c < nc; c++) count(c);
    for (int64_t c = 0; c < nc; c++) off[c + 1] += off[c];
    const size_t g = (size_t)off[nc];
    m.gx.resize(g); m.gy.resize(g); m.ghost_src.resize(g); m.ghost_xf.resize(g); m.ghost_shift.resize(g);
    m.ghost_img.resize(g);
    auto fill = [&](int64_t c) {
        int64_t k = off[c];
        for (const int32_t i : cand[c])
            visit(i, [&](double X, double Y, int32_t xf, int32_t sh, int32_t img) {
                m.gx[k] = X; m.gy[k] = Y; m.ghost_src[k] = i; m.ghost_xf[k] = xf; m.ghost_shift[k] = sh;
                m.ghost_img[k] = img;
                k++;
            });
    };
    if (pool && nc > 1) pool->parallel_for(nc, fill);
    else
        for (int64_t c = 0; c < nc; c++) fill(c);
    m.g = (int32_t)g;
}

namespace {

// Circumdisk of the triangle (a, b, c), radius padded for round-off so that a
// containment test against it errs on the safe side.
struct Disk {
    double ux, uy, R;
};

inline Disk circumdisk(const double *X, const double *Y, int32_t a, int32_t b, int32_t c, double pad)
{
    double ax = X[a], ay = Y[a];
    double bx = X[b] - ax, by = Y[b] - ay, cx = X[c] - ax, cy = Y[c] - ay;
    const double rd = 1.0 / (2.0 * (bx * cy - by * cx));
    double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    double ux = (cy * b2 - by * c2) * rd, uy = (bx * c2 - cx * b2) * rd;
    return Disk{ux + ax, uy + ay, std::sqrt(ux * ux + uy * uy) * (1.0 + 1e-9) + pad};
}

// Points bucketed on a G x G grid over a rectangle.
struct PointGrid {
    int G = 1;
    double x0 = 0.0, y0 = 0.0, sx = 0.0, sy = 0.0;
    const int32_t *start = nullptr, *ids = nullptr;
    PointGrid() = default;
    explicit PointGrid(const MeshWork::GridBufs &b)
        : G(b.G), x0(b.x0), y0(b.y0), sx(b.sx), sy(b.sy), start(b.start.data()), ids(b.ids.data())
    {
    }
    // bucket column / row of a coordinate, clamped to the grid (infinite
    // and NaN coordinates included)
    int col(double x) const { return clampi((x - x0) * sx); }
    int row(double y) const { return clampi((y - y0) * sy); }
    int clampi(double f) const { return !(f > 0.0) ? 0 : (f >= G ? G - 1 : (int)f); }
};

// Counting sort of the point ids q0 .. q1-1 by bucket of a grid over the
// rectangle ext, in chunks on the pool: a histogram per chunk, offsets per
// (bucket, chunk), then each chunk scatters its ids in increasing order.
void build_grid(int32_t q0, int32_t q1, const double *X, const double *Y, const double ext[4],
                MeshWork::GridBufs &w, ThreadPool *pool)
{
    const int32_t np = q1 - q0;
    w.G = std::max(1, std::min(1024, (int)std::sqrt(np / 32.0)));
    const int G = w.G;
    const int64_t GG = (int64_t)G * G;
    w.x0 = ext[0];
    w.y0 = ext[2];
    w.sx = ext[1] > ext[0] ? G / (ext[1] - ext[0]) : 0.0;
    w.sy = ext[3] > ext[2] ? G / (ext[3] - ext[2]) : 0.0;
    PointGrid g(w);
    const int64_t C = pool ? std::max(1, std::min(pool->size(), (int)(np / 8192) + 1)) : 1;
    const int64_t chunk = (np + C - 1) / C;
    w.cell.resize(np);
    w.hist.assign(C * GG, 0);
    w.start.assign(GG + 1, 0);
    w.ids.resize(np);
    auto count = [&](int64_t c) {
        int32_t *h = w.hist.data() + c * GG;
        for (int64_t q = c * chunk; q < std::min<int64_t>(np, (c + 1) * chunk); q++) {
            const int32_t b = g.row(Y[q0 + q]) * G + g.col(X[q0 + q]);
            w.cell[q] = b;
            h[b]++;
        }
    };
    if (pool && C > 1) pool->parallel_for(C, count);
    else
        for (int64_t c = 0; c < C; c++) count(c);
    // offsets: bucket-major, chunk-minor, so ids stay increasing in a
    // bucket; in ranges of buckets on the pool (their totals, a prefix over
    // the ranges, then each range from its start)
    const int64_t BR = 4096, nbr = (GG + BR - 1) / BR;
    std::vector<int64_t> rsum(nbr + 1, 0);
    auto range_total = [&](int64_t r) {
        int64_t t = 0;
        for (int64_t b = r * BR; b < std::min(GG, (r + 1) * BR); b++)
            for (int64_t c = 0; c < C; c++) t += w.hist[c * GG + b];
        rsum[r + 1] = t;
    };
    auto range_offsets = [&](int64_t r) {
        int32_t run = (int32_t)rsum[r];
        for (int64_t b = r * BR; b < std::min(GG, (r + 1) * BR); b++) {
            w.start[b] = run;
            for (int64_t c = 0; c < C; c++) {
                const int32_t k = w.hist[c * GG + b];
                w.hist[c * GG + b] = run;
                run += k;
            }
        }
    };
    if (pool && nbr > 1) pool->parallel_for(nbr, range_total);
    else
        for (int64_t r = 0; r < nbr; r++) range_total(r);
    for (int64_t r = 0; r < nbr; r++) rsum[r + 1] += rsum[r];
    if (pool && nbr > 1) pool->parallel_for(nbr, range_offsets);
    else
        for (int64_t r = 0; r < nbr; r++) range_offsets(r);
    w.start[GG] = (int32_t)rsum[nbr];
    auto scatter = [&](int64_t c) {
        int32_t *off = w.hist.data() + c * GG;
        for (int64_t q = c * chunk; q < std::min<int64_t>(np, (c + 1) * chunk); q++)
            w.ids[off[w.cell[q]]++] = (int32_t)(q0 + q);
    };
    if (pool && C > 1) pool->parallel_for(C, scatter);
    else
        for (int64_t c = 0; c < C; c++) scatter(c);
}

// Outcome of one tile: the rings of its real core cells, the triangles they
// use (global point ids, smallest id first), whether the halo and the ghost
// band were wide enough, and the halo its stars actually needed.
using SlabResult = TileStars;

// What every tile of one build shares.
struct SlabCtx {
    int32_t n = 0, np = 0;
    const double *X = nullptr, *Y = nullptr;  // real points, then ghosts
    const BoxConfig *box = nullptr;
    const HostMesh *m = nullptr;              // ghost sources and images
    const double *ext = nullptr;              // bounding box of all points
    const PointGrid *grid = nullptr;   // real points, possibly from an earlier build
    double slack = 0.0;                // how far a real point can be from where that grid saw it
    const PointGrid *ggrid = nullptr;  // ghosts of this build
    const double *band = nullptr;
    double pad = 0.0;
    const MeshWork *work = nullptr;           // ghost key lookup of this build
};

// internal: an updated triangulation cannot be used (a star touches an
// image that is no longer in the point set): build the tile afresh
constexpr int kRedo = -100;

inline int64_t point_key(const SlabCtx &c, int32_t q)
{
    if (q < c.n) return q;
    const int32_t g = q - c.n;
    return (int64_t)c.n + 9 * (int64_t)c.m->ghost_src[g] + c.m->ghost_img[g];
}

// The tile's rectangle with its halo (a halo that covers every point makes
// the tile's triangulation the whole one).
struct Rect {
    double xlo, xhi, ylo, yhi;
    bool whole;
};

Rect tile_rect(const SlabCtx &c, const Tile &tile, double H)
{
    Rect R{tile.fx ? -INFINITY : tile.x0 - H, tile.lx ? INFINITY : tile.x1 + H, tile.fy ? -INFINITY : tile.y0 - H,
           tile.ly ? INFINITY : tile.y1 + H, false};
    R.whole = R.xlo <= c.ext[0] && R.xhi > c.ext[1] && R.ylo <= c.ext[2] && R.yhi > c.ext[3];
    if (R.whole) R.xlo = R.ylo = -INFINITY, R.xhi = R.yhi = INFINITY;
    return R;
}

// Every point of the rectangle: the real points from the buckets of their
// grid that the rectangle widened by the grid's slack overlaps, the ghosts
// from theirs; each tested on its current position.
template <class F> void scan_grid(const SlabCtx &c, const PointGrid &grid, const Rect &R, double slack, F &&f)
{
    const int c0 = grid.col(R.xlo - slack), c1 = grid.col(R.xhi + slack);
    const int r0 = grid.row(R.ylo - slack), r1 = grid.row(R.yhi + slack);
    for (int rw = r0; rw <= r1; rw++)
        for (int32_t k = grid.start[rw * grid.G + c0]; k < grid.start[rw * grid.G + c1 + 1]; k++) {
            const int32_t q = grid.ids[k];
            if (c.X[q] >= R.xlo && c.X[q] < R.xhi && c.Y[q] >= R.ylo && c.Y[q] < R.yhi) f(q);
        }
}

template <class F> void for_rect_points(const SlabCtx &c, const Rect &R, F &&f)
{
    scan_grid(c, *c.grid, R, c.slack, f);
    if (c.np > c.n) scan_grid(c, *c.ggrid, R, 0.0, f);
}

// Update the tile's last triangulation for this build's points: move every
// vertex to its point's new position (an image that left the ghost band
// stays, at its source's new image position: it is still a point of the
// periodic or mirrored plane; the vertices of triangles that would turn
// over are taken out and inserted again), flip to Delaunay, and insert the
// points of the rectangle that are not vertices yet.  Returns false when
// the tile must be built afresh.
bool update_slab(const SlabCtx &c, const Rect &R, Delaunay &dt, std::vector<int32_t> &loc,
                 std::vector<int64_t> &keys, std::vector<uint32_t> &stamp, std::vector<double> &nx,
                 std::vector<double> &ny)
{
    const int32_t NL = dt.size();
    if ((int32_t)keys.size() != NL || NL < 3) return false;
    const MeshWork &w = *c.work;
    if ((int32_t)stamp.size() < c.np) stamp.resize(c.np, 0u);
    loc.resize(NL);
    nx.resize(NL);
    ny.resize(NL);
    int32_t stray = 0;
    for (int32_t v = 0; v < NL; v++) {
        const int64_t k = keys[v];
        if (k == -2) {
            loc[v] = -2;
            nx[v] = dt.x(v);
            ny[v] = dt.y(v);
            continue;
        }
        int32_t q;
        double px, py;
        if (k < c.n) {
            q = (int32_t)k;
            px = c.X[q];
            py = c.Y[q];
        } else {
            const int64_t gk = k - c.n;
            const int32_t src = (int32_t)(gk / 9), img = (int32_t)(gk % 9);
            if (w.gkey_stamp[gk] == w.gen) {
                q = c.n + w.gkey_idx[gk];
                px = c.X[q];
                py = c.Y[q];
            } else {
                q = -1;
                const int a = img % 3 - 1, b = img / 3 - 1;
                const BoxConfig &box = *c.box;
                const bool per = box.boundary == 1;
                px = image_coord(c.X[src], box.x0, box.x1, per ? 0 : a, per ? a : 0);
                py = image_coord(c.Y[src], box.y0, box.y1, per ? 0 : b, per ? b : 0);
            }
        }
        loc[v] = q;
        nx[v] = px;
        ny[v] = py;
        if (q >= 0) stamp[q] = w.gen;
        if (q < 0 || !(px >= R.xlo && px < R.xhi && py >= R.ylo && py < R.yhi)) stray++;
    }
    // vertices that are no longer needed are kept; rebuild once they are many
    if (stray > NL / 4) return false;
    // (at most 2 % of the vertices taken out and put back where triangles
    // would turn over; beyond that a fresh build is cheaper)
    if (!dt.move_all(nx, ny, std::max<int32_t>(16, NL / 50))) return false;
    bool ok = true;
    for_rect_points(c, R, [&](int32_t q) {
        if (!ok || stamp[q] == w.gen) return;
        const int32_t v = dt.insert_point(c.X[q], c.Y[q]);
        if (v < 0) {
            ok = false;
            return;
        }
        loc.push_back(q);
        keys.push_back(point_key(c, q));
        stamp[q] = w.gen;
    });
    return ok;
}

// Read off the stars of the tile's real core points from dt, whose vertex v
// is point loc[v] (negative: a corner of the enclosing triangle, or an
// image no longer in the point set).  A star is the true one when the
// circumdisk of each of its triangles lies inside the triangulated
// rectangle: every point of the whole set inside such a disk was then
// triangulated too, and an empty circumdisk among them is empty in the
// whole set.
void read_stars(const SlabCtx &c, const Tile &tile, const Rect &R, Delaunay &dt,
                const std::vector<int32_t> &loc, SlabResult &r)
{
    const int32_t n = c.n, nl = dt.size();
    const double xlo = R.xlo, xhi = R.xhi, ylo = R.ylo, yhi = R.yhi;
    const bool whole = R.whole;
    const double *band = c.band, pad = c.pad;
    const double *LX = dt.xs(), *LY = dt.ys();
    const std::vector<Tri> &T = dt.tris;
    // real points of the tile itself
    std::vector<uint8_t> &core = r.core;
    core.assign(nl, 0);
    int32_t ncore = 0;
    for (int32_t v = 0; v < nl; v++) {
        const double px = LX[v], py = LY[v];
        core[v] = loc[v] >= 0 && loc[v] < n && (tile.fx || px >= tile.x0) && (tile.lx || px < tile.x1) &&
                  (tile.fy || py >= tile.y0) && (tile.ly || py < tile.y1);
        ncore += core[v];
    }
    auto core_real = [&](int32_t v) { return core[v] != 0; };
    // the stars of the real core points: check and number their triangles
    // and, when the host builds the triangle list, number them and write
    // them with global ids, rotated so that the smallest id comes first (a
    // shared triangle then gives the same circumcentre in every slab)
    const bool host_tris = c.work->host_edges;
    std::vector<int32_t> &tnum = r.tnum;
    if (host_tris) {
        tnum.assign(T.size(), -1);
        r.tris.resize(3 * T.size());
    }
    // the strictest bound on each side: the band, the halo rectangle, and
    // the tile's own side where it is not open (the halo needed)
    const double fL = std::max(std::max(band[0], xlo), tile.fx ? -INFINITY : tile.x0);
    const double fR = std::min(std::min(band[1], xhi), tile.lx ? INFINITY : tile.x1);
    const double fB = std::max(std::max(band[2], ylo), tile.fy ? -INFINITY : tile.y0);
    const double fT = std::min(std::min(band[3], yhi), tile.ly ? INFINITY : tile.y1);
    int32_t *otris = host_tris ? r.tris.data() : nullptr;
    int32_t nt = 0;
    for (size_t t = 0; t < T.size(); t++) {
        const int32_t *v = T[t].v;
        if (!core_real(v[0]) && !core_real(v[1]) && !core_real(v[2])) continue;
        if (dt.is_corner(v[0]) || dt.is_corner(v[1]) || dt.is_corner(v[2])) {
            // a real point on the hull of the triangulated points: the ghost
            // band, or else the halo, is too narrow
            if (whole) r.band_ok = false;
            else r.halo_ok = false;
            return;
        }
        const int32_t g0 = loc[v[0]], g1 = loc[v[1]], g2 = loc[v[2]];
        if (g0 < 0 || g1 < 0 || g2 < 0) {
            r.rc = kRedo;
            return;
        }
        // most disks clear the strictest bound on every side (band, halo
        // rectangle, tile side) by far: that is decided on the squared
        // radius, with a margin well above the round-off of both sides, and
        // such a disk passes every test below and adds nothing to the halo
        // needed
        bool clear;
        {
            const double ax = LX[v[0]], ay = LY[v[0]];
            const double bx = LX[v[1]] - ax, by = LY[v[1]] - ay, cx = LX[v[2]] - ax, cy = LY[v[2]] - ay;
            const double rd = 1.0 / (2.0 * (bx * cy - by * cx));
            const double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
            const double ux = (cy * b2 - by * c2) * rd, uy = (bx * c2 - cx * b2) * rd;
            const double cl = std::min(ux + ax - fL, fR - (ux + ax)), cb = std::min(uy + ay - fB, fT - (uy + ay));
            const double mg = std::min(cl, cb) - pad;
            clear = mg > 0.0 && mg * mg > (ux * ux + uy * uy) * 1.00000001;
        }
        if (!clear) {
            const Disk D = circumdisk(LX, LY, v[0], v[1], v[2], pad);
            if (!(D.ux - D.R >= band[0] && D.ux + D.R <= band[1] && D.uy - D.R >= band[2] &&
                  D.uy + D.R <= band[3])) {
                r.band_ok = false;
                return;
            }
            if (!(D.ux - D.R >= xlo && D.ux + D.R <= xhi && D.uy - D.R >= ylo && D.uy + D.R <= yhi)) {
                r.halo_ok = false;
                return;
            }
            // how far this disk reaches past the tile: the halo it needs
            if (!tile.fx) r.needed = std::max(r.needed, tile.x0 - (D.ux - D.R));
            if (!tile.lx) r.needed = std::max(r.needed, D.ux + D.R - tile.x1);
            if (!tile.fy) r.needed = std::max(r.needed, tile.y0 - (D.uy - D.R));
            if (!tile.ly) r.needed = std::max(r.needed, D.uy + D.R - tile.y1);
        }
        if (!host_tris) continue;
        const int rot = (g0 < g1 && g0 < g2) ? 0 : (g1 < g2 ? 1 : 2);
        const int32_t gg[5] = {g0, g1, g2, g0, g1};
        int32_t *o = otris + 3 * (size_t)nt;
        o[0] = gg[rot];
        o[1] = gg[rot + 1];
        o[2] = gg[rot + 2];
        tnum[t] = nt++;
    }
    r.tris.resize(3 * (size_t)nt);
    // rings, counter-clockwise, starting at the smallest neighbour id.  A
    // vertex's ring changes only where a triangle slot holding it was
    // written since the last read-off (the triangulation's log; every slot
    // after a fresh build), or where a neighbour's global id changed (ghost
    // ids follow this build's ghost list): those rings, those of vertices
    // with no ring in the last read-off's output, and every ring when the
    // host builds the triangle list (whose numbers change from build to
    // build), are walked through the neighbour links from a slot holding the
    // vertex; the others are copied from the last output as they were.
    const bool all = dt.log_all() || host_tris;
    std::vector<uint8_t> &dirty = r.dirty;
    std::vector<int32_t> &vt = r.vt;
    dirty.assign(nl, all ? 1 : 0);
    if (dt.log_all()) {
        vt.assign(nl, -1);
        for (size_t t = 0; t < T.size(); t++)
            if (T[t].v[0] >= 0)
                for (int k = 0; k < 3; k++) vt[T[t].v[k]] = (int32_t)t;
    } else {
        vt.resize(nl, -1);
        for (const int32_t t : dt.log()) {
            if (t < 0 || t >= (int32_t)T.size() || T[t].v[0] < 0) continue;
            for (int k = 0; k < 3; k++) {
                dirty[T[t].v[k]] = 1;
                vt[T[t].v[k]] = t;
            }
        }
    }
    dt.clear_log();
    // the star of local vertex v through the neighbour links from vt[v]:
    // neighbour after v in each slot, and the slot; its size, or -1 when the
    // star does not close (or no slot is known to hold v: -2)
    constexpr int32_t kMaxStar = 64;
    auto walk = [&](int32_t v, int32_t *wnb, int32_t *wt) -> int32_t {
        int32_t t = vt[v];
        int k = t < 0 ? -1 : (T[t].v[0] == v ? 0 : (T[t].v[1] == v ? 1 : (T[t].v[2] == v ? 2 : -1)));
        if (k < 0) return -2;
        const int32_t t0 = t;
        int32_t deg = 0;
        do {
            if (deg == kMaxStar) return -1;
            // in slot t with v at position k the neighbour after v is
            // a = v[k+1]; the next slot counter-clockwise about v shares the
            // edge (v, v[k+2]), the one opposite a
            const Tri &U = T[t];
            wnb[deg] = U.v[(k + 1) % 3];
            wt[deg++] = t;
            const int32_t b = U.v[(k + 2) % 3];
            t = U.nb[(k + 1) % 3];
            if (t < 0) return -1;
            const Tri &V = T[t];
            k = V.v[0] == v ? 0 : (V.v[1] == v ? 1 : (V.v[2] == v ? 2 : -1));
            if (k < 0 || V.v[(k + 1) % 3] != b) return -1;
        } while (t != t0);
        return deg;
    };
    // a neighbour whose global id changed: walk the rings around it again
    std::vector<int32_t> &ploc = r.prev_loc;
    const int32_t nprev = all ? 0 : (int32_t)std::min<size_t>(r.out_off.size(), ploc.size());
    int32_t wnb[kMaxStar], wt[kMaxStar];
    for (int32_t v = 0; v < nprev; v++) {
        if (loc[v] == ploc[v]) continue;
        dirty[v] = 1;
        const int32_t d = walk(v, wnb, wt);
        if (d == -2) {
            r.rc = kRedo;  // no slot known to hold v
            return;
        }
        for (int32_t j = 0; j < d; j++) dirty[wnb[j]] = 1;
        if (d < 0)
            for (int32_t u = 0; u < nl; u++) dirty[u] = 1;  // (not expected) walk everything
    }
    ploc.assign(loc.begin(), loc.begin() + nl);
    // the outputs (core vertices in local order), sized for a mean degree
    // of 8 and grown if that is not enough (the mean is 6); the last output
    // is kept beside them until the copies are done
    std::vector<int32_t> &nb_prev = r.nb_prev, &noff = r.next_off, &nlen = r.next_len;
    r.nb.swap(nb_prev);
    noff.resize(nl);
    nlen.resize(nl);
    r.cells.resize(ncore);
    r.deg.resize(ncore);
    size_t cap = std::max<size_t>(std::max(r.nb.size(), nb_prev.size()), 8 * (size_t)ncore + 64);
    r.nb.resize(cap);
    if (host_tris) r.tri.resize(cap);
    size_t os = 0;
    int32_t oc = 0;
    for (int32_t v = 0; v < nl; v++) {
        noff[v] = -1;
        nlen[v] = 0;
        if (!core_real(v)) continue;
        int32_t deg;
        const bool copy = !dirty[v] && v < nprev && r.out_off[v] >= 0;
        if (copy) {
            deg = r.out_len[v];
        } else {
            deg = walk(v, wnb, wt);
            if (deg == -2) {
                r.rc = kRedo;
                return;
            }
            if (deg < 0) {
                r.rc = -3;  // the star is not closed, or inconsistent links
                return;
            }
        }
        if (deg < 3) {
            r.rc = -3;
            return;
        }
        if (os + deg > cap) {
            cap = 2 * cap + kMaxStar;
            r.nb.resize(cap);
            if (host_tris) r.tri.resize(cap);
        }
        noff[v] = (int32_t)os;
        nlen[v] = deg;
        r.cells[oc] = loc[v];
        r.deg[oc++] = deg;
        int32_t *onb = r.nb.data() + os;
        if (copy) {
            std::copy(nb_prev.data() + r.out_off[v], nb_prev.data() + r.out_off[v] + deg, onb);
        } else {
            // start at the smallest neighbour id
            int32_t G[kMaxStar];
            int32_t k = 0, kid = INT32_MAX;
            for (int32_t q = 0; q < deg; q++) {
                const int32_t id = loc[wnb[q]];
                G[q] = id;
                k = id < kid ? q : k;
                kid = id < kid ? id : kid;
            }
            for (int32_t j = 0; j < deg; j++) onb[j] = G[k + j < deg ? k + j : k + j - deg];
            if (host_tris) {
                // (a ring's triangles all touch its core vertex, so all are numbered)
                int32_t *otr = r.tri.data() + os;
                for (int32_t j = 0; j < deg; j++) otr[j] = tnum[wt[k + j < deg ? k + j : k + j - deg]];
            }
        }
        os += deg;
    }
    r.nb.resize(os);
    if (host_tris) r.tri.resize(os);
    r.out_off.swap(noff);
    r.out_len.swap(nlen);
}

// Triangulate the points of a tile plus a halo of width H (by updating the
// tile's last triangulation when `update` is set and that succeeds), keep
// the keys of its vertices for the next build, and read off the stars of its
// real core points.
void build_slab(const SlabCtx &c, const Tile &tile, double H, bool update, Delaunay &dt, std::vector<int32_t> &loc,
                std::vector<double> &LX, std::vector<double> &LY, std::vector<int64_t> &keys,
                std::vector<uint32_t> &stamp, bool &updated, SlabResult &r)
{
    r.reset();
    updated = false;
    const Rect R = tile_rect(c, tile, H);
    if (update && update_slab(c, R, dt, loc, keys, stamp, r.nx, r.ny)) {
        read_stars(c, tile, R, dt, loc, r);
        if (r.rc != kRedo) {
            updated = true;
            return;
        }
        r.reset();
    }
    // afresh: the points of the rectangle (bucket by bucket; the
    // triangulation does not depend on their order, and the rings and
    // triangles are put in canonical order)
    loc.clear();
    LX.clear();
    LY.clear();
    keys.clear();
    for_rect_points(c, R, [&](int32_t q) { loc.push_back(q); });
    // local vertices in increasing point id: the real points' ids follow a
    // space-filling curve, so the tile's rings land in the assembled arrays
    // in long ascending runs instead of scattered (the ghosts, with the
    // largest ids, come last)
    std::sort(loc.begin(), loc.end());
    for (const int32_t q : loc) {
        LX.push_back(c.X[q]);
        LY.push_back(c.Y[q]);
    }
    const int32_t nl = (int32_t)loc.size();
    if (nl == 0) return;
    r.rc = dt.build(LX.data(), LY.data(), nl);
    if (r.rc) return;
    loc.resize(nl + 3, -2);
    keys.resize(nl + 3, -2);
    for (int32_t v = 0; v < nl; v++) keys[v] = point_key(c, loc[v]);
    read_stars(c, tile, R, dt, loc, r);
    if (r.rc == kRedo) r.rc = -3;  // (a fresh build has no stale images)
}

}  // namespace

static double wall_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int build_host_mesh(const BoxConfig &box, int32_t n, const double *x, const double *y, MeshWork &work, HostMesh &m,
                    ThreadPool *pool)
{
    double t_mark = wall_ms();
    for (double &v : work.phase_ms) v = 0.0;
    auto lap = [&](int k) {
        const double t = wall_ms();
        work.phase_ms[k] += t - t_mark;
        t_mark = t;
    };
    const double Lx = box.x1 - box.x0, Ly = box.y1 - box.y0;
    const double h = std::sqrt(Lx * Ly / std::max(n, 1));
    const double wmax = std::min(Lx, Ly);
    const double pad = 1e-12 * (Lx + Ly);
    double w = std::min(5.0 * h, wmax);
    m.n = n;
    m.attempts = 0;
    // tiles: enough points each that the halo stays a small fraction, and
    // up to four per thread, so that the pool balances tiles of unequal cost
    // (one per thread left the slowest tile setting the pass: 1M points on
    // 8 threads, 97 ms per build against 81 ms with four); Kx columns of Ky
    // rows, as square as K allows
    const int threads = pool ? pool->size() : 1;
    const int K = std::max(1, std::min(threads > 1 ? 4 * threads : 1, n / 16384));
    int Ky = (int)std::sqrt((double)K);
    while (K % Ky) Ky--;
    const int Kx = K / Ky;
    if ((int)work.dts.size() < K) work.dts.resize(K);
    work.loc.resize(K);
    work.lx.resize(K);
    work.ly.resize(K);
    work.keys.resize(K);
    work.stamp.resize(K);
    // update the last build's tiles in place when there is one for these
    // points (same count, same tiling)
    const bool reuse = work.kinetic && work.n_kept == n && (int)work.tiles.size() == K &&
                       (int)work.tile_halo.size() == K;
    work.n_kept = -1;  // valid again only once this build succeeds
    if ((int)work.stars.size() < K) work.stars.resize(K);
    std::vector<TileStars> &res = work.stars;
    std::vector<uint8_t> updated(K, 0);
    std::vector<double> &X = work.X, &Y = work.Y;
    for (;;) {
        m.attempts++;
        make_ghosts(box, n, x, y, w, m, pool);
        const int32_t np = n + m.g;
        // ghost key -> this build's ghost index
        work.gen++;
        if (work.gkey_idx.size() < 9 * (size_t)n) {
            work.gkey_idx.assign(9 * (size_t)n, -1);
            work.gkey_stamp.assign(9 * (size_t)n, 0u);
        }
        {
            // (each ghost has its own key: chunks on the pool write apart)
            const int64_t gc = 8192, ngc = ((int64_t)m.g + gc - 1) / gc;
            auto keys = [&](int64_t c) {
                for (int32_t g = (int32_t)(c * gc); g < (int32_t)std::min<int64_t>(m.g, (c + 1) * gc); g++) {
                    const size_t k = 9 * (size_t)m.ghost_src[g] + (size_t)m.ghost_img[g];
                    work.gkey_idx[k] = g;
                    work.gkey_stamp[k] = work.gen;
                }
            };
            if (pool && ngc > 1) pool->parallel_for(ngc, keys);
            else
                for (int64_t c = 0; c < ngc; c++) keys(c);
        }
        X.resize(np);
        Y.resize(np);
        // the points copied in chunks on the pool (one thread copies ~5
        // GB/s), each chunk's bounding box taken on the way; the ghosts' box
        // from their own list
        double ext[4];
        {
            const int64_t cc = 32768, ncc = (n + cc - 1) / cc;
            std::vector<std::array<double, 4>> part(ncc + 1);
            // (and each chunk's largest move of a coordinate since the last
            // build, whose points X, Y still hold when the grid is kept)
            std::vector<double> moved(ncc, 0.0);
            const bool track = work.grid_n == n;
            auto copy = [&](int64_t c) {
                const int64_t q0 = c * cc, q1 = std::min<int64_t>(n, q0 + cc);
                std::array<double, 4> bb = {x[q0], x[q0], y[q0], y[q0]};
                double mv = 0.0;
                for (int64_t q = q0; q < q1; q++) {
                    const double xq = x[q], yq = y[q];
                    if (track) mv = std::max(mv, std::max(std::fabs(xq - X[q]), std::fabs(yq - Y[q])));
                    X[q] = xq;
                    Y[q] = yq;
                    bb[0] = std::min(bb[0], xq);
                    bb[1] = std::max(bb[1], xq);
                    bb[2] = std::min(bb[2], yq);
                    bb[3] = std::max(bb[3], yq);
                }
                part[c] = bb;
                moved[c] = mv;
            };
            if (pool && ncc > 1) pool->parallel_for(ncc, copy);
            else
                for (int64_t c = 0; c < ncc; c++) copy(c);
            std::memcpy(X.data() + n, m.gx.data(), sizeof(double) * m.g);
            std::memcpy(Y.data() + n, m.gy.data(), sizeof(double) * m.g);
            part[ncc] = part[0];
            for (int32_t g = 0; g < m.g; g++) {
                part[ncc][0] = std::min(part[ncc][0], m.gx[g]);
                part[ncc][1] = std::max(part[ncc][1], m.gx[g]);
                part[ncc][2] = std::min(part[ncc][2], m.gy[g]);
                part[ncc][3] = std::max(part[ncc][3], m.gy[g]);
            }
            if (track)
                for (const double mv : moved) work.grid_slack += mv;
            ext[0] = ext[1] = X[0];
            ext[2] = ext[3] = Y[0];
            for (const auto &bb : part) {
                ext[0] = std::min(ext[0], bb[0]);
                ext[1] = std::max(ext[1], bb[1]);
                ext[2] = std::min(ext[2], bb[2]);
                ext[3] = std::max(ext[3], bb[3]);
            }
        }
        const double band[4] = {box.x0 - w, box.x1 + w, box.y0 - w, box.y1 + w};
        // the real points' grid over the box, kept while they have moved
        // less than half a bucket since it was built (a NaN move rebuilds)
        {
            const MeshWork::GridBufs &gr = work.grid_real;
            const double half_bucket = 0.5 / std::max(gr.sx, gr.sy);
            if (work.grid_n != n || !(work.grid_slack < half_bucket)) {
                const double bext[4] = {box.x0, box.x1, box.y0, box.y1};
                build_grid(0, n, X.data(), Y.data(), bext, work.grid_real, pool);
                work.grid_n = n;
                work.grid_slack = 0.0;
            }
        }
        build_grid(n, np, X.data(), Y.data(), ext, work.grid_ghost, pool);
        const PointGrid grid(work.grid_real), ggrid(work.grid_ghost);
        lap(0);
        SlabCtx ctx;
        ctx.n = n;
        ctx.np = np;
        ctx.X = X.data();
        ctx.Y = Y.data();
        ctx.box = &box;
        ctx.m = &m;
        ctx.ext = ext;
        ctx.grid = &grid;
        // (widened a little beyond the summed moves against their rounding)
        ctx.slack = work.grid_slack > 0.0
                        ? work.grid_slack * (1.0 + 1e-6) +
                              1e-12 * std::max({std::fabs(box.x0), std::fabs(box.x1), std::fabs(box.y0),
                                                std::fabs(box.y1)})
                        : 0.0;
        ctx.ggrid = &ggrid;
        ctx.band = band;
        ctx.pad = pad;
        ctx.work = &work;
        // column cuts at x-quantiles of (a sample of) the real + ghost
        // points, then row cuts at y-quantiles within each column (or the
        // last build's tiles, to update them in place)
        std::vector<Tile> tiles(K);
        if (reuse) tiles = work.tiles;
        else {
            std::vector<int32_t> smp;
            smp.reserve(np / 8 + 1);
            for (int32_t q = 0; q < np; q += 8) smp.push_back(q);
            auto byx = [&](int32_t a, int32_t c) { return X[a] < X[c]; };
            auto byy = [&](int32_t a, int32_t c) { return Y[a] < Y[c]; };
            // (each cut value is read right after its selection: a later
            // selection on the remaining range moves the elements)
            std::vector<size_t> cb(Kx + 1);
            std::vector<double> xc(Kx + 1, 0.0);
            for (int i = 0; i <= Kx; i++) cb[i] = (size_t)i * smp.size() / Kx;
            for (int i = 1; i < Kx; i++) {
                std::nth_element(smp.begin() + cb[i - 1], smp.begin() + cb[i], smp.end(), byx);
                xc[i] = X[smp[cb[i]]];
            }
            for (int i = 0; i < Kx; i++) {
                const double x0 = xc[i], x1 = xc[i + 1];
                const size_t m0 = cb[i], m1 = cb[i + 1];
                std::vector<size_t> rb(Ky + 1);
                std::vector<double> yc(Ky + 1, 0.0);
                for (int j = 0; j <= Ky; j++) rb[j] = m0 + (size_t)j * (m1 - m0) / Ky;
                for (int j = 1; j < Ky; j++) {
                    std::nth_element(smp.begin() + rb[j - 1], smp.begin() + rb[j], smp.begin() + m1, byy);
                    yc[j] = Y[smp[rb[j]]];
                }
                for (int j = 0; j < Ky; j++) {
                    Tile &t = tiles[i * Ky + j];
                    t.x0 = x0;
                    t.x1 = x1;
                    t.y0 = yc[j];
                    t.y1 = yc[j + 1];
                    t.fx = i == 0;
                    t.lx = i + 1 == Kx;
                    t.fy = j == 0;
                    t.ly = j + 1 == Ky;
                }
            }
        }
        // halo: what the stars needed last time (in mean spacings), else 6 h
        // (a tile updated in place keeps its own)
        std::vector<double> H(K, (work.halo > 0 ? work.halo : 6.0) * h);
        if (reuse) H = work.tile_halo;
        std::vector<uint8_t> upd(K, reuse ? 1 : 0);
        std::vector<int> todo(K);
        for (int s = 0; s < K; s++) todo[s] = s;
        bool band_ok = true;
        while (!todo.empty()) {
            auto run = [&](int64_t k) {
                const int s = todo[k];
                bool up = false;
                build_slab(ctx, tiles[s], H[s], upd[s] != 0, work.dts[s], work.loc[s], work.lx[s], work.ly[s],
                           work.keys[s], work.stamp[s], up, res[s]);
                updated[s] = up ? 1 : 0;
            };
            if (pool && todo.size() > 1) pool->parallel_for((int64_t)todo.size(), run);
            else
                for (size_t k = 0; k < todo.size(); k++) run((int64_t)k);
            std::vector<int> again;
            for (int s : todo) {
                if (res[s].rc) return res[s].rc;
                if (!res[s].band_ok) band_ok = false;
                else if (!res[s].halo_ok) {
                    H[s] *= 1.5;
                    upd[s] = 0;  // a wider rectangle: build afresh
                    again.push_back(s);
                }
            }
            if (!band_ok) break;
            todo.swap(again);
        }
        lap(1);
        if (!band_ok) {
            if (w >= wmax) return -4;
            w = std::min(2.0 * w, wmax);
            continue;
        }
        m.band = w;
        // next time: the widest reach seen, with a margin for the points'
        // motion in one step
        double need = 0.0;
        for (int s = 0; s < K; s++) need = std::max(need, res[s].needed);
        work.halo = std::max(2.0, 1.25 * need / h + 0.5);
        for (int s = 0; s < K; s++) {
            if (updated[s]) work.kinetic_tiles++;
            else work.fresh_tiles++;
        }
        work.tiles = tiles;
        work.tile_halo = H;
        work.reinserted = 0;
        for (const Delaunay &d : work.dts) work.reinserted += d.reinserted;
        break;
    }
    // triangles (when the host builds their list): concatenation of the
    // slabs' lists
    const bool host_tris = work.host_edges;
    std::vector<int64_t> toff(K + 1, 0);
    for (int s = 0; s < K; s++) toff[s + 1] = toff[s] + (host_tris ? (int64_t)res[s].tris.size() / 3 : 0);
    m.tri.resize(3 * (size_t)toff[K]);
    // ring offsets
    // (tiles own disjoint cells: each writes its own cells' degrees; a cell
    // no tile wrote keeps degree 0 and fails the check)
    m.cell_ptr.resize((size_t)n + 1);
    {
        const int64_t zc = 65536, nzc = ((int64_t)n + 1 + zc - 1) / zc;
        auto zero = [&](int64_t c) {
            std::fill(m.cell_ptr.begin() + c * zc, m.cell_ptr.begin() + std::min<int64_t>(n + 1, (c + 1) * zc), 0);
        };
        if (pool && nzc > 1) pool->parallel_for(nzc, zero);
        else
            for (int64_t c = 0; c < nzc; c++) zero(c);
    }
    auto degs = [&](int64_t s) {
        for (size_t k = 0; k < res[s].cells.size(); k++) m.cell_ptr[res[s].cells[k] + 1] = res[s].deg[k];
    };
    if (pool && K > 1) pool->parallel_for(K, degs);
    else
        for (int s = 0; s < K; s++) degs(s);
    size_t owned = 0;
    for (int s = 0; s < K; s++) owned += res[s].cells.size();
    if (owned != (size_t)n) return -3;
    {
        // prefix sum of the degrees: chunk sums, their prefix, chunk scans
        const int64_t pc = 16384, npc = (n + pc - 1) / pc;
        std::vector<int64_t> csum(npc + 1, 0);
        std::vector<int> low(npc, 0);
        auto sums = [&](int64_t c) {
            int64_t t = 0;
            for (int64_t i = c * pc; i < std::min<int64_t>(n, (c + 1) * pc); i++) {
                if (m.cell_ptr[i + 1] < 3) low[c] = 1;
                t += m.cell_ptr[i + 1];
            }
            csum[c + 1] = t;
        };
        if (pool && npc > 1) pool->parallel_for(npc, sums);
        else
            for (int64_t c = 0; c < npc; c++) sums(c);
        for (int64_t c = 0; c < npc; c++) {
            if (low[c]) return -3;
            csum[c + 1] += csum[c];
        }
        if (csum[npc] > INT32_MAX) return -3;
        auto scan = [&](int64_t c) {
            int64_t run = csum[c];
            for (int64_t i = c * pc; i < std::min<int64_t>(n, (c + 1) * pc); i++) {
                run += m.cell_ptr[i + 1];
                m.cell_ptr[i + 1] = (int32_t)run;
            }
        };
        if (pool && npc > 1) pool->parallel_for(npc, scan);
        else
            for (int64_t c = 0; c < npc; c++) scan(c);
    }
    const size_t S = (size_t)m.cell_ptr[n];
    m.slot_nb.resize(S);
    m.slot_tri.resize(host_tris ? S : 0);
    // edges: each physical edge once, owned by its smaller real cell; a
    // periodic edge between a cell and its own copy by the +shift slot
    auto owns = [&](int32_t i, int32_t j) -> int {  // 1 own, 0 partner's, -1 inconsistent
        if (j < n) return j > i ? 1 : (j < i ? 0 : -1);
        if (box.boundary != 1) return 1;
        const int32_t gq = j - n;
        const int32_t src = m.ghost_src[gq];
        if (src != i) return src > i ? 1 : 0;
        const int32_t sh = m.ghost_shift[gq];
        const int32_t sx = sh % 3 - 1, sy = sh / 3 - 1;
        return (sy < 0 || (sy == 0 && sx < 0)) ? 0 : 1;
    };
    // owned edges per cell (kept in edge_off for the device-built list) and,
    // for a device-built triangle list, owned triangles per cell: those of
    // the cell's ring slots whose other two vertices have larger ids; both
    // counted while each tile's rings are placed (still in cache)
    m.edge_off.resize((size_t)n + 1);
    m.tri_off.resize(host_tris ? 0 : (size_t)n + 1);
    std::vector<int> tile_bad(K, 0);
    auto fill = [&](int64_t s) {
        const SlabResult &r = res[s];
        size_t q = 0;
        int self = 0;
        if (host_tris) std::copy(r.tris.begin(), r.tris.end(), m.tri.begin() + 3 * toff[s]);
        for (size_t k = 0; k < r.cells.size(); k++) {
            const int32_t i = r.cells[k], d = r.deg[k];
            const int32_t *ring = r.nb.data() + q;
            std::copy(ring, ring + d, m.slot_nb.begin() + m.cell_ptr[i]);
            if (host_tris)
                for (int32_t j = 0; j < d; j++) m.slot_tri[m.cell_ptr[i] + j] = (int32_t)(toff[s] + r.tri[q + j]);
            int32_t ke = 0;
            for (int32_t j = 0; j < d; j++) {
                const int32_t nb = ring[j];
                if (nb < n) {
                    // a real neighbour: without a branch on the comparison,
                    // whose outcome is random
                    ke += nb > i;
                    self |= nb == i;
                    continue;
                }
                const int o = owns(i, nb);
                if (o < 0) self = 1;
                ke += o > 0;
            }
            m.edge_off[i] = ke;
            if (!host_tris) {
                int32_t kt = 0;
                for (int32_t j = 0; j < d; j++) kt += (ring[j] > i) & (ring[j + 1 < d ? j + 1 : 0] > i);
                m.tri_off[i] = kt;
            }
            q += d;
        }
        if (self) tile_bad[s] = 1;
    };
    if (pool && K > 1) pool->parallel_for(K, fill);
    else
        for (int s = 0; s < K; s++) fill(s);
    for (int s = 0; s < K; s++)
        if (tile_bad[s]) return -3;
    lap(2);
    const int64_t chunk = 8192;
    static_assert(8192 % kOrderWindow == 0, "ordering windows must not straddle chunks");
    const int64_t nchunks = (n + chunk - 1) / chunk;
    std::vector<int64_t> ecount(nchunks + 1, 0), tcount(nchunks + 1, 0);
    auto sums = [&](int64_t c) {
        int64_t e = 0, tc = 0;
        for (int32_t i = (int32_t)(c * chunk); i < std::min<int64_t>(n, (c + 1) * chunk); i++) {
            e += m.edge_off[i];
            if (!host_tris) tc += m.tri_off[i];
        }
        ecount[c + 1] = e;
        tcount[c + 1] = tc;
    };
    if (pool) pool->parallel_for(nchunks, sums);
    else
        for (int64_t c = 0; c < nchunks; c++) sums(c);
    for (int64_t c = 0; c < nchunks; c++) {
        ecount[c + 1] += ecount[c];
        tcount[c + 1] += tcount[c];
    }
    const size_t E = (size_t)ecount[nchunks];
    if (E > (size_t)INT32_MAX / 2 || (size_t)tcount[nchunks] > (size_t)INT32_MAX / 3) return -3;
    m.n_edges = (int32_t)E;
    m.n_tris = host_tris ? (int32_t)(m.tri.size() / 3) : (int32_t)tcount[nchunks];
    // counts -> offsets: each chunk from its own start
    auto offsets = [&](int64_t c) {
        int64_t run = ecount[c], trun = tcount[c];
        for (int32_t i = (int32_t)(c * chunk); i < std::min<int64_t>(n, (c + 1) * chunk); i++) {
            const int32_t k = m.edge_off[i];
            m.edge_off[i] = (int32_t)run;
            run += k;
            if (!host_tris) {
                const int32_t kt = m.tri_off[i];
                m.tri_off[i] = (int32_t)trun;
                trun += kt;
            }
        }
    };
    if (pool) pool->parallel_for(nchunks, offsets);
    else
        for (int64_t c = 0; c < nchunks; c++) offsets(c);
    m.edge_off[n] = (int32_t)E;
    if (!host_tris) m.tri_off[n] = m.n_tris;
    if (!work.host_edges) {
        // the device builds the list; the processing order is still needed
        m.slot_edge.clear();
        m.edge_l.clear();
        m.edge_r.clear();
        m.edge_ta.clear();
        m.edge_tb.clear();
        m.cell_order.resize(n);
        auto order = [&](int64_t c) {
            const int32_t i0 = (int32_t)(c * chunk), i1 = (int32_t)std::min<int64_t>(n, (c + 1) * chunk);
            degree_order(i1 - i0, m.cell_ptr.data() + i0, m.cell_order.data() + i0);
            for (int32_t i = i0; i < i1; i++) m.cell_order[i] += i0;
        };
        if (pool) pool->parallel_for(nchunks, order);
        else
            for (int64_t c = 0; c < nchunks; c++) order(c);
        work.n_kept = n;
        lap(3);
        return 0;
    }
    m.slot_edge.assign(S, -1);
    m.edge_l.resize(E);
    m.edge_r.resize(E);
    m.edge_ta.resize(E);
    m.edge_tb.resize(E);
    auto place = [&](int64_t c) {
        int64_t e = ecount[c];
        for (int32_t i = (int32_t)(c * chunk); i < std::min<int64_t>(n, (c + 1) * chunk); i++) {
            const int32_t lo = m.cell_ptr[i], deg = m.cell_ptr[i + 1] - lo;
            for (int32_t k = 0; k < deg; k++) {
                const int32_t s = lo + k, j = m.slot_nb[s];
                if (owns(i, j) <= 0) continue;
                m.edge_l[e] = i;
                m.edge_r[e] = j;
                m.edge_ta[e] = m.slot_tri[lo + (k + deg - 1) % deg];
                m.edge_tb[e] = m.slot_tri[s];
                m.slot_edge[s] = (int32_t)(2 * e);
                // the same edge seen from the other cell's ring
                int32_t pc = -1;
                if (j < n) pc = j;
                else if (box.boundary == 1) pc = m.ghost_src[j - n];
                if (pc >= 0) {
                    int32_t want_shift = -1;
                    if (j >= n) {
                        const int32_t sh = m.ghost_shift[j - n];
                        want_shift = (-(sh % 3 - 1) + 1) + 3 * (-(sh / 3 - 1) + 1);
                    }
                    for (int32_t q = m.cell_ptr[pc]; q < m.cell_ptr[pc + 1]; q++) {
                        const int32_t c2 = m.slot_nb[q];
                        const bool hit = j < n ? c2 == i
                                               : (c2 >= n && m.ghost_src[c2 - n] == i && m.ghost_shift[c2 - n] == want_shift &&
                                                  q != s);
                        if (hit) {
                            m.slot_edge[q] = (int32_t)(2 * e + 1);
                            break;
                        }
                    }
                }
                e++;
            }
        }
    };
    if (pool) pool->parallel_for(nchunks, place);
    else
        for (int64_t c = 0; c < nchunks; c++) place(c);
    // every slot has its edge; the processing order, one window per task
    std::vector<int> missing(nchunks, 0);
    m.cell_order.resize(n);
    auto finish = [&](int64_t c) {
        const int32_t i0 = (int32_t)(c * chunk), i1 = (int32_t)std::min<int64_t>(n, (c + 1) * chunk);
        for (int32_t s = m.cell_ptr[i0]; s < m.cell_ptr[i1]; s++)
            if (m.slot_edge[s] < 0) missing[c] = 1;
        // chunk is a multiple of kOrderWindow: windows never straddle chunks
        degree_order(i1 - i0, m.cell_ptr.data() + i0, m.cell_order.data() + i0);
        for (int32_t i = i0; i < i1; i++) m.cell_order[i] += i0;
    };
    if (pool) pool->parallel_for(nchunks, finish);
    else
        for (int64_t c = 0; c < nchunks; c++) finish(c);
    for (int64_t c = 0; c < nchunks; c++)
        if (missing[c]) return -3;
    work.n_kept = n;
    lap(3);
    return 0;
}

}  // namespace rich
