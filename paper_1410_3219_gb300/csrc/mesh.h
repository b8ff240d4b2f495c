// Host-side tessellation (paper Section 2.1) producing the connectivity the
// device sweep consumes.
//
//   1. ghost images of the real generating points inside a band of width w
//      around the box: mirror images across reflecting walls (corners mirrored
//      twice) or shifted copies for a periodic box;
//   2. Delaunay triangulation of real + ghost points by incremental point
//      insertion with Lawson edge flips, exact tie-broken predicates,
//      Hilbert-curve insertion order and walking point location;
//   3. a band check: every triangle that touches a real point must have its
//      circumdisk inside the band, so that every real cell's neighbourhood
//      equals that of the infinite mirrored / periodic point set; otherwise w
//      doubles and the construction repeats;
//   4. per real cell, its neighbours in counter-clockwise order starting at
//      the smallest neighbour id; per ring slot
//      the triangle (i, nb[k], nb[k+1]) whose circumcentre is the Voronoi
//      vertex after that slot; and a list of Voronoi edges in which every
//      physical edge appears once (periodic copies of one edge are merged).
#pragma once

#include <cstdint>
#include <vector>

namespace rich {

struct BoxConfig {
    int boundary;  // 0 reflecting walls, 1 periodic
    double x0, x1, y0, y1;
};

// ghost transform flags
enum : int32_t {
    XF_MIRROR_X = 1,   // velocity x and d/dx of scalars change sign
    XF_MIRROR_Y = 2,
};

struct HostMesh {
    int32_t n = 0;                      // real cells
    int32_t g = 0;                      // ghost points
    std::vector<double> gx, gy;         // ghost positions
    std::vector<int32_t> ghost_src;     // real cell each ghost copies
    std::vector<int32_t> ghost_xf;      // XF_* flags
    std::vector<int32_t> ghost_shift;   // periodic shift code: (sx+1) + 3*(sy+1)
    std::vector<int32_t> tri;           // 3 per triangle touching a real cell (point ids; ghosts n..n+g-1)
    std::vector<int32_t> cell_ptr;      // n+1 ring offsets
    std::vector<int32_t> slot_nb;       // neighbour point id
    std::vector<int32_t> slot_tri;      // triangle (i, nb[k], nb[k+1])
    std::vector<int32_t> slot_edge;     // 2*edge + (1 if the cell is the edge's right side)
    std::vector<int32_t> edge_l, edge_r;   // left (real) and right (real or ghost) points
    std::vector<int32_t> edge_ta, edge_tb; // Voronoi edge runs from cc[ta] to cc[tb], ccw about left
    std::vector<int32_t> cell_order;    // processing order of the per-cell kernels (see degree_order)
    double band = 0.0;
    int attempts = 0;
};

struct Tri {
    int32_t v[3];   // counter-clockwise
    int32_t nb[3];  // nb[k]: triangle across the edge opposite v[k], -1 if none
};

class Delaunay {
public:
    // Triangulate np distinct points.  Returns 0, or -2 for coincident points,
    // -3 if the construction failed.  Vertices np..np+2 are the corners of an
    // enclosing triangle.
    int build(const double *x, const double *y, int32_t np);
    std::vector<Tri> tris;

private:
    int locate(int32_t p, int32_t &t, int &edge);
    void insert_inside(int32_t t, int32_t p);
    void insert_on_edge(int32_t t, int k, int32_t p);
    void legalize(int32_t p);
    int incircle(int32_t t, int32_t d) const;
    void set_nb(int32_t t, int32_t old_nb, int32_t new_nb);

    std::vector<double> px_, py_;
    std::vector<int32_t> order_;
    std::vector<int32_t> stack_;
    int32_t hint_ = 0;
    uint32_t rng_ = 12345u;
};

// Reusable buffers of build_host_mesh (one triangulator per slab).
struct MeshWork {
    std::vector<Delaunay> dts;
    std::vector<std::vector<int32_t>> loc;
    std::vector<std::vector<double>> lx, ly;
    // the points bucketed on a uniform grid over their bounding box (ids in
    // increasing order within a bucket), so that a tile gathers its points
    // from the buckets it overlaps instead of testing every point
    std::vector<int32_t> grid_start, grid_ids, grid_cell, grid_hist;
    double halo = 0.0;  // slab halo of the last build, in mean point spacings
};

class ThreadPool;

// Build the whole host mesh for n real points (x, y).  With a pool the real
// + ghost points are cut into tiles (columns at x-quantiles, rows at
// y-quantiles; one per thread, at least 16384 real points each); each tile
// is triangulated with a halo that widens by 1.5x until every circumdisk of
// its real points' stars lies inside it, so the stars equal those of the
// whole set, and the rings and the edge list are filled in parallel.
// Rings start at their smallest neighbour id and triangles at their
// smallest vertex id, so the mesh seen by the sweep does not depend on the
// number of tiles (only the triangle numbering does).  Returns 0, -2 for coincident points, -3 for a failed triangulation,
// -4 when the box holds too few points for the band check to succeed.
int build_host_mesh(const BoxConfig &box, int32_t n, const double *x, const double *y, MeshWork &work,
                    HostMesh &out, ThreadPool *pool = nullptr);

// Processing order for the per-cell device loops over ring slots: within
// each window of kOrderWindow consecutive cells, cells by decreasing ring
// degree (stable), so that the 32 cells of a warp have nearly equal degrees
// and the warp's loop runs close to their mean length rather than to the
// largest degree among 32 random ones.  Windows keep Hilbert locality.
constexpr int32_t kOrderWindow = 1024;
void degree_order(int32_t n, const int32_t *cell_ptr, int32_t *order);

// Order of points along a Hilbert curve over their bounding box.
void hilbert_order(int32_t n, const double *x, const double *y, std::vector<int32_t> &order);

}  // namespace rich
