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
    std::vector<int32_t> ghost_img;     // which image of its source: (a+1) + 3*(b+1), a, b in {-1, 0, 1}
    std::vector<int32_t> tri;           // 3 per triangle touching a real cell (point ids; ghosts n..n+g-1)
    std::vector<int32_t> cell_ptr;      // n+1 ring offsets
    std::vector<int32_t> slot_nb;       // neighbour point id
    std::vector<int32_t> slot_tri;      // triangle (i, nb[k], nb[k+1])
    // tri and slot_tri are filled only with MeshWork::host_edges; otherwise
    // the device builds them from the rings, and the host gives tri_off
    // (n+1): the first triangle owned by each cell, a triangle being owned by
    // its smallest vertex id (always a real cell: ghost ids follow the real
    // ones) and numbered in its owner's ring order
    std::vector<int32_t> tri_off;
    int32_t n_tris = 0;
    std::vector<int32_t> slot_edge;     // 2*edge + (1 if the cell is the edge's right side)
    std::vector<int32_t> edge_l, edge_r;   // left (real) and right (real or ghost) points
    std::vector<int32_t> edge_ta, edge_tb; // Voronoi edge runs from cc[ta] to cc[tb], ccw about left
    std::vector<int32_t> cell_order;    // processing order of the per-cell kernels (see degree_order)
    std::vector<int32_t> edge_off;      // n+1: first edge owned by each cell (edges in ring order)
    int32_t n_edges = 0;
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

    // Vertices, corners included (corner() .. corner() + 2), and positions.
    int32_t size() const { return (int32_t)px_.size(); }
    int32_t corner() const { return corner_; }
    bool is_corner(int32_t v) const { return v >= corner_ && v < corner_ + 3; }
    double x(int32_t v) const { return px_[v]; }
    double y(int32_t v) const { return py_[v]; }
    const double *xs() const { return px_.data(); }
    const double *ys() const { return py_.data(); }

    // Triangle slots written since the last clear_log() (log_all(): every
    // slot, after a build): only the stars of their vertices can have
    // changed.  Moving vertices (move_all without flips) writes none.
    bool log_all() const { return log_all_; }
    const std::vector<int32_t> &log() const { return log_; }
    void clear_log()
    {
        log_.clear();
        log_all_ = false;
    }

    // Updating a built triangulation for moved points (the points keep their
    // vertex numbers).  move_all moves every vertex to (nx[v], ny[v]); where
    // that would turn triangles over it puts their vertices back until none
    // is, flips to Delaunay, takes those vertices out (flipping their edges
    // away until three are left, then merging the three triangles) and
    // inserts them again at their new positions.  It returns false if that
    // needs more than max_back vertices or fails (the caller then builds
    // afresh); on success the triangulation is the unique (tie-broken)
    // Delaunay one of the new positions.  make_delaunay flips edges until
    // every edge is locally Delaunay (Lawson), which from any triangulation
    // of the same points ends at that one; given `seed`, it starts from the
    // edges of those triangles only (valid when every other edge is locally
    // Delaunay already).  insert_point adds a point after
    // the corners (returns the new vertex, -2 for a point that coincides
    // with one, -3 if location fails).
    bool move_all(const std::vector<double> &nx, const std::vector<double> &ny, int32_t max_back);
    void make_delaunay(const std::vector<int32_t> *seed = nullptr);
    int32_t insert_point(double x, double y);
    // vertices taken out and inserted again by move_all, over the object's life
    int64_t reinserted = 0;

private:
    int locate(int32_t p, int32_t &t, int &edge);
    void insert_inside(int32_t t, int32_t p);
    void insert_on_edge(int32_t t, int k, int32_t p);
    void legalize(int32_t p);
    int incircle(int32_t t, int32_t d) const;
    void set_nb(int32_t t, int32_t old_nb, int32_t new_nb);
    void alloc2(int32_t &a, int32_t &b);
    bool flip_ok(int32_t t, int k) const;
    void flip(int32_t t, int k);
    bool remove_vertex(int32_t v, int32_t t);
    int insert_at(int32_t v);

    std::vector<double> px_, py_;
    std::vector<int32_t> order_;
    std::vector<int32_t> stack_;
    std::vector<int64_t> edges_;
    std::vector<int32_t> free_;
    std::vector<int32_t> touched_;  // triangles remove_vertex rewrote
    std::vector<int32_t> rewritten_;  // all of them, over one move_all
    // move_all's scratch: old positions, the vertices put back, and a
    // triangle of each
    std::vector<double> old_x_, old_y_;
    std::vector<uint8_t> back_;
    std::vector<int32_t> back_list_, where_;
    void note(int32_t t)
    {
        if (!log_all_) log_.push_back(t);
    }
    std::vector<int32_t> log_;
    bool log_all_ = true;
    int32_t corner_ = 0;
    int32_t hint_ = 0;
    uint32_t rng_ = 12345u;
};

// A tile of the point set: x in [x0, x1), y in [y0, y1); open sides (the
// first / last along an axis) extend to infinity.
struct Tile {
    double x0, x1, y0, y1;
    bool fx, lx, fy, ly;
};

// One tile's part of a build: the stars of its real core points, and the
// buffers the tile works in.  Kept per tile from build to build, so that a
// build reuses their capacity instead of allocating (and page-faulting) the
// same sizes again.
struct TileStars {
    int rc = 0;
    bool halo_ok = true, band_ok = true;
    double needed = 0.0;          // how far the stars' circumdisks reach past the tile
    std::vector<int32_t> cells;   // real core cells
    std::vector<int32_t> deg;     // ring length of each
    std::vector<int32_t> nb;      // concatenated rings: neighbour point ids
    std::vector<int32_t> tri;     // concatenated rings: tile-local triangle number
    std::vector<int32_t> tris;    // 3 per tile-local triangle (point ids)
    // the last read-off's output by local vertex: where the vertex's ring
    // starts in nb (-1: not a core vertex then) and its length, and each
    // local vertex's point id then; the next ones are written beside them
    // and swapped in (nb_prev holds the last output while the next is
    // written)
    std::vector<int32_t> out_off, out_len, next_off, next_len, prev_loc, nb_prev;
    // scratch of the read-off: core flags, triangle numbers, rings to walk
    // again, and a triangle slot holding each local vertex (kept between
    // read-offs, updated from the triangulation's log)
    std::vector<uint8_t> core, dirty;
    std::vector<int32_t> tnum, vt;
    // scratch of the in-place update: the local vertices' new positions
    std::vector<double> nx, ny;
    void reset()
    {
        rc = 0;
        halo_ok = band_ok = true;
        needed = 0.0;
        // (nb and tri keep their size: they are read only through cells
        // and deg, and a read-off sets them)
        cells.clear();
        deg.clear();
        tris.clear();
    }
};

// Reusable buffers of build_host_mesh (one triangulator per tile), and what
// the next build needs to update each tile's triangulation instead of
// building it again.
struct MeshWork {
    std::vector<Delaunay> dts;
    std::vector<TileStars> stars;
    std::vector<std::vector<int32_t>> loc;
    std::vector<std::vector<double>> lx, ly;
    // the points bucketed on uniform grids (ids in increasing order within a
    // bucket), so that a tile gathers its points from the buckets it
    // overlaps instead of testing every point: the real points on a grid
    // over the box, kept from build to build while they have moved less
    // than half a bucket since (grid_slack: the sum over builds of the
    // largest move of a coordinate; grid_n: the point count it holds, -1
    // none), the ghosts on a grid of their own every build
    struct GridBufs {
        std::vector<int32_t> start, ids, cell, hist;
        int G = 1;
        double x0 = 0.0, y0 = 0.0, sx = 0.0, sy = 0.0;
    };
    GridBufs grid_real, grid_ghost;
    double grid_slack = 0.0;
    int32_t grid_n = -1;
    // real then ghost coordinates of the current build
    std::vector<double> X, Y;
    double halo = 0.0;  // slab halo of the last build, in mean point spacings
    // update in place (false: every build inserts every point again)
    bool kinetic = true;
    // build the edge list (slot_edge, edge_l/r/ta/tb) and the triangle list
    // (tri, slot_tri) on the host; false: only edge_off, n_edges, tri_off and
    // n_tris, for a device that builds both lists itself
    bool host_edges = true;
    // the last build's tiles, their halos, and per tile the key of every
    // local vertex: its real point's id, n + 9 src + image for a ghost (the
    // image of real point src, see HostMesh::ghost_img), -2 for a corner of
    // the enclosing triangle; n_kept = the real count they refer to (-1: none)
    std::vector<Tile> tiles;
    std::vector<double> tile_halo;
    std::vector<std::vector<int64_t>> keys;
    int32_t n_kept = -1;
    // per tile: build stamp of each point present (sized to the points)
    std::vector<std::vector<uint32_t>> stamp;
    uint32_t gen = 0;
    // new ghost index of each ghost key, valid where gkey_stamp == gen
    std::vector<int32_t> gkey_idx;
    std::vector<uint32_t> gkey_stamp;
    // tiles updated in place and tiles built afresh, over all builds
    int64_t kinetic_tiles = 0, fresh_tiles = 0;
    // vertices taken out and put back by the updates, over all builds
    int64_t reinserted = 0;
    // wall time of the last build's phases (ms): ghosts, point copies,
    // bounding box and bucket grid; the tiles (triangulation, star checks,
    // rings per tile); triangle and ring assembly; edge counts and order
    double phase_ms[4] = {0.0, 0.0, 0.0, 0.0};
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
