// Device data of one simulation and the launchers of the sweep kernels
// (steps a1-a9 of one extrapolated-fluxes time step, paper Section 2.3).
//
// The sweep is instantiated for two reconstruction precisions R:
//   R = double  every step in FP64;
//   R = float   split precision: primitives, gradients, limiter, mesh
//               velocity, edge states and HLLC in FP32, while positions,
//               Voronoi vertices, areas, centres of mass, the coordinate
//               differences feeding every edge quantity, and the conserved
//               variables (with the flux accumulation) stay in FP64.
//
// Layout in HBM (cells in Hilbert order):
//   points     x[2][n], y[2][n] ping-pong real generators (FP64); gx, gy ghosts
//   state      U[2][4*n] ping-pong extensive (m, Px, Py, E), component-major, FP64
//   mesh       tri[3*T]; cell_ptr[n+1]; slot_nb/slot_tri/slot_edge[S];
//              edge_l/edge_r/edge_ta/edge_tb[E]; ghost_src/ghost_xf[g]
//   geometry   ccx, ccy[T] (FP64); A[n] (FP64); per edge (R): L, unit normal
//              (nx, ny), q = c_ij/|r_ij| (qx, qy), midpoint minus left
//              generator (mlx, mly) and minus right generator (mrx, mry);
//              ePM[E] = {P, M}: Eq. 1 as a sum over neighbours reads
//              g_i = (sum_j phi_j P_ij + phi_i sum_j M_ij)/A_i with
//              P = L(q + n/2), M = L(n/2 - q) (right cells use -M, -P)
//   order      cell_order[n]: per-cell kernels visit cells in this order
//   cell (R)   W[n] = {rho, vx, vy, p}; o[n] = centre of mass - generator;
//              cs[n]; gl[2n] limited gradient {drho/dx, drho/dy, dvx/dx,
//              dvx/dy}, {dvy/dx, dvy/dy, dp/dx, dp/dy}; w[n] mesh velocity;
//              psrc[n] cell terms of the half-step prediction;
//              diagnostics g[2n] (unlimited), alpha[n], tess[n];
//              rounding[n] (uint8) and, in split precision, p64[n] (FP64):
//              the two discontinuous decisions of the step (rounding trigger,
//              pressure-ratio switch) are taken on FP64 values
//   flux       F[E] = L_ij * F_ij (mass, momentum x, y, energy), outward
//              from the edge's left cell, in R: in split precision the FP32
//              flux is stored as computed and the update widens it exactly
//              (integer pipe) into its FP64 sums, so both cells of an edge
//              add the same FP64 value
//   per sim    inst[] scheme parameters and remaining time; dtmin (bits of the
//              smallest cell time step), dt, status
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rich {

enum : int32_t {
    ST_NEGATIVE = 1,  // m <= 0 or thermal energy <= 0
    ST_NAN = 2,       // non-finite value
    ST_LEFT_BOX = 4,  // a generating point crossed a wall
};

template <class R> struct alignas(4 * sizeof(R)) Vec4 { R x, y, z, w; };
template <class R> struct alignas(2 * sizeof(R)) Vec2 { R x, y; };

// Scheme parameters of one simulation of a batch (device table).
struct InstParams {
    double gamma, cfl, chi, eta, theta, delta_v, delta_p;
    double x0, x1, y0, y1;
    double remaining;  // t_end - t: the step is shortened to land on t_end
    double igm1;       // 1/(gamma - 1)
    int32_t boundary, motion, limiter;
    int32_t init;      // the geometry stage with primitives given sets this simulation's U
    // Section 2.3 time advancement of this sweep: 0 extrapolated fluxes (edge
    // states advanced dt/2 in time, full update); 1 first sweep of the
    // time-centred scheme (spatial extrapolation only, Courant dt, half
    // update); 2 its second sweep (spatial extrapolation only, the dt of
    // sweep 1 from dt_out, full update)
    int32_t phase;
    // gamma, 1/(gamma - 1), chi, theta and delta_v rounded to FP32 (by the
    // host), for the split-precision stages
    float gamma_f, igm1_f, chi_f, theta_f, delta_v_f;
    int32_t pad;
};

template <class R> struct SweepParams {
    // per-simulation parameters; cell_inst[i] names the simulation of real
    // cell i (nullptr: every cell belongs to simulation 0)
    const InstParams *inst;
    const int32_t *cell_inst;
    int32_t n_inst, diagnostics;
    // 1 in a sweep, where the geometry stage also takes the mesh velocity
    // and the Courant candidates (a5, a6); 0 when only the geometry of the
    // current points is wanted (the last sweep's velocities are kept)
    int32_t motion;
    // sizes (all simulations together)
    int32_t n, ng, T, E, S;
    // points (current and next), FP64
    const double *x, *y;
    double *xn, *yn;
    const double *gx, *gy;
    // mesh
    const int32_t *tri, *cell_ptr, *slot_nb, *slot_tri, *slot_edge;
    // processing order of the per-cell stages: thread k handles cell
    // cell_order[k] (cells of equal ring degree side by side in a warp)
    const int32_t *cell_order;
    const int32_t *edge_l, *edge_r, *edge_ta, *edge_tb;
    const int32_t *ghost_src, *ghost_xf;
    // geometry
    double *ccx, *ccy, *A;
    R *eL, *enx, *eny, *eqx, *eqy, *emlx, *emly, *emrx, *emry;
    Vec4<R> *ePM;  // Eq. 1 weights of the edge's left cell: P = L(q + n/2), M = L(n/2 - q)
    // state: U gives the primitives, the update writes Un = U0 - dt... and
    // xn = x0 + dt w (U0 = U and x0 = x except in the time-centred scheme's
    // second sweep, which starts again from the state at the start of the step)
    const double *U;
    double *Un;
    const double *U0, *x0, *y0;
    Vec4<R> *W;
    Vec2<R> *o;
    R *cs;
    uint8_t *rounding;  // 1 where the Section 6 rounding velocity is on (decided in FP64)
    double *p64;        // FP64 pressure for the shock switch (split precision only)
    Vec4<R> *gl, *g, *alpha;
    // per cell, from the limited gradient: the cell-only terms of the
    // half-step prediction {rho div v, (dp/dx)/rho, (dp/dy)/rho, gamma p div v}
    Vec4<R> *psrc;
    Vec2<R> *w;
    int32_t *tess;
    Vec4<R> *F;  // L_ij F_ij in the reconstruction precision (see the flux layout)
    // per simulation: bits of the smallest cell time step, the step taken,
    // status flags
    unsigned long long *dtmin_bits;
    double *dt_out;
    int32_t *status;
};

// Stages of one step, in launch order.  GEOMETRY_STAGES = a1 + a2;
// the remaining stages are a9 and a3-a8.  The points' motion needs only the
// mesh velocity and the step's dt, both known once the geometry stage is
// done, so the new points are written before the gradients and fluxes:
// a caller can read them, and build the next mesh on the host, while the
// rest of the sweep runs.
enum Stage : int {
    K_CIRCUMCENTRE = 0,   // a1 Voronoi vertices (and clears the time-step minimum)
    K_GEOMETRY = 1,       // a1 + a2 in one launch: per-edge L, midpoint, normal,
                          // c_ij/|r_ij| (the first blocks) and per-cell area,
                          // centre of mass, primitives, then (in a sweep) a5
                          // mesh velocity and a6 Courant candidates (the rest)
    K_ADVANCE = 2,        // a9 point motion, dt recorded
    K_CELL_GRADIENT = 3,  // a3-a4 gradients, limiter, prediction terms
    K_EDGE_FLUX = 4,      // a7 predicted edge states + HLLC
    K_CELL_UPDATE = 5,    // a8 conservative update
    NUM_STAGES = 6,
    GEOMETRY_STAGES = 2,
};

const char *stage_name(int k);

// Launch one stage.  For K_GEOMETRY a non-null init_W (4*n FP64 primitives,
// component-major) sets the conserved variables from it instead.
template <class R> void launch_stage(int k, const SweepParams<R> &p, const double *init_W, cudaStream_t st);

// Sizes of the packed mesh, read by the persistent sweep from device memory
// so that one recorded launch serves every step.
struct DeviceSizes {
    int32_t n, ng, T, E, n_inst, pad[3];
};

// State of the persistent sweep's grid barrier (zeroed before each launch).
struct GridSync {
    unsigned int count, gen;
    int32_t timeout;     // set when a barrier wait gave up; the sweep then stops
    int32_t spin_limit;  // polls before a wait gives up (0: about a second's worth)
    int32_t extra;       // blocks the barrier waits for beyond the grid (0; a
                         // test sets 1 to make every wait run out)
    int32_t pad[3];
};

// The whole step a1-a9 in one cooperative launch of `grid` blocks of `block`
// threads (grid <= co-resident blocks): grid-stride loops over triangles,
// edges and cells, separated by four grid barriers whose waits give up after
// about a second (GridSync::timeout); the point motion runs beside the
// gradients, between the second and third barriers.
template <class R>
cudaError_t launch_persistent(const SweepParams<R> &p, const DeviceSizes *sizes, GridSync *sync, int block, int grid,
                              cudaStream_t st);
// Co-resident blocks per SM of the persistent sweep for a block size.
template <class R> int persistent_blocks_per_sm(int block);

// U_new[c][i] = U_old[c][src[i]] for the 4 components (component-major
// arrays of n_old and n_new cells); cells with src[i] < 0 are left alone.
void launch_repack(const int32_t *src, int32_t n_new, int32_t n_old, const double *U_old, double *U_new,
                   cudaStream_t st);

// The triangle list from the rings, on the device.  The triangle of ring
// slot k of real cell i is (i, nb[k], nb[k+1]); it is owned by its smallest
// vertex id (a real cell: ghost ids follow the real ones), numbered in its
// owner's ring order from tri_off[owner] (tri_off[n] = T, from the host) and
// written rotated to start at the owner, as the host builder writes it.
// Writes tri (3 T) and slot_tri (S), and sets *bad to 1 if a cell owns more
// or fewer triangles than tri_off gives, if a slot's triangle is missing
// from its owner's ring, or if a slot ends without a triangle.
cudaError_t launch_build_tris(int32_t n, int32_t S, const int32_t *cell_ptr, const int32_t *slot_nb,
                              const int32_t *tri_off, int32_t *tri, int32_t *slot_tri, int32_t *bad, cudaStream_t st);

// The edge list from the rings, on the device (the host then ships rings
// only).  Real cell i owns its edges to larger real cells, to mirror images
// and (periodic box) to images of larger cells or of itself shifted to the
// +x / +y side; its owned edges are numbered in ring order from
// edge_off[i] (edge_off[n] = E, from the host).  Writes slot_edge (2 e, or
// 2 e + 1 on the partner's slot), edge_l / edge_r / edge_ta / edge_tb
// (Voronoi edge from circumcentre ta to tb, counter-clockwise about the
// left cell), and sets *bad to 1 if a slot ends without an edge.  S slots
// in all; the ghost arrays are read only for a periodic box.  In a packed
// batch (cell_inst non-null) each cell's box type comes from its
// simulation's parameters instead of `periodic`.
cudaError_t launch_build_edges(int32_t n, int32_t S, const int32_t *cell_ptr, const int32_t *slot_nb,
                               const int32_t *slot_tri, const int32_t *ghost_src, const int32_t *ghost_shift,
                               const int32_t *edge_off, int32_t periodic, const InstParams *inst,
                               const int32_t *cell_inst, int32_t *slot_edge, int32_t *edge_l, int32_t *edge_r,
                               int32_t *edge_ta, int32_t *edge_tb, int32_t *bad, cudaStream_t st);

}  // namespace rich
