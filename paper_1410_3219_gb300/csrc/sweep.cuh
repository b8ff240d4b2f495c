// Device data of one simulation and the launchers of the sweep kernels
// (steps a1-a9 of one extrapolated-fluxes time step, paper Section 2.3).
//
// Layout in HBM (structure of arrays, cells in Hilbert order):
//   points     x[2][n], y[2][n] ping-pong real generators; gx, gy ghost images
//   state      U[2][4*n] ping-pong extensive (m, Px, Py, E), component-major
//   mesh       tri[3*T]; cell_ptr[n+1]; slot_nb/slot_tri/slot_edge[S];
//              edge_l/edge_r/edge_ta/edge_tb[E]; ghost_src/ghost_xf[g]
//   geometry   ccx, ccy[T]; per edge L, midpoint-minus-left (mlx, mly),
//              midpoint-minus-right (mrx, mry), unit normal (nx, ny),
//              q = c_ij/|r_ij| (qx, qy); per cell A, centre of mass minus
//              generator (ox, oy)
//   cell       W[4*n] (rho, vx, vy, p), cs[n], g[8*n] unlimited and
//              gl[8*n] limited gradients (d/dx,d/dy of each primitive,
//              component-major), alpha[4*n], tess[n], wx, wy[n]
//   flux       F[4*E] = L_ij * F_ij, outward from the edge's left cell
//   scalars    dtmin (bits of the smallest positive cell time step), dt, status
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rich {

enum : int32_t {
    ST_NEGATIVE = 1,  // m <= 0 or thermal energy <= 0
    ST_NAN = 2,       // non-finite value
    ST_LEFT_BOX = 4,  // a generating point crossed a wall
};

struct SweepParams {
    // scheme
    double gamma, cfl, chi, eta, theta, delta_v, delta_p;
    double x0, x1, y0, y1;
    int32_t boundary, motion, limiter;
    // sizes
    int32_t n, ng, T, E, S;
    // points (current and next)
    const double *x, *y;
    double *xn, *yn;
    const double *gx, *gy;
    // mesh
    const int32_t *tri, *cell_ptr, *slot_nb, *slot_tri, *slot_edge;
    const int32_t *edge_l, *edge_r, *edge_ta, *edge_tb;
    const int32_t *ghost_src, *ghost_xf;
    // geometry
    double *ccx, *ccy;
    double *eL, *emlx, *emly, *emrx, *emry, *enx, *eny, *eqx, *eqy;
    double *A, *ox, *oy;
    // state
    const double *U;
    double *Un;
    double *W, *cs, *g, *gl, *alpha, *wx, *wy;
    int32_t *tess;
    double *F;
    // scalars
    unsigned long long *dtmin_bits;
    double *dt_out;
    int32_t *status;
    double remaining;  // t_end - t
};

// Stages of one step, in launch order.  GEOMETRY_STAGES = a1 + a2;
// the remaining stages are a3-a9.
enum Stage : int {
    K_CIRCUMCENTRE = 0,   // a1 Voronoi vertices
    K_EDGE_GEOMETRY = 1,  // a1 per-edge L, midpoint, normal, c_ij/|r_ij|
    K_CELL_GEOMETRY = 2,  // a1 + a2 area, centre of mass, primitives
    K_DT_RESET = 3,       // clears the time-step minimum (memset, not a kernel)
    K_CELL_GRADIENT = 4,  // a3-a6 gradients, limiter, mesh velocity, dt
    K_EDGE_FLUX = 5,      // a7 predicted edge states + HLLC
    K_CELL_UPDATE = 6,    // a8 + a9 conservative update, point motion
    NUM_STAGES = 7,
    GEOMETRY_STAGES = 3,
};

const char *stage_name(int k);

// Launch one stage.  For K_CELL_GEOMETRY a non-null init_W (4*n primitives,
// component-major) sets the conserved variables from it instead.
void launch_stage(int k, const SweepParams &p, const double *init_W, cudaStream_t st);

}  // namespace rich
