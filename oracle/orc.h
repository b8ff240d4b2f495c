/*
 * ORACLE (test infrastructure only).  A plain, slow, single-threaded FP64
 * restatement of one time step of the moving-mesh Godunov scheme of
 * Yalinewich, Steinberg & Sari (RICH), Section 2, with the
 * "extrapolated fluxes" time advancement of Section 2.3.  Only the test
 * suite, the smoke check and the CPU baseline of the benchmark may load it;
 * the CUDA library never does.
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double gamma, cfl;
    int boundary; /* 0: reflecting walls, 1: periodic */
    double x0, x1, y0, y1;
    int motion; /* 0: Lagrangian + cell rounding (Section 6), 1: static (Eulerian) */
    double chi, eta;
    double theta, delta_v, delta_p;
    int limiter; /* 0: AREPO with switch to TESS near shocks, 1: AREPO, 2: TESS */
    int scheme;  /* Section 2.3: 0 extrapolated fluxes, 1 time-centred fluxes */
} orc_config;

typedef struct orc_sim orc_sim;

/* exact predicates (orc_exact.c) */
int orc_orient(double ax, double ay, double bx, double by, double cx, double cy);
int orc_incircle_raw(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy);
int orc_incircle_sos(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy);

/* Delaunay by point insertion (orc_delaunay.c) */
int orc_delaunay(int n, const double *x, const double *y, int *ntri, int **tris);
void orc_free(void *p);

/* simulation (orc_hydro.c) */
int orc_create(const orc_config *cfg, int n, const double *x, const double *y, const double *rho,
               const double *vx, const double *vy, const double *p, orc_sim **out);
void orc_destroy(orc_sim *s);
int orc_tessellate(orc_sim *s);
int orc_sweep(orc_sim *s, double t_end, double *dt_out);
int orc_step(orc_sim *s, double t_end, double *dt_out);
double orc_time(const orc_sim *s);
int orc_num_points(const orc_sim *s); /* real + ghost points of the last tessellation */
int orc_get_points(const orc_sim *s, double *X, double *Y, int *src);
int orc_ring_total(const orc_sim *s);
int orc_get_ring(const orc_sim *s, int *ptr, int *nb);
int orc_get_conserved(const orc_sim *s, double *x, double *y, double *m, double *px, double *py, double *E);
int orc_get_cells(const orc_sim *s, int field, double *out);
int orc_get_primitives(orc_sim *s, double *rho, double *vx, double *vy, double *p, double *area);
double orc_band(const orc_sim *s);

/* building blocks exposed for pins */
void orc_hllc(double gamma, const double WL[4], const double WR[4], double F[4]);
void orc_predict(double gamma, double hdt, const double W[4], const double g[8], double offx, double offy,
                 const double wf[2], double out[4]);
int orc_riemann_exact(double gamma, double rl, double ul, double pl, double rr, double ur, double pr,
                      double *ps, double *us);
void orc_riemann_sample(double gamma, double rl, double ul, double pl, double rr, double ur, double pr,
                        double ps, double us, double xi, double out[3]);

#ifdef __cplusplus
}
#endif
#endif
