/*
 * CPU oracle for one timestep of the particle path of the non-hybrid PDF method
 * (Bakosi, Franzese & Boybeyi).  TEST INFRASTRUCTURE ONLY: plain, slow, FP64, single
 * thread.  Only the tests, the smoke check and the benchmark's CPU-baseline leg use it;
 * the library never calls it and shares no code with it.
 *
 * Every routine follows the paper's steps in the paper's order; the comments name the
 * section, equation or appendix that defines it.  Where the paper is silent or
 * ambiguous, the reading taken is stated at the routine.
 */
#ifndef PDFX_ORACLE_H
#define PDFX_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
    /* Table 4 */
    double C1, C2, C3, C4, CT, CL, Ceta, Cv, gamma5, Cw1, Cw2;
    double nu;                 /* kinematic viscosity */
    int    c0_mode;            /* 0: C0 from Eq. 11; 1: constant C0 */
    double C0;
    int    tm_mode;            /* 0: t_m from Eq. 25; 1: t_m = 2k / (Cphi eps) */
    double Cs, Ct, Cphi;
    double src_x, src_y, src_r;/* scalar source disc (Sect. 4.1.2): psi = 1 inside */
    int    bins[3];            /* requested conditioning bins per velocity component */
    int    min_per_bin;        /* minimum particles per bin (Sect. 3.5) */
    int    minnpel;            /* Appendix B threshold; 0 disables particle-number control */
    int    interp_mode;        /* 0: shapefunctions at X (Eq. 37); 1: element average */
    int    source_on;          /* 1: apply the source disc */
    uint64_t seed;             /* Philox key = (seed_lo, seed_hi ^ instance) */
    uint32_t instance;
    double period_x;           /* 0 = not periodic */
    int    cond_mode;          /* 0: hierarchical bins (Sect. 3.5, Appendix A); 1: Fox's
                                  projection (Eqs. 64-66) with fox_bins intervals */
    int    fox_bins;
    int    model;              /* 0: the full model; 1: the simplified model of Eqs. 46-47
                                  (particle-redistribution test, Sect. 3.7; no no-slip walls) */
    double alpha;              /* Eq. 47 */
    double cfl;                /* Eq. 26 CFL constant (a step with dt <= 0 takes Eq. 26's dt) */
} orc_params;

typedef struct orc_diag {
    long long hops_total, walk_fallback, walk_brute, lost;
    long long wall_hits, wall_hits_a, freeslip_hits, omega_reflect, c0_clamp, gamma_exhausted;
    long long moves, source_hits;
    long long hop_hist[8];     /* 0,1,2,3,4,5,6,7+ hops */
} orc_diag;

typedef struct orc_ctx orc_ctx;

/* Primitives (exposed so tests can pin them). */
void   orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t w);
void   orc_box_muller(uint32_t w1, uint32_t w2, double *g1, double *g2);
double orc_gamma_draw(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t step,
                      uint32_t purpose, double shape, double scale, int *exhausted);
void   orc_step_gaussians(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t step,
                          double xi[6], double *eta);

/* Context. */
int  orc_create(orc_ctx **out, const orc_params *p, int nn, const double *node_xy,
                int ne, const int32_t *tri, const int8_t *edge_tag);
void orc_destroy(orc_ctx *c);
int  orc_set_params(orc_ctx *c, const orc_params *p);
int  orc_set_fields(orc_ctx *c, const double *fields /* [nn][32] */);

/* Geometry queries (Sect. 3.4, 3.6). */
void orc_lambda(const orc_ctx *c, int e, double x, double y, double lam[3]);
int  orc_walk(orc_ctx *c, int e0, double x, double y, int *hops);
int  orc_brute_locate(const orc_ctx *c, double x, double y);
void orc_interp(const orc_ctx *c, int e, const double lam[3], double q[32]);
int  orc_neighbors(const orc_ctx *c, int32_t *nbr /* [ne][3] */);

/* Particles (stored by particle id). */
int  orc_init_particles(orc_ctx *c, int ppe);
int  orc_init_elements(orc_ctx *c, int ppe, int n, const int32_t *elems);
int  orc_set_particles_ids(orc_ctx *c, int np, const double *x, const double *y, const double *u,
                           const double *v, const double *w, const double *om, const double *psi,
                           const int32_t *elem, const uint32_t *pid, uint32_t step);
int  orc_get_pids(const orc_ctx *c, uint32_t *out);
int  orc_set_particles(orc_ctx *c, int np, const double *x, const double *y, const double *u,
                       const double *v, const double *w, const double *om, const double *psi,
                       const int32_t *elem, uint32_t step);
int  orc_get_particles(const orc_ctx *c, double *x, double *y, double *u, double *v, double *w,
                       double *om, double *psi, int32_t *elem, uint8_t *cp);
int  orc_num_particles(const orc_ctx *c);
uint32_t orc_step_index(const orc_ctx *c);

/* One timestep and its stages (Table 1 order restricted to the particle path).  Parity
 * unpinned as a whole: the paper prints no worked example of a full step.  Its stages are
 * pinned one by one, and whole steps run inside the pins that need them (Eq. 24's bin
 * means and deviation decay across the statistics and the advance, Eq. 11's energy rate,
 * Eq. 20's frequency source, the walls' reflection principle). */
int  orc_step(orc_ctx *c, double dt);   /* dt <= 0: the time step of Eq. 26 */
int  orc_cfl_dt(const orc_ctx *c, double *dt);
/* Sect. 3.4: node-transferred gradient of a nodal quantity q[nn] (Eqs. 39-40, then the mean
 * over the elements around each node): grad[nn][2]. */
void orc_node_gradient(const orc_ctx *c, const double *q, double *grad);
/* Nodal fields from the particles' nodal statistics (slots 0-2, 5-13, 23-29). */
int  orc_derive_fields(orc_ctx *c);
int  orc_get_fields(const orc_ctx *c, double *out /* [nn][32] */);
/* Eq. 31 (rho = 1) applied to the particles: U_i -= dt d(dP)/dx_i with the element-constant
 * gradient (Eqs. 39-40) of the nodal pressure change dP[nn] of the particle's element. */
int  orc_correct_velocity(orc_ctx *c, const double *dp, double dt);
double orc_last_dt(const orc_ctx *c);
/* Eqs. 12-18: the local right-hand side of Eq. 12 (rhs[nn][9], row-major i, j) and its
 * length scale L[nn] at every node from the nodal fields. */
int  orc_wp_rhs(const orc_ctx *c, double *rhs, double *L);
/* Eq. 12 solved by Galerkin FEM and Jacobi-PCG with the conditions of Eq. 59 and Sect. 4.1;
 * wp[nn][9]: initial guess in, solution out. */
int  orc_wp_solve(const orc_ctx *c, const double *rhs, const double *L, double *wp, double tol,
                  int max_iter, int *iters);
/* orc_wp_rhs, then orc_wp_solve from the fields' wp_ij (slots 14-22), written back there. */
int  orc_update_wp(orc_ctx *c, double tol, int max_iter, int *iters);
/* Eq. 33's nodal right-hand side src[nn] from the nodal means ustar[nn][3] and the nodal
 * pressure P[nn] (rho = 1), and the increment's normal derivative flux[nn] at no-slip nodes
 * from Eq. 61. */
int  orc_pressure_rhs(const orc_ctx *c, const double *ustar, const double *P, double dt, double Cp,
                      double *src, double *flux);
/* Eq. 33 by Galerkin FEM and Jacobi-PCG; dP[nn]: initial guess in, zero-mean solution out. */
int  orc_pressure_solve(const orc_ctx *c, const double *src, const double *flux, double *dP,
                        double tol, int max_iter, int *iters);
/* y = M x (which = 0, consistent mass matrix) or K x (which = 1, laplacian stiffness). */
void orc_fem_apply(const orc_ctx *c, int which, const double *x, double *y);
/* y = (M + K_L) x, Eq. 12's Galerkin operator with the nodal length scale L[nn]. */
void orc_wp_apply(const orc_ctx *c, const double *L, const double *x, double *y);
/* One step of the coupled loop in Table 1's order (see pdfx_oracle.c). */
int  orc_coupled_step(orc_ctx *c, double dt, double Cp, double *P, double *dP, double tol,
                      int max_iter, int *wp_iters, int *p_iters);
int  orc_advance(orc_ctx *c, double dt);      /* Eqs. 7, 27, 19, 24, Sect. 3.8, 3.6 */
int  orc_redistribute(orc_ctx *c);            /* Sect. 3.7, Appendix B */
int  orc_statistics(orc_ctx *c);              /* Sect. 3.3 and 3.5, Appendix A */
void orc_finish_step(orc_ctx *c);             /* step counter + 1 */

/* Outputs. */
int  orc_get_element_stats(const orc_ctx *c, double *out /* [ne][13] */, int32_t *counts);
int  orc_get_nodal_stats(const orc_ctx *c, double *out /* [nn][13] */);
int  orc_get_bins(const orc_ctx *c, double *vcce /* [ne][G] */, int32_t *g /* [ne][3] */);
int  orc_bins_capacity(const orc_ctx *c);

/* Scalar statistics of probe elements (Sect. 4.1.2, Eqs. 67-69): see pdfx_oracle.c. */
int  orc_scalar_stats(const orc_ctx *c, int n, const int32_t *elems, int nb, int32_t *count,
                      double *phit, double *cdiff, double *cdiss, double *mom);
void orc_get_diag(const orc_ctx *c, orc_diag *d);
void orc_reset_diag(orc_ctx *c);
int  orc_redistribution_counts(const int32_t *counts, int ne, int minnpel, int32_t *final_counts);

#ifdef __cplusplus
}
#endif
#endif
