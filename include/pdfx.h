/*
 * pdfx -- one timestep of the particle path of the non-hybrid PDF method for turbulent
 * flows on unstructured triangle grids (Bakosi, Franzese & Boybeyi), on one GB300 GPU.
 *
 * One call of pdfx_step advances every Lagrangian particle by one explicit Euler-Maruyama
 * step (Sect. 3.1): it interpolates the nodal Eulerian fields with linear shapefunctions
 * (Eqs. 37-38), updates position (Eq. 7), velocity (Eq. 27, the generalised Langevin
 * model with the elliptic-relaxation closure of Eq. 11), turbulent frequency (Eqs. 18-20)
 * and passive scalar (IECM, Eqs. 24-25), applies the wall conditions (Eqs. 53-58) and the
 * scalar source (Sect. 4.1.2), tracks the particle to its new element (Sect. 3.6),
 * redistributes particles to keep every element above a minimum count (Sect. 3.7,
 * Appendix B), and recomputes the element and nodal statistics (Sect. 3.3, Eqs. 34-36)
 * and the velocity-conditioned scalar means used by the next step (Sect. 3.5, Appendix A,
 * or Fox's projection, Eqs. 64-66).  Also: batches of independent grids stepped together,
 * the simplified model of the particle-redistribution test (Eqs. 46-47), scalar
 * post-processing of probe elements (Eqs. 67-69), and the Eulerian solves of the coupled
 * loop (elliptic relaxation, Eqs. 12-18 and 59; pressure projection, Eqs. 33 and 61; one
 * coupled step in the order of Table 1).
 *
 * Conventions for every call:
 *  - Return value: PDFX_OK (0) or a negative PDFX_ERR_* code.  No exception crosses this
 *    boundary.  pdfx_strerror() names a code.
 *  - Device work is enqueued on the caller's CUDA stream (a cudaStream_t passed as void*,
 *    NULL = the legacy default stream) and is asynchronous unless a call says otherwise.
 *    The statistics of a step fork onto two streams of the context's own and join back
 *    (events), so that the caller's stream sees every call's work in order, and a stream
 *    capture of a call records the branches as parallel nodes.
 *    Problems found on the device (a particle found in no element, an element above the
 *    per-element capacity, a non-finite state) set a device error word; it is read by
 *    pdfx_get_diag() and pdfx_check(), which synchronise the stream.
 *  - Pointers marked "host" are read or written before the call returns.  Pointers marked
 *    "device" must stay valid until the stream has executed the call.  The caller owns
 *    every buffer it passes; the library copies what it keeps.
 *  - Device memory of a context comes from the allocator given to pdfx_create (or
 *    cudaMalloc when none is given) and is released by pdfx_destroy.
 *  - A context is used by one host thread at a time.
 */
#ifndef PDFX_H
#define PDFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDFX_OK                 0
#define PDFX_ERR_ARG           -1   /* invalid argument or parameter */
#define PDFX_ERR_MESH          -2   /* invalid grid: bad index, non-positive area, open edge */
#define PDFX_ERR_ORDER         -3   /* call made before the state it needs exists */
#define PDFX_ERR_CUDA          -4   /* a CUDA runtime call failed */
#define PDFX_ERR_ALLOC         -5   /* device allocation failed */
#define PDFX_ERR_LOST_PARTICLE -6   /* a particle was found in no element (device word) */
#define PDFX_ERR_CAPACITY      -7   /* an element exceeded PDFX_MAX_PER_ELEMENT (device word) */
#define PDFX_ERR_NONFINITE     -8   /* a particle state became NaN or infinite (device word) */
#define PDFX_ERR_SOLVE         -9   /* an iterative solve did not converge within its limit */
#define PDFX_ERR_ELEMENT      -10   /* a particle's element id lies outside the grid (device word) */

#define PDFX_NF 32                  /* nodal field slots, layout below */
#define PDFX_NSTAT 13               /* statistics per element or node, layout below */
#define PDFX_MAX_PER_ELEMENT 4096   /* particles one element may hold for the binning */
#define PDFX_MAX_SCALAR_BINS 4096  /* psi bins of pdfx_scalar_stats */
#define PDFX_MAX_PARTICLES (1 << 28) /* particles per context (ids fit the binning sort keys) */

/*
 * Nodal field layout, [nn][32] FP64 (pdfx_set_fields):
 *   0-2   <U_i>                         3-4   d<P>/dx_j (rho = 1), j = x, y
 *   5-10  d<U_i>/dx_j, i-major, j = x, y
 *   11-13 laplacian of <U_i>            14-22 elliptic-relaxation tensor wp_ij, row-major
 *   23-28 <u_i u_j>: xx, yy, zz, xy, xz, yz
 *   29    <omega>                       30    omega_w, the Eq. 58 wall frequency mean
 *   31    unused
 * Statistics layout, [.][13] FP64: N, <U>, <V>, <W>, <uu>, <vv>, <ww>, <uv>, <uw>, <vw>,
 *   <omega>, <phi>, <phi'^2>.  For an element N is its particle count; for a node it is
 *   the mean count of the surrounding elements that hold particles.
 */

typedef struct pdfx_params {
    /* Table 4 of the paper */
    double C1, C2, C3, C4, CT, CL, Ceta, Cv, gamma5, Cw1, Cw2;
    double nu;                /* kinematic viscosity */
    int    c0_mode;           /* 0: C0 from Eq. 11; 1: the constant C0 below */
    double C0;
    int    tm_mode;           /* 0: t_m from Eq. 25; 1: t_m = 2k / (Cphi eps) */
    double Cs, Ct, Cphi;      /* Eq. 25 constants (Sect. 4.1.2: 0.02, 0.7) and IEM constant */
    double src_x, src_y, src_r; /* source disc: particles inside get psi = 1 */
    int    bins[3];           /* requested conditioning bins per velocity component, 1..16 */
    int    min_per_bin;       /* fewest particles a conditioning bin may hold (>= 1) */
    int    minnpel;           /* Appendix B threshold MINNPEL; 0 disables redistribution */
    int    interp_mode;       /* 0: shapefunctions at the particle; 1: element average */
    int    source_on;         /* 1: apply the source disc */
    uint64_t seed;            /* Philox key = (seed low word, seed high word ^ instance) */
    uint32_t instance;
    double period_x;          /* period of the x direction; 0 = not periodic */
    /* GPU form, fixed at pdfx_create */
    int    precision;         /* 0: FP64 state and arithmetic; 1: FP32 state and SDE
                                 arithmetic with FP64 statistics and conditional means */
    int    sort_every;        /* re-order particles by element every this many steps */
    int    acc64;             /* FP32 form: 1 accumulates element moments and conditional
                                 means in FP64, 0 (default) in compensated FP32 */
    int    cond_mode;         /* velocity conditioning of the scalar mean: 0 hierarchical
                                 bins (Sect. 3.5, Appendix A); 1 Fox's projection (Eqs.
                                 64-66) onto fox_bins intervals of the projected velocity */
    int    fox_bins;          /* 1..256 (cond_mode 1) */
    int    model;             /* particle model: 0 the full model (Eqs. 7, 19, 24, 27, walls
                                 of Sect. 3.8); 1 the simplified model of Eqs. 46-47 used to
                                 measure the particle-redistribution error (Sect. 3.7): the
                                 velocity relaxes to alpha times the particles' own nodal
                                 mean velocity of the previous statistics pass, the position
                                 moves with the velocity, omega and psi are kept; the grid may
                                 have free-slip boundaries but no no-slip walls */
    double alpha;             /* Eq. 47 (model 1), finite */
    double cfl;               /* Eq. 26 CFL constant (default 0.7), > 0: a step with dt <= 0
                                 takes dt = cfl min_n sqrt(A_n) / max_n ||<Z>_n||_2 */
} pdfx_params;

typedef struct pdfx_allocator {
    void *(*alloc)(size_t bytes, void *user);            /* returns device memory or NULL */
    void  (*release)(void *ptr, size_t bytes, void *user);
    void  *user;
} pdfx_allocator;

/* Particle state by particle id, FP64 values (converted for the FP32 form). */
typedef struct pdfx_soa {
    double  *x, *y, *u, *v, *w, *om, *psi;   /* [np] */
    int32_t *elem;                            /* [np] host element */
    uint8_t *cp;                              /* [np] conditioning pointer (get only) */
} pdfx_soa;

typedef struct pdfx_diag {
    int64_t steps;
    int64_t hops_total, walk_fallback, walk_brute, lost;
    int64_t wall_hits, freeslip_hits, omega_reflect, c0_clamp, gamma_exhausted;
    int64_t moves, source_hits, capacity_overflow, nonfinite;
    int64_t hop_hist[8];      /* particles that needed 0, 1, ..., 6, 7+ hops */
    int32_t error;            /* first device error code seen (PDFX_ERR_*), 0 if none */
    int32_t lost_records;     /* entries of lost[] in use */
    double  lost_xy[4][4];    /* first lost particles: x, y, old element, particle id */
    int64_t bad_element;      /* particles whose element id, given in device memory, lay
                                 outside 0 .. ne - 1 (PDFX_ERR_ELEMENT) */
} pdfx_diag;

/* Defaults: Table 4 constants, Cs = 0.02, Ct = 0.7 (Sect. 4.1.2), C0 from Eq. 11,
 * t_m from Eq. 25, (4, 4, 4) bins with at least 2 particles, FP64 form, re-order every 8
 * steps.  Host: writes *p. */
void pdfx_default_params(pdfx_params *p);

/* Creates a context.  p: host, copied.  alloc: host, copied, may be NULL (cudaMalloc).
 * The current CUDA device is the context's device; the context also creates two
 * non-blocking streams and three events there for the statistics' parallel branches
 * (without them the branches run on the caller's stream).  PDFX_ERR_ARG for invalid params. */
int  pdfx_create(const pdfx_params *p, const pdfx_allocator *alloc, void **out_ctx);

/* Releases all device memory of the context (synchronises the device first). */
void pdfx_destroy(void *ctx);

/* Replaces the model parameters (everything except bins, precision, sort_every, acc64,
 * cond_mode and fox_bins, which are fixed at creation).  Host pointer.  PDFX_ERR_ARG if those differ, and for a batch of
 * more than one instance (its parameters come from pdfx_set_instances). */
int  pdfx_set_params(void *ctx, const pdfx_params *p);

/* Batches of independent instances (the paper has no counterpart: each instance is one run
 * of the method on its own grid, and a batch steps them all with one launch per stage).
 * Call before pdfx_set_grid.  n instances; p[n] their parameters (host, copied): each may
 * have its own constants, seed, instance number, source, period_x and MINNPEL, while
 * precision, sort_every, acc64, bins, min_per_bin, cond_mode and fox_bins must equal the
 * context's (else
 * PDFX_ERR_ARG).  elem_first[n + 1] (host): instance k owns the elements elem_first[k] ..
 * elem_first[k + 1] - 1 of the union grid that pdfx_set_grid receives next (elem_first[0]
 * = 0, increasing, elem_first[n] = its ne; the instances may share no edge and no node,
 * else pdfx_set_grid returns PDFX_ERR_MESH).  Fields are the union's nodal fields; particle
 * ids restart at 0 in every instance, and particle arrays are ordered by (instance, id).
 * Statistics are those of the union (element and node ranges of each instance).  With n =
 * 1 the context becomes a single instance with parameters p[0].  Discards the grid, fields
 * and particles.  Synchronous. */
int  pdfx_set_instances(void *ctx, int32_t n, const pdfx_params *p, const int32_t *elem_first);

/* Number of instances (1 for a single grid); writes elem_first[K + 1] and part_first[K + 1]
 * (first particle slot of each instance) where the pointers are not NULL. */
int  pdfx_instance_ranges(const void *ctx, int32_t *elem_first, int64_t *part_first);

/* Sets the Eulerian grid (Sect. 3.3, Fig. 1): nn nodes node_xy[nn][2] (FP64, host),
 * ne counter-clockwise triangles tri[ne][3] (int32 node ids, host) and edge tags
 * edge_tag[ne][3] (int8, host) for the edge opposite local vertex k: 0 interior,
 * 1 no-slip wall (Sect. 3.8), 2 free-slip boundary (Sect. 4.2).  With period_x > 0, x is
 * periodic and a triangle may span the seam (its vertices are taken as minimum images).
 * Builds element geometry (Eq. 40), neighbours across each edge and node-to-element lists
 * (Sect. 3.6).  Synchronous.  PDFX_ERR_MESH for a bad index, a non-positive area or an
 * edge that is neither shared nor tagged.  Discards particles. */
int  pdfx_set_grid(void *ctx, int32_t nn, const double *node_xy, int32_t ne,
                   const int32_t *tri, const int8_t *edge_tag);

/* Sets the nodal fields [nn][32] (layout above), FP64, host (on_device = 0) or device
 * (on_device = 1) memory, enqueued on stream.  PDFX_ERR_ORDER before pdfx_set_grid. */
int  pdfx_set_fields(void *ctx, const double *fields, int on_device, void *stream);

/* Sect. 3.7: ppe particles per element, uniform in the element; velocity Gaussian about
 * the local mean with variance 2k/3 per component; frequency gamma with the local mean
 * and variance C4 <omega>^2; psi = 1 inside the source, else 0.  Particle id =
 * element * ppe + k.  Then computes the statistics and conditional means.  Resets the
 * step counter to 0.  PDFX_ERR_ORDER without grid and fields; PDFX_ERR_ARG if ppe * ne
 * reaches PDFX_MAX_PARTICLES. */
int  pdfx_init_particles(void *ctx, int32_t ppe, void *stream);

/* As pdfx_init_particles with ppe[k] particles per element in instance k (host array of
 * K entries); instance k's ids are 0 .. ppe[k] ne_k - 1.  PDFX_ERR_ARG if an instance
 * reaches PDFX_MAX_PARTICLES or the batch reaches 2^31 - 1 particles. */
int  pdfx_init_particles_batch(void *ctx, const int32_t *ppe, void *stream);

/* Replaces the particle state by np particles with ids 0..np-1 (FP64 arrays of s, host
 * or device per on_device; cp is ignored) and sets the step counter.  In a batch, host
 * arrays only, ordered by instance (ids restart at 0 in each instance; PDFX_ERR_ARG
 * otherwise).  Computes the statistics and conditional means of that state.  Element ids
 * outside 0 .. ne - 1 are PDFX_ERR_ARG for host input; for device input the device checks
 * them: such a particle is placed in element 0 (the next step's walk relocates it), counted
 * (pdfx_diag.bad_element), and the device error word and the return value become
 * PDFX_ERR_ELEMENT.  Synchronous. */
int  pdfx_set_particles(void *ctx, int64_t np, const pdfx_soa *s, uint32_t step,
                        int on_device, void *stream);

/* Writes the particle state by particle id into the caller's arrays of s (any pointer may
 * be NULL to skip it), host or device memory.  Synchronous for host output. */
int  pdfx_get_particles(void *ctx, pdfx_soa *s, int on_device, void *stream);

/* Number of particles (0 before initialisation). */
int64_t pdfx_num_particles(const void *ctx);

/* Step counter (the Philox counter word of the next step). */
uint32_t pdfx_step_index(const void *ctx);

/* One timestep (Table 1 order restricted to the particle path): advance and track every
 * particle, particle-number control, statistics and conditional means.  Asynchronous on
 * stream for dt > 0.  dt <= 0 takes the step of Eq. 26 from the nodal means of the last
 * statistics pass: dt = cfl min_n sqrt(A_n) / max_n ||<Z>_n||_2, A_n the mean area of the
 * elements around node n and <Z>_n = (<U>, <V>, <W>, <omega>, <psi>) (the norm as the paper
 * prints it, omega and psi included); this reads one number back and synchronises the
 * stream, and is for a single instance (PDFX_ERR_ARG in a batch, or when every nodal mean
 * vector is zero).  PDFX_ERR_ORDER without particles and fields; PDFX_ERR_ARG for model 1
 * on a grid with no-slip walls (Eqs. 46-47 define none). */
int  pdfx_step(void *ctx, double dt, void *stream);

/* The time step of the last pdfx_step (host, 0 before the first step). */
int  pdfx_last_dt(const void *ctx, double *dt);

/* The nodal fields the particles' own statistics provide (the non-hybrid coupling of Sect.
 * 3.3-3.4), from the nodal statistics of the last statistics pass, written into the
 * context's fields: <U_i> (slots 0-2), d<U_i>/dx_j (slots 5-10) = the node transfer (mean
 * over the elements around a node) of Eq. 39's element gradients with Eq. 40's
 * shapefunction derivatives, the laplacian of <U_i> (slots 11-13) by the same procedure
 * applied to the first derivatives (Sect. 3.4's two passes), <u_i u_j> (slots 23-28) and
 * <omega> (slot 29).  The slots the Eulerian solves provide (mean-pressure gradient 3-4,
 * elliptic-relaxation tensor 14-22, wall frequency 30) keep the values of pdfx_set_fields.
 * Asynchronous on stream (a scratch block of 18 (ne + nn) doubles is allocated and freed).
 * PDFX_ERR_ORDER before fields and statistics exist. */
int  pdfx_derive_fields(void *ctx, void *stream);

/* The mean-velocity correction of Eq. 31 applied to the particles (rho = 1; the velocity
 * field is the particles'): U_i -= dt d(dP)/dx_i, with the gradient of the nodal pressure
 * change dP = <P>^{n+1} - <P>^n (host array [nn], from the caller's solution of Eq. 33)
 * constant over each particle's element (Eq. 39 with Eq. 40's derivatives); W is unchanged.
 * dt > 0.  Complete on return (a scratch block of nn + 2 ne doubles is allocated and
 * freed).  PDFX_ERR_ORDER before particles exist. */
int  pdfx_correct_velocity(void *ctx, const double *dp, double dt, void *stream);

/* The context's nodal fields [nn][32] in FP64 (host; the FP32 form's are widened). */
int  pdfx_get_fields(void *ctx, double *out, void *stream);

/* One timestep of each of n independent contexts (distinct, each with its own grid,
 * parameters and particles), in array order on one stream: the same work and results as n
 * calls of pdfx_step.  A set of instances stepped with one launch per stage is a single
 * context made by pdfx_set_instances.  Stops at the first failing context and returns its
 * code; PDFX_ERR_ARG for n < 1, a NULL or repeated context. */
int  pdfx_batch_step(void *const *ctxs, int32_t n, double dt, void *stream);

/* nsteps calls of pdfx_step with the same dt (dt <= 0: each step takes Eq. 26's step, and
 * no graph is used).  With use_graph != 0 the steps of whole
 * re-order cycles (2 sort_every steps, or 1 without re-ordering) are replayed from a CUDA
 * graph captured on the first such call (steps before the next cycle start and after the
 * last whole cycle run as plain launches); the results are those of plain steps.  The
 * graph is rebuilt after a change of dt, grid, instances, parameters or particle state.
 * Capture runs on a stream of the library's own; the graph is launched on stream. */
int  pdfx_step_many(void *ctx, double dt, int32_t nsteps, int use_graph, void *stream);

/* Picks the launch shapes that do not change any result: the advance kernel's block size
 * (128 or 256 threads) and the re-order period sort_every (4, 8 or 16 steps; results do
 * not depend on the slots' order), then, with those, the binning's size-class split (the
 * largest element, 0, 128, 192 or 256 particles, taken by the tile of 256; larger ones up
 * to 512 take the tile of 512; every tile gives the same order).  Each candidate runs one
 * re-order cycle of dt steps from a snapshot of the current state, which is restored
 * afterwards (particles, statistics, step counter and diagnostics as before the call).
 * Writes the block size and period to adv_block and sort_every where not NULL (all three
 * shapes: pdfx_get_launch_shapes).  Needs temporary device memory of one particle buffer
 * plus the statistics.  Synchronous on stream. */
int  pdfx_autotune(void *ctx, double dt, int32_t *adv_block, int32_t *sort_every, void *stream);

/* The launch shapes in use (host outputs, any may be NULL): the advance block size, the
 * re-order period and the binning's size-class split. */
int  pdfx_get_launch_shapes(const void *ctx, int32_t *adv_block, int32_t *sort_every, int32_t *tile_split);

/* Sets the launch shapes (a negative value keeps the current one): the advance block size
 * (128 or 256), the re-order period (0 = never) and the binning's size-class split (0 to
 * 256 particles).  None of them changes a result.  PDFX_ERR_ARG for any other value. */
int  pdfx_set_launch_shapes(void *ctx, int32_t adv_block, int32_t sort_every, int32_t tile_split);

/* Nodal statistics [nn][13] and element statistics [ne][13] with counts [ne] of the last
 * step (or initialisation), into host or device memory.  Synchronous for host output. */
int  pdfx_get_nodal_stats(void *ctx, double *out, int on_device, void *stream);
int  pdfx_get_element_stats(void *ctx, double *out, int32_t *counts, int on_device,
                            void *stream);

/* Conditional scalar means vcce[ne][G] (G = bins[0]*bins[1]*bins[2]; bins past the
 * element's effective count are 0) and effective bins g[ne][3] (Sect. 3.5, Appendix A). */
int  pdfx_get_bins(void *ctx, double *vcce, int32_t *g, int on_device, void *stream);
int  pdfx_bins_capacity(const void *ctx);

/* Scalar statistics of n probe elements (Sect. 4.1.2, Figs. 12-15; Eqs. 67-69), from the
 * current particles and the conditioning pointers and conditional means of the last
 * statistics pass.  elems[n]: distinct element ids (host array).  The scalar sample space
 * [0, 1] is cut into nb (1..PDFX_MAX_SCALAR_BINS) equal bins, dpsi = 1/nb; a particle's bin
 * is floor(psi nb) clamped to 0..nb-1.  Outputs, row-major per probe, any may be NULL:
 *   count[n][nb]  particles per bin (the empirical PDF is count / (N dpsi));
 *   phit[n][nb]   Eq. 68: the bin average of the particles' conditional means <phi|V>;
 *   cdiff[n][nb]  t_m <Gamma lap phi | psi>: the bin average of <phi|V> - psi (IECM, Eq.
 *                 24), per unit 1/t_m;
 *   cdiss[n][nb]  t_m <2 Gamma (grad phi)^2 | psi> by Eq. 67 at the bin centre on the
 *                 empirical PDF: -2 dpsi (S_<b + S_b / 2) / count_b, S the sums of
 *                 psi - <phi|V> over the bins below b and over b; per unit 1/t_m;
 *   mom[n][6]     <phi>, <phi'^2>, <phi'^3>, <phi'^4> (1/N central moments), min and max
 *                 of psi.
 * Empty bins and elements give zeros.  The sums are fixed point (2^-46 and, for the
 * moments, 2^-40 resolution per term), so results do not depend on the order the GPU meets
 * the particles; they assume psi within [-1, 2].  Host outputs (on_device 0) are complete
 * on return; device outputs are ready on stream.  PDFX_ERR_ARG for a bad or repeated
 * element id or nb; PDFX_ERR_ORDER before particles exist. */
int  pdfx_scalar_stats(void *ctx, int32_t n, const int32_t *elems, int32_t nb, int32_t *count,
                       double *phit, double *cdiff, double *cdiss, double *mom, int on_device,
                       void *stream);

/* Diagnostic counters accumulated since creation or the last reset, and the device error
 * word.  Synchronises stream.  pdfx_check returns the device error word as a code. */
int  pdfx_get_diag(void *ctx, pdfx_diag *d, void *stream);
int  pdfx_reset_diag(void *ctx, void *stream);
int  pdfx_check(void *ctx, void *stream);

/* Per-stage GPU time.  When enabled, each stage of pdfx_step is bracketed by CUDA events
 * on the step's stream; pdfx_stage_times synchronises and writes, for stage i < n,
 * ms[i] = accumulated milliseconds and launches[i] = number of timed launches, then
 * clears them.  Stages: 0 advance, 1 plan, 2 lists, 3 redistribution, 4 statistics and
 * binning, 5 nodal average.  Returns the number of stages. */
int  pdfx_set_profiling(void *ctx, int on);
int  pdfx_stage_times(void *ctx, double *ms, int64_t *launches, int n, void *stream);

/* Element statistics, conditional means and nodal statistics of a caller's particle
 * state, computed without allocating device memory.  The paper has no counterpart: this
 * is a service for callers that cannot allocate while they run (an application whose own
 * pool owns all device memory, a service that must keep its footprint fixed, a loop that
 * cannot take the device-wide synchronisation cudaMalloc may cause).
 *   ctx: a context with a grid (its bins, min_per_bin and node lists are used).
 *   np particles indexed by particle id; u, v, w, om, psi [np] FP64 and elem [np] int32,
 *   device memory, read only.  np <= PDFX_NOALLOC_MAX_PARTICLES and the grid's element
 *   count <= PDFX_NOALLOC_MAX_ELEMENTS, else PDFX_ERR_ARG.
 *   Outputs, device memory written on stream: emom [ne][13], vcce [ne][G], gbin [ne][3],
 *   cp [np] (conditioning pointers), nmom [nn][13] (may be NULL to skip).
 * The results equal those the context computes for the same state (pdfx_set_particles
 * followed by pdfx_get_element_stats / pdfx_get_bins / pdfx_get_nodal_stats), in FP64,
 * with the context's conditioning (hierarchical bins or Fox's projection).  A particle whose
 * element id lies outside 0 .. ne - 1 is left out of every element (its cp is not written),
 * counted (pdfx_diag.bad_element) and sets the context's device error word to
 * PDFX_ERR_ELEMENT (read by pdfx_check).
 * Scratch is one fixed device array of the library (about 10 MB) that every GPU loading
 * the library reserves until exit; the first call on a device looks up its address with
 * cudaGetSymbolAddress, so make that first call before any stream capture.  Every call
 * reuses the same array: calls that overlap on the GPU (other streams, other host
 * threads, other contexts) race and must be serialised by the caller.  Asynchronous. */
#define PDFX_NOALLOC_MAX_PARTICLES (1 << 20)
#define PDFX_NOALLOC_MAX_ELEMENTS (1 << 16)
int  pdfx_element_stats_noalloc(void *ctx, int64_t np, const double *u, const double *v,
                                const double *w, const double *om, const double *psi,
                                const int32_t *elem, double *emom, double *vcce, int32_t *gbin,
                                uint8_t *cp, double *nmom, void *stream);

/* ---------------------------------------------------------------------------------------
 * Eulerian solves of the coupled loop (Sect. 3.2), FP64 on the device for both forms.
 * Single grids only (PDFX_ERR_ARG for a batch).  The first of these calls after
 * pdfx_set_grid builds the grid's Galerkin matrices for linear triangles in CSR: the
 * consistent mass matrix and the laplacian stiffness, from Eq. 40's derivatives.  It also
 * classifies the nodes: a node on a no-slip edge (tag 1), with its outward unit normal
 * (the normalised sum of its wall edges' normals), else a node on a free-slip edge (tag
 * 2), else interior; a node that belongs to no element gives PDFX_ERR_MESH.  The linear
 * systems are solved by conjugate gradients with the
 * Jacobi preconditioner, started from the given initial guess.  Each system iterates
 * until the 2-norm of its preconditioned residual over the free nodes is at most tol
 * times that of its preconditioned reduced load (the load minus the Dirichlet columns;
 * a zero reduced load gives the zero solution on the free nodes).  More than max_iter
 * iterations is PDFX_ERR_SOLVE.  *iters (may be NULL) receives the largest iteration
 * count.  Host arrays; every call returns after its results are on the host (or in the
 * context).
 * ------------------------------------------------------------------------------------- */

/* Eqs. 12-18 at every node from the context's nodal fields: the local right-hand side
 *     rhs_ij = (1 - C1)/2 k <omega> delta_ij + k H_ijkl d<U_k>/dx_l
 * (H of Eq. 13, A_v of Eq. 14, b of Eq. 15; d/dz = 0) into rhs[nn][9] (row-major i, j), and
 * the length scale L of Eq. 16 (C_xi of Eq. 17 = 2.3 when the grid has a no-slip edge,
 * else 1; eps of Eq. 18) into L[nn].  Inputs: d<U_i>/dx_j (slots 5-10), <u_i u_j>
 * (23-28), <omega> (29).  A node with eps <= 0 gives PDFX_ERR_ARG. */
int  pdfx_wp_rhs(void *ctx, double *rhs, double *L, void *stream);

/* Eq. 12, wp - div(L_e^2 grad wp) = rhs, by Galerkin FEM.  The nine components share the
 * matrix M + L_e^2 K, where L_e^2 is the mean of the element's nodal L^2; the load is M rhs.
 * Conditions: wp_ij = -4.5 eps n_i n_j at no-slip nodes (Eq. 59, eps from the node's
 * fields); at free-slip nodes wp_ij = 0 for i != j and the natural condition for i == j
 * (the symmetry conditions of Sect. 4.1).  rhs[nn][9], L[nn]; wp[nn][9] holds the initial
 * guess on entry and the solution on exit. */
int  pdfx_wp_solve(void *ctx, const double *rhs, const double *L, double *wp, double tol,
                   int32_t max_iter, int32_t *iters, void *stream);

/* The elliptic-relaxation update of the coupled loop: pdfx_wp_rhs and pdfx_wp_solve on the
 * context's own fields, from their wp_ij (slots 14-22) as the initial guess, the solution
 * written back to slots 14-22. */
int  pdfx_update_wp(void *ctx, double tol, int32_t max_iter, int32_t *iters, void *stream);

/* Eq. 33's nodal source with rho = 1, src = (div <U>* - Cp lap P) / dt, into src[nn]:
 * div <U>* from the node-transferred gradients (Sect. 3.4) of ustar[nn][3] (the nodal
 * means of the predicted velocities), and lap P by Sect. 3.4's two passes applied to
 * P[nn].  Also, into flux[nn], the outward normal derivative of the pressure increment at
 * no-slip nodes (0 elsewhere).  That is Eq. 61's value from the fields, nu lap<U_i> n_i
 * (slots 11-12) - d<u_i u_j>/dx_j n_i (node-transferred gradients of slots 23, 24, 26),
 * minus n . grad P.  dt > 0. */
int  pdfx_pressure_rhs(void *ctx, const double *ustar, const double *P, double dt, double Cp,
                       double *src, double *flux, void *stream);

/* Eq. 33 by Galerkin FEM: the laplacian stiffness K against the load -M src plus the edge
 * integrals of flux along no-slip edges (flux linear along the edge).  The matrix is
 * singular (periodic and natural boundaries), so the load's nodal mean is removed, and the
 * solution is shifted to zero integral over the domain.  src[nn], flux[nn]; dP[nn] holds
 * the initial guess on entry and the solution on exit. */
int  pdfx_pressure_solve(void *ctx, const double *src, const double *flux, double *dP, double tol,
                         int32_t max_iter, int32_t *iters, void *stream);

/* The context's nodal mean pressure P[nn] (rho = 1; zero after the FEM data is built) and
 * the last pressure increment dP[nn] (the next step's initial guess; set_pressure clears
 * it).  get_pressure writes whichever pointer is not NULL. */
int  pdfx_set_pressure(void *ctx, const double *P, void *stream);
int  pdfx_get_pressure(void *ctx, double *P, double *dP, void *stream);

/* One step of the coupled loop, in the order of Table 1:
 *   1. the time step (Eq. 26 when dt <= 0);
 *   2. the elliptic-relaxation update (pdfx_update_wp);
 *   3. the particle step of pdfx_step (velocity prediction of Eq. 27 with the other
 *      particle equations, walls, tracking, particle-number control, statistics);
 *   4. the pressure projection: pdfx_pressure_rhs with the predicted nodal means and the
 *      context's P, then pdfx_pressure_solve from the last increment;
 *   5. the correction of Eq. 31 and the statistics of the corrected state.  The correction
 *      is one vector per element (dt times its pressure-increment gradient), so the
 *      corrected statistics are the step's own with each element's mean U and V shifted
 *      by it (central moments, conditioning pointers and conditional means unchanged) and
 *      averaged at the nodes again.  The particles' velocities take the correction as the
 *      next advance (pdfx_step, pdfx_batch_step, pdfx_coupled_step) reads them, or before
 *      any other call that reads or replaces them (pdfx_get_particles,
 *      pdfx_correct_velocity, pdfx_step_many, pdfx_autotune);
 *   6. P += dP; the fields the statistics provide (pdfx_derive_fields) and the pressure
 *      gradient (slots 3-4: the node-transferred gradient of P) from the new state.
 * Eq. 33 is stable only for Cp < 2 dt.  iters[2] (may be NULL) receives the iteration
 * counts of the two solves. */
int  pdfx_coupled_step(void *ctx, double dt, double Cp, double tol, int32_t max_iter,
                       int32_t *iters, void *stream);

/* A measurement helper with no counterpart in the paper: the FP64 fused multiply-add rate
 * of the current device, 2 FLOP per FMA, from a kernel of independent FMA chains (no memory
 * traffic; 8 blocks of 256 threads per SM) timed with CUDA events on stream after one
 * warm-up launch.  The FP64 form's advance is bound by this rate.  Writes *flops_per_s
 * (host); synchronises stream.  PDFX_ERR_ARG for a NULL pointer. */
int  pdfx_measure_fp64_rate(double *flops_per_s, void *stream);

/* Number of kernel launches the library issued since creation. */
int64_t pdfx_kernel_launches(const void *ctx);

const char *pdfx_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
