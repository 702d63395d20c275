/*
 * CPU oracle for one timestep of the particle path of the non-hybrid PDF method.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain FP64 C, one thread, compiled with
 * -ffp-contract=off.  It is the definition the CUDA library is checked against and
 * it shares no code with that library.
 *
 * Paper passages followed (section / equation / appendix of the paper):
 *   Sect. 3.1          explicit forward Euler (Euler-Maruyama) in time
 *   Eq. 7              particle position
 *   Eq. 10 / Eq. 27    generalised Langevin velocity (prediction form)
 *   Eq. 11             G_ij and C0 from the elliptic-relaxation tensor
 *   Eq. 18             dissipation
 *   Eqs. 19-20         gamma (van Slooten) frequency model and its source
 *   Eqs. 24-25         IECM mixing and the micromixing time scale
 *   Eqs. 34-36         two-pass element/node statistics
 *   Eqs. 37-38, 40     linear triangle shapefunctions
 *   Eqs. 43-45         inside-element test and area coordinates (Fig. 1)
 *   Sect. 3.5, App. A  adaptive sort-and-divide binning, conditioning pointers
 *   Sect. 3.6          neighbour walk, concave-boundary fall-back (Fig. 2)
 *   Sect. 3.7, App. B  initial particles, particle redistribution
 *   Eqs. 53-58         wall crossing probability, reflection, no-slip, wall frequency
 *   Sect. 3.9          six Gaussians per particle per step, plus one uniform for Eq. 55
 *   Sect. 4.1.2        source disc with psi = 1
 *   Sect. 4.2          free-slip reflection (also beyond the start element, in the walk)
 *   Eq. 26             CFL time step for steps with dt <= 0
 *   Eq. 31             mean-velocity correction applied to the particles
 *   Eqs. 39-40         element gradients and their node transfer (Sect. 3.4)
 *   Eqs. 46-47         simplified model of the particle-redistribution test (Sect. 3.7)
 *   Eqs. 64-66         Fox's projection conditioning
 *   Eqs. 67-69         scalar statistics of probe elements (PDF, conditional diffusion and
 *                      dissipation, moments)
 *   Eqs. 12-18         local right-hand side and length scale of the elliptic relaxation
 *   Sect. 3.2, Eq. 59  Galerkin FEM and Jacobi-PCG solve of Eq. 12, its wall condition and
 *                      the symmetry conditions of Sect. 4.1 at free-slip boundaries
 *   Eqs. 30-33, 61     pressure projection by Galerkin FEM with the Neumann condition of Eq. 61
 *   Table 1            order of the coupled step (time step, elliptic relaxation, advance,
 *                      pressure projection, mean-velocity correction, statistics)
 *
 * Readings where the paper is silent, ambiguous or garbled are marked "Reading:".
 */
#include "pdfx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NF 32
#define NS 13
#define HOP_LIMIT 64
#define GAMMA_ATTEMPTS 32

/* Philox purposes (counter word 2). */
enum { PUR_STEP = 0, PUR_INIT = 1, PUR_WALL_GAMMA = 2, PUR_REDIST = 3, PUR_INIT_GAMMA = 4 };

struct orc_ctx {
    orc_params p;
    int nn, ne;
    double *node_xy;      /* [nn][2] */
    int32_t *tri;         /* [ne][3] */
    int8_t *tag;          /* [ne][3] */
    /* per element: vertices unwrapped across a periodic seam into vertex A's image
     * (vx, vy [ne][3]), edge vectors B - A and C - A, and twice the signed area */
    double *vx, *vy;
    double *ax, *ay, *bx, *by, *cx, *cy, *area2;
    int32_t *nbr;         /* [ne][3]: neighbour across the edge opposite vertex k, -1 outside */
    int32_t *ne_off, *ne_list;   /* node -> elements (ascending element id) */
    /* boundary lines: point, inward unit normal (in element frame) */
    int8_t *wall_type;    /* number of no-slip lines of the element (0, 1 or 2) */
    double *wall_px, *wall_py, *wall_nx, *wall_ny;   /* [ne][2] */
    int8_t *fs_type;      /* 0 none, 2 free-slip */
    double *fs_px, *fs_py, *fs_nx, *fs_ny;
    double *fields;       /* [nn][32] */
    /* particles, indexed by particle id */
    int np;
    double *x, *y, *u, *v, *w, *om, *psi;
    int32_t *elem;
    uint8_t *cp;
    uint32_t *pid;        /* particle ids (ascending), NULL: the index is the id */
    double *uphi;         /* [ne][3] element <u_a phi'> (Fox's projection, Eq. 66) */
    uint32_t step;
    double last_dt;       /* the time step of the last orc_step */
    /* statistics */
    int32_t *count;       /* [ne] */
    double *emom;         /* [ne][13] */
    double *nmom;         /* [nn][13] */
    int G;                /* bins capacity per element = b1 b2 b3 */
    double *vcce;         /* [ne][G] */
    int32_t *gbin;        /* [ne][3] */
    orc_diag diag;
};

/* ------------------------------------------------------------------------------------ */
/* Random numbers (Sect. 3.9).  Reading: counter-based Philox4x32-10 replaces the paper's
 * per-step tables; a particle's draws depend only on (seed, particle id, step, purpose,
 * block), so they are identical in any execution order.                                 */
/* ------------------------------------------------------------------------------------ */

/* Philox4x32-10 of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of two 32x32->64
 * multiplications with Weyl-sequence key increments between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on the open interval (0, 1): (w + 1/2) 2^-32. */
double orc_uniform(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* Box & Muller (1958): two independent standard Gaussians from two uniforms. */
void orc_box_muller(uint32_t w1, uint32_t w2, double *g1, double *g2)
{
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = orc_uniform(w1), u2 = orc_uniform(w2);
    double r = sqrt(-2.0 * log(u1));
    double th = two_pi * u2;
    *g1 = r * cos(th);
    *g2 = r * sin(th);
}

static void philox_draw(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t step,
                        uint32_t purpose, uint32_t block, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ instance};
    uint32_t ctr[4] = {pid, step, purpose, block};
    orc_philox4x32_10(ctr, key, out);
}

/* Gamma(shape, scale) by Marsaglia & Tsang (2000) for shape >= 1; attempt j uses Philox
 * block j.  Each attempt draws one Gaussian (Box-Muller of words 0-1, cosine branch) and
 * one uniform (word 2).  Reading: at most 32 attempts; if all are rejected the mean
 * shape*scale is returned and counted. */
double orc_gamma_draw(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t step,
                      uint32_t purpose, double shape, double scale, int *exhausted)
{
    double d = shape - 1.0 / 3.0;
    double c = 1.0 / sqrt(9.0 * d);
    *exhausted = 0;
    for (uint32_t j = 0; j < GAMMA_ATTEMPTS; ++j) {
        uint32_t r[4];
        double xg, dummy;
        philox_draw(seed, instance, pid, step, purpose, j, r);
        orc_box_muller(r[0], r[1], &xg, &dummy);
        double uu = orc_uniform(r[2]);
        double t = 1.0 + c * xg;
        if (t <= 0.0) continue;
        double vv = t * t * t;
        if (log(uu) < 0.5 * xg * xg + d - d * vv + d * log(vv)) return d * vv * scale;
    }
    *exhausted = 1;
    return shape * scale;
}

/* Sect. 3.9: the six Gaussians of one particle step and the uniform eta of Eq. 55.
 * Block 0 -> (xi1, xi2), (xi3, xi4); block 1 -> (xi5, xi6) and eta from word 2. */
/* The step's draws: six Gaussians, eta (word 2 of block 1) for the first wall line of the
 * element and eta2 (word 3) for a second one. */
static void step_draws(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t step,
                       double xi[6], double *eta, double *eta2)
{
    uint32_t r0[4], r1[4];
    philox_draw(seed, instance, pid, step, PUR_STEP, 0, r0);
    philox_draw(seed, instance, pid, step, PUR_STEP, 1, r1);
    orc_box_muller(r0[0], r0[1], &xi[0], &xi[1]);
    orc_box_muller(r0[2], r0[3], &xi[2], &xi[3]);
    orc_box_muller(r1[0], r1[1], &xi[4], &xi[5]);
    *eta = orc_uniform(r1[2]);
    *eta2 = orc_uniform(r1[3]);
}

void orc_step_gaussians(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t step,
                        double xi[6], double *eta)
{
    double eta2;
    step_draws(seed, instance, pid, step, xi, eta, &eta2);
}

/* ------------------------------------------------------------------------------------ */
/* Grid preprocessing.                                                                  */
/* ------------------------------------------------------------------------------------ */

/* Id of the particle at index p (the Philox counter word). */
static uint32_t pid_of(const orc_ctx *c, int p) { return c->pid ? c->pid[p] : (uint32_t)p; }

static double min_image(double d, double L)
{
    if (L <= 0.0) return d;
    if (d > 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
    return d;
}

static int elem_has_node(const orc_ctx *c, int e, int n)
{
    return c->tri[3 * e] == n || c->tri[3 * e + 1] == n || c->tri[3 * e + 2] == n;
}

/* Line of edge k of element f (the edge opposite its vertex k), with the unit normal
 * pointing toward vertex k, i.e. into the domain.  Returned in f's frame. */
static void edge_line(const orc_ctx *c, int f, int k, double *px, double *py, double *nx, double *ny)
{
    const double *vx = c->vx + 3 * f, *vy = c->vy + 3 * f;
    int a = (k + 1) % 3, b = (k + 2) % 3;
    double tx = vx[b] - vx[a], ty = vy[b] - vy[a];
    double len = sqrt(tx * tx + ty * ty);
    double mx = -ty / len, my = tx / len;
    if ((vx[k] - vx[a]) * mx + (vy[k] - vy[a]) * my < 0.0) { mx = -mx; my = -my; }
    *px = vx[a]; *py = vy[a]; *nx = mx; *ny = my;
}

/* Reading of Sect. 3.8 (last paragraph), extended to corners: an element's boundary lines
 * of a type are, in this order, its own edges of that type (local edge order), then the
 * edges of that type incident to one of its nodes (nodes in local order, elements in
 * ascending id, edges in local order) whose line, oriented into the fluid by the edge's
 * own element, has the element's centroid strictly in front; a line equal to one already
 * taken is skipped; at most max_lines lines.  Returns the number found; line j is written
 * to px[j], py[j] (in e's frame), nx[j], ny[j]. */
static int same_line(double px, double py, double nx, double ny,
                     double qx, double qy, double mx, double my)
{
    if (nx * mx + ny * my < 1.0 - 1e-9) return 0;
    double d = (qx - px) * nx + (qy - py) * ny;
    return fabs(d) <= 1e-9 * (1.0 + fabs(px) + fabs(py));
}

static int find_boundary_lines(orc_ctx *c, int e, int type, int max_lines,
                               double *px, double *py, double *nx, double *ny)
{
    int n_found = 0;
    for (int k = 0; k < 3 && n_found < max_lines; ++k) {
        if (c->tag[3 * e + k] != type) continue;
        double qx, qy, mx, my;
        edge_line(c, e, k, &qx, &qy, &mx, &my);
        int dup = 0;
        for (int j = 0; j < n_found; ++j)
            dup |= same_line(px[j], py[j], nx[j], ny[j], qx, qy, mx, my);
        if (dup) continue;
        px[n_found] = qx; py[n_found] = qy; nx[n_found] = mx; ny[n_found] = my;
        ++n_found;
    }
    /* centroid in e's frame (b, c are offsets from vertex A) */
    const double gx = c->ax[e] + (c->bx[e] + c->cx[e]) / 3.0;
    const double gy = c->ay[e] + (c->by[e] + c->cy[e]) / 3.0;
    for (int kv = 0; kv < 3 && n_found < max_lines; ++kv) {
        int n = c->tri[3 * e + kv];
        for (int i = c->ne_off[n]; i < c->ne_off[n + 1] && n_found < max_lines; ++i) {
            int f = c->ne_list[i];
            for (int k = 0; k < 3 && n_found < max_lines; ++k) {
                if (c->tag[3 * f + k] != type) continue;
                int a = c->tri[3 * f + (k + 1) % 3], b = c->tri[3 * f + (k + 2) % 3];
                if (a != n && b != n) continue;
                double qx, qy, mx, my;
                edge_line(c, f, k, &qx, &qy, &mx, &my);
                qx = c->ax[e] + min_image(qx - c->ax[e], c->p.period_x);   /* e's frame */
                if ((gx - qx) * mx + (gy - qy) * my <= 0.0) continue;       /* not in front */
                int dup = 0;
                for (int j = 0; j < n_found; ++j)
                    dup |= same_line(px[j], py[j], nx[j], ny[j], qx, qy, mx, my);
                if (dup) continue;
                px[n_found] = qx; py[n_found] = qy; nx[n_found] = mx; ny[n_found] = my;
                ++n_found;
            }
        }
    }
    return n_found;
}

static int params_valid(const orc_params *p)
{
    /* Marsaglia-Tsang needs shape 1/C4 >= 1; bins are 1..16 per component, <= 256 total */
    if (!(p->C4 > 0.0 && p->C4 <= 1.0)) return 0;
    for (int l = 0; l < 3; ++l)
        if (p->bins[l] < 1 || p->bins[l] > 16) return 0;
    if (p->bins[0] * p->bins[1] * p->bins[2] > 256 || p->min_per_bin < 1) return 0;
    if (p->cond_mode != 0 && p->cond_mode != 1) return 0;
    if (p->cond_mode == 1 && (p->fox_bins < 1 || p->fox_bins > 256)) return 0;
    if (p->model != 0 && p->model != 1) return 0;
    if (!isfinite(p->alpha)) return 0;
    if (!(p->cfl > 0.0) || !isfinite(p->cfl)) return 0;
    return 1;
}

int orc_create(orc_ctx **out, const orc_params *p, int nn, const double *node_xy,
               int ne, const int32_t *tri, const int8_t *edge_tag)
{
    *out = NULL;
    if (nn <= 0 || ne <= 0 || !params_valid(p)) return -1;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->p = *p;
    c->nn = nn;
    c->ne = ne;
    c->node_xy = (double *)malloc(sizeof(double) * 2 * nn);
    memcpy(c->node_xy, node_xy, sizeof(double) * 2 * nn);
    c->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * ne);
    memcpy(c->tri, tri, sizeof(int32_t) * 3 * ne);
    c->tag = (int8_t *)malloc(3 * ne);
    memcpy(c->tag, edge_tag, 3 * ne);
    double **geo[7] = {&c->ax, &c->ay, &c->bx, &c->by, &c->cx, &c->cy, &c->area2};
    for (int i = 0; i < 7; ++i) *geo[i] = (double *)malloc(sizeof(double) * ne);
    c->vx = (double *)malloc(sizeof(double) * 3 * ne);
    c->vy = (double *)malloc(sizeof(double) * 3 * ne);
    for (int e = 0; e < ne; ++e) {
        int A = tri[3 * e], B = tri[3 * e + 1], C = tri[3 * e + 2];
        if (A < 0 || B < 0 || C < 0 || A >= nn || B >= nn || C >= nn) { orc_destroy(c); return -2; }
        const int n3[3] = {A, B, C};
        for (int k = 0; k < 3; ++k) {
            double x = node_xy[2 * n3[k]];
            /* the image of the node nearest to vertex A (periodic in x) */
            if (p->period_x > 0.0 && k > 0) {
                double d = x - node_xy[2 * A];
                if (d > 0.5 * p->period_x) x -= p->period_x;
                else if (d < -0.5 * p->period_x) x += p->period_x;
            }
            c->vx[3 * e + k] = x;
            c->vy[3 * e + k] = node_xy[2 * n3[k] + 1];
        }
        c->ax[e] = node_xy[2 * A];
        c->ay[e] = node_xy[2 * A + 1];
        c->bx[e] = min_image(node_xy[2 * B] - node_xy[2 * A], p->period_x);
        c->by[e] = node_xy[2 * B + 1] - node_xy[2 * A + 1];
        c->cx[e] = min_image(node_xy[2 * C] - node_xy[2 * A], p->period_x);
        c->cy[e] = node_xy[2 * C + 1] - node_xy[2 * A + 1];
        /* 2 A_e: twice the signed area, positive for counter-clockwise vertices */
        c->area2[e] = c->bx[e] * c->cy[e] - c->by[e] * c->cx[e];
        if (!(c->area2[e] > 0.0)) { orc_destroy(c); return -3; }
    }
    /* node -> elements (Sect. 3.3 linked lists), ascending element id */
    c->ne_off = (int32_t *)calloc(nn + 1, sizeof(int32_t));
    for (int e = 0; e < ne; ++e)
        for (int k = 0; k < 3; ++k) c->ne_off[tri[3 * e + k] + 1]++;
    for (int n = 0; n < nn; ++n) c->ne_off[n + 1] += c->ne_off[n];
    c->ne_list = (int32_t *)malloc(sizeof(int32_t) * 3 * ne);
    int32_t *fill = (int32_t *)calloc(nn, sizeof(int32_t));
    for (int e = 0; e < ne; ++e)
        for (int k = 0; k < 3; ++k) {
            int n = tri[3 * e + k];
            c->ne_list[c->ne_off[n] + fill[n]++] = e;
        }
    free(fill);
    /* elements surrounding elements (Sect. 3.6): neighbour across edge k */
    c->nbr = (int32_t *)malloc(sizeof(int32_t) * 3 * ne);
    for (int e = 0; e < ne; ++e)
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * e + (k + 1) % 3], b = tri[3 * e + (k + 2) % 3];
            int found = -1;
            for (int i = c->ne_off[a]; i < c->ne_off[a + 1]; ++i) {
                int f = c->ne_list[i];
                if (f != e && elem_has_node(c, f, b)) { found = f; break; }
            }
            c->nbr[3 * e + k] = found;
            if ((found < 0) != (edge_tag[3 * e + k] != 0)) { orc_destroy(c); return -4; }
        }
    c->wall_type = (int8_t *)calloc(ne, 1);
    c->fs_type = (int8_t *)calloc(ne, 1);
    double **wl[4] = {&c->wall_px, &c->wall_py, &c->wall_nx, &c->wall_ny};
    for (int i = 0; i < 4; ++i) *wl[i] = (double *)calloc(2 * (size_t)ne, sizeof(double));
    double **fl[4] = {&c->fs_px, &c->fs_py, &c->fs_nx, &c->fs_ny};
    for (int i = 0; i < 4; ++i) *fl[i] = (double *)calloc(ne, sizeof(double));
    for (int e = 0; e < ne; ++e) {
        c->wall_type[e] = (int8_t)find_boundary_lines(c, e, 1, 2, c->wall_px + 2 * e,
                                                       c->wall_py + 2 * e, c->wall_nx + 2 * e,
                                                       c->wall_ny + 2 * e);
        c->fs_type[e] = (int8_t)(2 * find_boundary_lines(c, e, 2, 1, c->fs_px + e, c->fs_py + e,
                                                          c->fs_nx + e, c->fs_ny + e));
    }
    c->fields = (double *)calloc((size_t)nn * NF, sizeof(double));
    c->count = (int32_t *)calloc(ne, sizeof(int32_t));
    c->emom = (double *)calloc((size_t)ne * NS, sizeof(double));
    c->uphi = (double *)calloc((size_t)ne * 3, sizeof(double));
    c->nmom = (double *)calloc((size_t)nn * NS, sizeof(double));
    c->G = p->cond_mode == 1 ? p->fox_bins : p->bins[0] * p->bins[1] * p->bins[2];
    if (c->G < 1 || c->G > 256) { orc_destroy(c); return -5; }
    c->vcce = (double *)calloc((size_t)ne * c->G, sizeof(double));
    c->gbin = (int32_t *)calloc((size_t)ne * 3, sizeof(int32_t));
    *out = c;
    return 0;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    void *ptrs[] = {c->node_xy, c->tri, c->tag, c->vx, c->vy, c->ax, c->ay, c->bx, c->by, c->cx, c->cy,
                    c->area2, c->nbr, c->ne_off, c->ne_list, c->wall_type, c->wall_px,
                    c->wall_py, c->wall_nx, c->wall_ny, c->fs_type, c->fs_px, c->fs_py,
                    c->fs_nx, c->fs_ny, c->fields, c->x, c->y, c->u, c->v, c->w, c->om,
                    c->psi, c->elem, c->cp, c->count, c->emom, c->nmom, c->vcce, c->gbin,
                    c->pid, c->uphi};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(c);
}

int orc_set_params(orc_ctx *c, const orc_params *p)
{
    if (!params_valid(p)) return -1;
    if (p->bins[0] * p->bins[1] * p->bins[2] != c->G) return -5;
    c->p = *p;
    return 0;
}

int orc_set_fields(orc_ctx *c, const double *fields)
{
    memcpy(c->fields, fields, sizeof(double) * (size_t)c->nn * NF);
    return 0;
}

int orc_neighbors(const orc_ctx *c, int32_t *nbr)
{
    memcpy(nbr, c->nbr, sizeof(int32_t) * 3 * (size_t)c->ne);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Area coordinates and interpolation (Eqs. 37-38, 43-45).                              */
/* ------------------------------------------------------------------------------------ */

/* Eqs. 44-45 and Fig. 1: the area coordinate of a vertex is half the signed cross product
 * of the edge opposite that vertex with the vector from one end of that edge to the
 * particle, over A_e (N^A from (r_C - r_B) x (r_P - r_B), Eq. 44; N^C from
 * (r_P - r_B) x (r_A - r_B), Eq. 45; N^B likewise).  Readings: the paper prints |.| but
 * calls the values signed, so the signed z-component is used (counter-clockwise
 * vertices); every N^k is formed by the same construction (N^B is not taken as
 * A_e - N^A - N^C, the same number in exact arithmetic); and each edge is pivoted at its
 * lower-numbered node, with node x taken as the minimum image, so the two elements
 * sharing an edge evaluate it with the same rounding and opposite signs: every point of
 * the domain lies in at least one element (Eq. 43 closed).  area_cross returns 2 N^k. */
static double edge_cross(const orc_ctx *c, int a, int b, double x, double y)
{
    const double *xy = c->node_xy;
    double sign = 1.0;
    if (a > b) { int t = a; a = b; b = t; sign = -1.0; }
    double ex = min_image(xy[2 * b] - xy[2 * a], c->p.period_x), ey = xy[2 * b + 1] - xy[2 * a + 1];
    double px = min_image(x - xy[2 * a], c->p.period_x), py = y - xy[2 * a + 1];
    return sign * (ex * py - ey * px);
}

static void area_cross(const orc_ctx *c, int e, double x, double y, double N2[3])
{
    const int32_t *t = c->tri + 3 * e;
    for (int k = 0; k < 3; ++k) N2[k] = edge_cross(c, t[(k + 1) % 3], t[(k + 2) % 3], x, y);
}

void orc_lambda(const orc_ctx *c, int e, double x, double y, double lam[3])
{
    double N2[3];
    area_cross(c, e, x, y, N2);
    for (int k = 0; k < 3; ++k) lam[k] = N2[k] / c->area2[e];
}

/* Eq. 43 as a closed test on the signed areas (Reading: the strict inequalities would
 * leave edge points in no element). */
static int lambda_inside(const double lam[3])
{
    return lam[0] >= 0.0 && lam[1] >= 0.0 && lam[2] >= 0.0;
}

/* Eq. 37: q(x) = sum_j N^j(x) q_j over the three nodes of the element. */
void orc_interp(const orc_ctx *c, int e, const double lam[3], double q[32])
{
    const double *fa = c->fields + (size_t)NF * c->tri[3 * e];
    const double *fb = c->fields + (size_t)NF * c->tri[3 * e + 1];
    const double *fc = c->fields + (size_t)NF * c->tri[3 * e + 2];
    for (int f = 0; f < NF; ++f) q[f] = lam[0] * fa[f] + lam[1] * fb[f] + lam[2] * fc[f];
}

/* ------------------------------------------------------------------------------------ */
/* Particle tracking (Sect. 3.6).                                                       */
/* ------------------------------------------------------------------------------------ */

int orc_brute_locate(const orc_ctx *c, double x, double y)
{
    double N2[3];
    for (int e = 0; e < c->ne; ++e) {
        area_cross(c, e, x, y, N2);
        if (lambda_inside(N2)) return e;
    }
    return -1;
}

/* Neighbour-to-neighbour walk: if the particle is outside the element, continue in the
 * neighbour opposite the vertex with the lowest area coordinate.  Reading: equal minima
 * go to the lowest local vertex; after 64 hops, or when the next guess is outside the
 * domain (a tagged boundary edge, Fig. 2), search the elements surrounding the nodes of
 * the old host element in ascending id; if that fails, search all elements (counted as
 * an error).  Returns -1 if the point lies in no element. */
int orc_walk(orc_ctx *c, int e0, double x, double y, int *hops)
{
    double lam[3];   /* 2 N^k: same signs and order as the area coordinates */
    int e = e0;
    *hops = 0;
    for (;;) {
        area_cross(c, e, x, y, lam);
        if (lambda_inside(lam)) return e;
        if (*hops >= HOP_LIMIT) break;
        int k = 0;
        if (lam[1] < lam[k]) k = 1;
        if (lam[2] < lam[k]) k = 2;
        int nb = c->nbr[3 * e + k];
        if (nb < 0) break;
        e = nb;
        (*hops)++;
    }
    c->diag.walk_fallback++;
    int best = -1;
    for (int kv = 0; kv < 3; ++kv) {
        int n = c->tri[3 * e0 + kv];
        for (int i = c->ne_off[n]; i < c->ne_off[n + 1]; ++i) {
            int f = c->ne_list[i];
            if (best >= 0 && f >= best) continue;
            area_cross(c, f, x, y, lam);
            if (lambda_inside(lam)) best = f;
        }
    }
    if (best >= 0) return best;
    c->diag.walk_brute++;
    return orc_brute_locate(c, x, y);
}

/* ------------------------------------------------------------------------------------ */
/* Particle advance (Sect. 3.1; Eqs. 7, 27, 19, 24; Sect. 3.8).                         */
/* ------------------------------------------------------------------------------------ */

static double wrap_x(double x, double L)
{
    if (L <= 0.0) return x;
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    return x;
}

/* Source disc of Sect. 4.1.2: particles inside get psi = phi_0 = 1. */
static int in_source(const orc_ctx *c, double x, double y)
{
    if (!c->p.source_on) return 0;
    double dx = min_image(x - c->p.src_x, c->p.period_x);
    double dy = y - c->p.src_y;
    return dx * dx + dy * dy <= c->p.src_r * c->p.src_r;
}

static void finish_particle(orc_ctx *c, int p, int e, double Xn, double Yn, double Un[3],
                            double wn, double psin);

static void advance_particle(orc_ctx *c, int p, double dt)
{
    const orc_params *P = &c->p;
    const int e = c->elem[p];
    double lam[3], q[NF];

    /* Eqs. 37-38 and 44-45 at X^n (Reading: interp_mode 1 is the element average the
     * paper uses, Sect. 3.3; mode 0 the shapefunction interpolation). */
    if (P->interp_mode == 1) {
        lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
    } else {
        orc_lambda(c, e, c->x[p], c->y[p], lam);
    }
    orc_interp(c, e, lam, q);

    const double Um[3] = {q[0], q[1], q[2]};
    const double dP[3] = {q[3], q[4], 0.0};
    double gradU[3][2];
    for (int i = 0; i < 3; ++i) { gradU[i][0] = q[5 + 2 * i]; gradU[i][1] = q[6 + 2 * i]; }
    const double lapU[3] = {q[11], q[12], q[13]};
    double wp[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) wp[i][j] = q[14 + 3 * i + j];
    double R[3][3];
    R[0][0] = q[23]; R[1][1] = q[24]; R[2][2] = q[25];
    R[0][1] = R[1][0] = q[26];
    R[0][2] = R[2][0] = q[27];
    R[1][2] = R[2][1] = q[28];
    const double Om = q[29];
    const double om_w = q[30];

    /* k = <u_i u_i>/2 and Eq. 18.  Reading: k and eps are floored at 1e-30 so that a
     * particle exactly on a wall (k = 0) keeps finite coefficients. */
    double k = 0.5 * (R[0][0] + R[1][1] + R[2][2]);
    if (k < 1e-30) k = 1e-30;
    double eps = Om * (k + P->nu * P->CT * P->CT * Om);
    if (eps < 1e-30) eps = 1e-30;

    /* Eq. 11 */
    double G[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G[i][j] = (wp[i][j] - (i == j ? 0.5 * eps : 0.0)) / k;
    double C0;
    if (P->c0_mode == 1) {
        C0 = P->C0;
    } else {
        double s = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s += wp[i][j] * R[i][j];
        C0 = -2.0 * s / (3.0 * k * eps);
    }
    /* Production P = -<u_i u_j> d<U_i>/dx_j (two space dimensions) and Eq. 20 */
    double prod = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 2; ++j) prod -= R[i][j] * gradU[i][j];
    double Somega = P->Cw2 - P->Cw1 * prod / eps;

    /* Eq. 25, or t_m = 2k / (C_phi eps).  Reading of Eq. 25: d_r = |X^n - x_s|,
     * U_c = |<U>(X^n)| over three components; U_c = 0 makes the first argument infinite. */
    double tm;
    if (P->tm_mode == 1) {
        tm = 2.0 * k / (P->Cphi * eps);
    } else {
        double ddx = min_image(c->x[p] - P->src_x, P->period_x);
        double ddy = c->y[p] - P->src_y;
        double dr = sqrt(ddx * ddx + ddy * ddy);
        double Uc = sqrt(Um[0] * Um[0] + Um[1] * Um[1] + Um[2] * Um[2]);
        double a1 = (Uc > 0.0) ? P->Cs * cbrt(P->src_r * P->src_r / eps) + P->Ct * dr / Uc
                               : INFINITY;
        double kt = k / eps, kol = P->CT * sqrt(P->nu / eps);
        double a2 = kt > kol ? kt : kol;
        tm = a1 < a2 ? a1 : a2;
    }

    /* Sect. 3.9 draws */
    double xi[6], eta, eta2;
    step_draws(P->seed, P->instance, pid_of(c, p), c->step, xi, &eta, &eta2);
    const double sdt = sqrt(dt);
    const double dWx = sdt * xi[0], dWy = sdt * xi[1];
    const double dWp[3] = {sdt * xi[2], sdt * xi[3], sdt * xi[4]};
    const double dWw = sdt * xi[5];
    const double s2nu = sqrt(2.0 * P->nu);

    const double U0[3] = {c->u[p], c->v[p], c->w[p]};
    const double X0 = c->x[p], Y0 = c->y[p];
    const double w0 = c->om[p], psi0 = c->psi[p];

    /* Eq. 27 (Reading: C0 eps < 0 is clamped to 0 under the square root, counted). */
    double c0e = C0 * eps;
    if (c0e < 0.0) { c0e = 0.0; c->diag.c0_clamp++; }
    const double sc0e = sqrt(c0e);
    double Un[3];
    for (int i = 0; i < 3; ++i) {
        double a = U0[i] - dP[i] * dt + 2.0 * P->nu * lapU[i] * dt
                   + s2nu * (gradU[i][0] * dWx + gradU[i][1] * dWy);
        double g = 0.0;
        for (int j = 0; j < 3; ++j) g += G[i][j] * (U0[j] - Um[j]);
        Un[i] = a + g * dt + sc0e * dWp[i];
    }
    /* Eq. 7 with the same dW as Eq. 27 */
    double Xn = X0 + U0[0] * dt + s2nu * dWx;
    double Yn = Y0 + U0[1] * dt + s2nu * dWy;
    /* Eq. 19 (Reading: max(omega, 0) under the square root, then |omega|) */
    double wpos = w0 > 0.0 ? w0 : 0.0;
    double wn = w0 - P->C3 * Om * (w0 - Om) * dt - Somega * Om * w0 * dt
                + sqrt(2.0 * P->C3 * P->C4 * Om * Om * wpos) * dWw;
    if (wn < 0.0) { wn = -wn; c->diag.omega_reflect++; }
    /* Eq. 24 with the conditional mean of the particle's bin (Appendix A pointer) */
    double phic = c->vcce[(size_t)e * c->G + c->cp[p]];
    double psin = psi0 - (psi0 - phic) * dt / tm;

    /* Sect. 3.8, Eqs. 53-58, only in elements touching a wall (Reading: distances to each of
     * the element's wall lines in turn, the second from the position after the first's
     * reflection, with its own uniform; reflect only when behind a line; a hit on either
     * sets U = 0 and draws omega once; psi is not changed). */
    int any_hit = 0;
    for (int j = 0; j < c->wall_type[e]; ++j) {
        const double nx = c->wall_nx[2 * e + j], ny = c->wall_ny[2 * e + j];
        const double lx = c->wall_px[2 * e + j], ly = c->wall_py[2 * e + j];
        double d0 = min_image(X0 - lx, P->period_x) * nx + (Y0 - ly) * ny;
        double d1 = min_image(Xn - lx, P->period_x) * nx + (Yn - ly) * ny;
        int hit = 0;
        if (d1 < 0.0) {
            hit = 1;
            c->diag.wall_hits_a++;
        } else {
            double dd0 = d0 > 0.0 ? d0 : 0.0;
            double fw = exp(-dd0 * d1 / (P->nu * dt));
            if ((j == 0 ? eta : eta2) < fw) hit = 1;
        }
        if (hit) {
            any_hit = 1;
            if (d1 < 0.0) { Xn -= 2.0 * d1 * nx; Yn -= 2.0 * d1 * ny; }
        }
    }
    if (any_hit) {
        c->diag.wall_hits++;
        Un[0] = Un[1] = Un[2] = 0.0;                             /* Eq. 56 */
        int ex = 0;
        double shape = 1.0 / P->C4;                               /* Eq. 58 */
        wn = orc_gamma_draw(P->seed, P->instance, pid_of(c, p), c->step, PUR_WALL_GAMMA,
                            shape, P->C4 * om_w, &ex);
        if (ex) c->diag.gamma_exhausted++;
    }
    finish_particle(c, p, e, Xn, Yn, Un, wn, psin);
}

/* Free-slip reflection (Sect. 4.2): a point behind the boundary line (point px, py, inward
 * unit normal nx, ny) is mirrored across it and the normal velocity reversed; returns 1 if
 * it was behind. */
static int reflect_free_slip(double px, double py, double nx, double ny, double L, double *x,
                             double *y, double U[3])
{
    const double d = min_image(*x - px, L) * nx + (*y - py) * ny;
    if (!(d < 0.0)) return 0;
    *x -= 2.0 * d * nx;
    *y -= 2.0 * d * ny;
    const double un = U[0] * nx + U[1] * ny;
    U[0] -= 2.0 * un * nx;
    U[1] -= 2.0 * un * ny;
    return 1;
}

/* The walk of a particle update (Sect. 3.6 as orc_walk).  Reading: when the edge the walk
 * would cross is a free-slip boundary edge, the particle has passed the boundary beyond its
 * start element; it is reflected across that edge's own line (Sect. 4.2) and the walk goes
 * on from the same element, each reflection counting as a hop.  At any other boundary edge,
 * after HOP_LIMIT hops, or when the point is not strictly behind the free-slip line, the
 * fall-back and brute force of orc_walk follow. */
static int walk_particle(orc_ctx *c, int e0, double *x, double *y, double U[3], int *hops,
                         int *refl)
{
    double lam[3];
    int e = e0;
    *hops = 0;
    for (;;) {
        area_cross(c, e, *x, *y, lam);
        if (lambda_inside(lam)) return e;
        if (*hops >= HOP_LIMIT) break;
        int k = 0;
        if (lam[1] < lam[k]) k = 1;
        if (lam[2] < lam[k]) k = 2;
        int nb = c->nbr[3 * e + k];
        if (nb < 0) {
            if (c->tag[3 * e + k] != 2) break;
            double px, py, nx, ny;
            edge_line(c, e, k, &px, &py, &nx, &ny);
            if (!reflect_free_slip(px, py, nx, ny, c->p.period_x, x, y, U)) break;
            *refl = 1;
            (*hops)++;
            continue;
        }
        e = nb;
        (*hops)++;
    }
    c->diag.walk_fallback++;
    int best = -1;
    for (int kv = 0; kv < 3; ++kv) {
        int n = c->tri[3 * e0 + kv];
        for (int i = c->ne_off[n]; i < c->ne_off[n + 1]; ++i) {
            int f = c->ne_list[i];
            if (best >= 0 && f >= best) continue;
            area_cross(c, f, *x, *y, lam);
            if (lambda_inside(lam)) best = f;
        }
    }
    if (best >= 0) return best;
    c->diag.walk_brute++;
    return orc_brute_locate(c, *x, *y);
}

/* The end of one particle update in either model: free-slip boundary of the start element
 * (Sect. 4.2: perfect reflection, normal velocity reversed), periodic wrap, neighbour walk
 * (Sect. 3.6, with the reflections of walk_particle), source disc, and the store of the new
 * state.  A particle reflected at all counts once as a free-slip hit. */
static void finish_particle(orc_ctx *c, int p, int e, double Xn, double Yn, double Un[3],
                            double wn, double psin)
{
    const orc_params *P = &c->p;
    int refl = 0;
    if (c->fs_type[e] == 2)
        refl = reflect_free_slip(c->fs_px[e], c->fs_py[e], c->fs_nx[e], c->fs_ny[e],
                                 P->period_x, &Xn, &Yn, Un);
    Xn = wrap_x(Xn, P->period_x);

    /* Sect. 3.6 */
    int hops, wrefl = 0;
    int en = walk_particle(c, e, &Xn, &Yn, Un, &hops, &wrefl);
    c->diag.hops_total += hops;
    c->diag.hop_hist[hops < 7 ? hops : 7]++;
    if (en < 0) { en = e; c->diag.lost++; }
    if (wrefl) Xn = wrap_x(Xn, P->period_x);
    if (refl || wrefl) c->diag.freeslip_hits++;
    if (in_source(c, Xn, Yn)) { psin = 1.0; c->diag.source_hits++; }

    c->x[p] = Xn; c->y[p] = Yn;
    c->u[p] = Un[0]; c->v[p] = Un[1]; c->w[p] = Un[2];
    c->om[p] = wn; c->psi[p] = psin;
    c->elem[p] = en;
}

/* Eqs. 46-47, the simplified model of the particle-redistribution test (Sect. 3.7):
 *   dX_i = U_i dt,   dU_i = -(U_i - alpha <U_i>) dt + sqrt(2) dW_i.
 * Reading: <U_i> is the particles' own mean velocity, the nodal means of the previous
 * statistics pass interpolated at X^n like every Eulerian statistic at a particle (Sect.
 * 3.3; interp_mode 1: element average); explicit Euler-Maruyama with both right-hand sides
 * at time n; dW_i = sqrt(dt) xi_i with xi_1..3 the first three Gaussians of the step's draws;
 * omega and psi are not changed; the domain has free-slip boundaries and no no-slip walls. */
static void advance_particle_simple(orc_ctx *c, int p, double dt)
{
    const orc_params *P = &c->p;
    const int e = c->elem[p];
    double lam[3];
    if (P->interp_mode == 1) {
        lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
    } else {
        orc_lambda(c, e, c->x[p], c->y[p], lam);
    }
    double Um[3];
    for (int i = 0; i < 3; ++i) {
        Um[i] = 0.0;
        for (int k = 0; k < 3; ++k) Um[i] += lam[k] * c->nmom[(size_t)NS * c->tri[3 * e + k] + 1 + i];
    }
    double xi[6], eta, eta2;
    step_draws(P->seed, P->instance, pid_of(c, p), c->step, xi, &eta, &eta2);
    const double U0[3] = {c->u[p], c->v[p], c->w[p]};
    double Un[3];
    for (int i = 0; i < 3; ++i)
        Un[i] = U0[i] - (U0[i] - P->alpha * Um[i]) * dt + sqrt(2.0 * dt) * xi[i];   /* Eq. 47 */
    const double Xn = c->x[p] + U0[0] * dt;                                         /* Eq. 46 */
    const double Yn = c->y[p] + U0[1] * dt;
    finish_particle(c, p, e, Xn, Yn, Un, c->om[p], c->psi[p]);
}

int orc_advance(orc_ctx *c, double dt)
{
    if (!c->x) return -1;
    if (c->p.model == 1) {
        for (int e = 0; e < c->ne; ++e)
            if (c->wall_type[e] > 0) return -2;      /* Eqs. 46-47 define no wall treatment */
        for (int p = 0; p < c->np; ++p) advance_particle_simple(c, p, dt);
        return 0;
    }
    for (int p = 0; p < c->np; ++p) advance_particle(c, p, dt);
    return 0;
}

void orc_finish_step(orc_ctx *c) { c->step++; }

/* ------------------------------------------------------------------------------------ */
/* Particle-number control (Sect. 3.7, Appendix B).                                     */
/* ------------------------------------------------------------------------------------ */

/* The Appendix B loop, literally: find the elements with the fewest and the most
 * particles; while min < MINNPEL and the two differ, move one particle from the max to
 * the min element.  Reading: ties go to the lowest element id; the loop also stops when
 * max - min <= 1, where a move only swaps the two counts and the printed loop would not
 * terminate. */
int orc_redistribution_counts(const int32_t *counts, int ne, int minnpel, int32_t *fc)
{
    memcpy(fc, counts, sizeof(int32_t) * (size_t)ne);
    int moves = 0;
    if (minnpel <= 0) return 0;
    for (;;) {
        int mine = 0, maxe = 0;
        for (int e = 1; e < ne; ++e) {
            if (fc[e] < fc[mine]) mine = e;
            if (fc[e] > fc[maxe]) maxe = e;
        }
        if (!(fc[mine] < minnpel && fc[maxe] - fc[mine] >= 2)) break;
        fc[mine]++;
        fc[maxe]--;
        moves++;
    }
    return moves;
}

/* Appendix B and its closing paragraph.  Reading of what the paper leaves open:
 *  - pairing: recipients in ascending element id, each repeated by its gain; donor slots
 *    in ascending donor id, each donor giving its highest particle ids first; the k-th
 *    recipient slot receives the k-th donor particle, which keeps its id;
 *  - the moved particle is placed uniformly in the recipient triangle (Philox purpose 3,
 *    words 0-1, square-root method) and copies (U, omega, psi) of the recipient's
 *    resident with rank floor(u * n) in ascending id among its residents before the move
 *    (word 2); an empty recipient copies from its lowest-id non-empty edge neighbour,
 *    and with none the particle keeps its own properties;
 *  - the source disc is re-applied at the new position. */
int orc_redistribute(orc_ctx *c)
{
    const int ne = c->ne;
    int32_t *cnt = (int32_t *)calloc(ne, sizeof(int32_t));
    for (int p = 0; p < c->np; ++p) cnt[c->elem[p]]++;
    int32_t *fin = (int32_t *)malloc(sizeof(int32_t) * ne);
    int T = orc_redistribution_counts(cnt, ne, c->p.minnpel, fin);
    if (T == 0) { free(cnt); free(fin); return 0; }

    /* residents of every element, ascending particle id */
    int32_t *off = (int32_t *)calloc(ne + 1, sizeof(int32_t));
    for (int e = 0; e < ne; ++e) off[e + 1] = off[e] + cnt[e];
    int32_t *res = (int32_t *)malloc(sizeof(int32_t) * (c->np > 0 ? c->np : 1));
    int32_t *fillc = (int32_t *)calloc(ne, sizeof(int32_t));
    for (int p = 0; p < c->np; ++p) res[off[c->elem[p]] + fillc[c->elem[p]]++] = p;
    free(fillc);

    int32_t *rslot = (int32_t *)malloc(sizeof(int32_t) * T);
    int32_t *dpart = (int32_t *)malloc(sizeof(int32_t) * T);
    int nr = 0, nd = 0;
    for (int e = 0; e < ne; ++e) {
        for (int g = 0; g < fin[e] - cnt[e]; ++g) rslot[nr++] = e;
        for (int l = 0; l < cnt[e] - fin[e]; ++l) dpart[nd++] = res[off[e + 1] - 1 - l];
    }
    /* all new values first (from the state before any move), then apply */
    double (*nv)[7] = malloc(sizeof(double[7]) * T);
    for (int k = 0; k < T; ++k) {
        int p = dpart[k], r = rslot[k];
        uint32_t rw[4];
        philox_draw(c->p.seed, c->p.instance, pid_of(c, p), c->step, PUR_REDIST, 0, rw);
        double s = sqrt(orc_uniform(rw[0]));
        double t = orc_uniform(rw[1]);
        /* uniform point in a triangle: (1-s) A + s (1-t) B + s t C, Osada et al. */
        double px = c->ax[r] + s * (1.0 - t) * c->bx[r] + s * t * c->cx[r];
        double py = c->ay[r] + s * (1.0 - t) * c->by[r] + s * t * c->cy[r];
        px = wrap_x(px, c->p.period_x);
        int src = r;
        if (cnt[r] == 0) {
            src = -1;
            for (int k2 = 0; k2 < 3; ++k2) {
                int nb = c->nbr[3 * r + k2];
                if (nb >= 0 && cnt[nb] > 0 && (src < 0 || nb < src)) src = nb;
            }
        }
        int q = p;
        if (src >= 0) {
            int n = cnt[src];
            int j = (int)(orc_uniform(rw[2]) * (double)n);
            if (j >= n) j = n - 1;
            q = res[off[src] + j];
        }
        nv[k][0] = px; nv[k][1] = py;
        nv[k][2] = c->u[q]; nv[k][3] = c->v[q]; nv[k][4] = c->w[q];
        nv[k][5] = c->om[q];
        nv[k][6] = in_source(c, px, py) ? 1.0 : c->psi[q];
    }
    for (int k = 0; k < T; ++k) {
        int p = dpart[k];
        c->x[p] = nv[k][0]; c->y[p] = nv[k][1];
        c->u[p] = nv[k][2]; c->v[p] = nv[k][3]; c->w[p] = nv[k][4];
        c->om[p] = nv[k][5]; c->psi[p] = nv[k][6];
        c->elem[p] = rslot[k];
    }
    c->diag.moves += T;
    free(nv); free(rslot); free(dpart); free(res); free(off); free(cnt); free(fin);
    return T;
}

/* ------------------------------------------------------------------------------------ */
/* Statistics (Sect. 3.3, Eqs. 35-36) and conditional means (Sect. 3.5, Appendix A).   */
/* ------------------------------------------------------------------------------------ */

static const double *g_sort_key;

/* Sort order of Sect. 3.5 at one level: by the velocity component, ties by particle id. */
static int cmp_by_key(const void *a, const void *b)
{
    int32_t pa = *(const int32_t *)a, pb = *(const int32_t *)b;
    double ka = g_sort_key[pa], kb = g_sort_key[pb];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (pa > pb) - (pa < pb);
}

/* Effective bins.  Reading of Sect. 3.5 ("stopped at any stage ... at least 2 particles
 * ... only use two groups"): level l divides each group into
 * g_l = max(1, min(b_l, floor(N / (g_1 ... g_{l-1} * min_per_bin)))) parts, so every bin
 * keeps at least min_per_bin particles. */
static void effective_bins(const orc_params *P, int N, int g[3])
{
    int Gp = 1;
    for (int l = 0; l < 3; ++l) {
        int cap = N / (Gp * P->min_per_bin);
        int gl = P->bins[l] < cap ? P->bins[l] : cap;
        if (gl < 1) gl = 1;
        g[l] = gl;
        Gp *= gl;
    }
}

/* Fox's projection (Eqs. 64-66).  Per element: rho_a = <u_a phi'> / (s_a s_phi) and
 * rho_ab = <u_a u_b> / (s_a s_b) from the element's central moments (s the standard
 * deviations); alpha solves rho_ab alpha_b = rho_a (Cramer's rule); alpha = 0 when s_phi,
 * an s_a or the determinant vanishes (|det| <= 1e-12).  Reading of Eq. 64: the projected
 * velocity of a particle is U_rho = sum_a alpha_a (U_a - <U_a>) / s_a (the normalised
 * fluctuations the correlations refer to).  The element's particles are ordered by
 * (U_rho, id) and divided into N_c = max(1, min(fox_bins, N / min_per_bin)) equal
 * intervals, position n in interval floor(N_c n / N); the conditional mean of an interval
 * is its mean psi. */
static void fox_alpha(const double *m, const double *uphi, double alpha_over_s[3])
{
    alpha_over_s[0] = alpha_over_s[1] = alpha_over_s[2] = 0.0;
    const double var[3] = {m[4], m[5], m[6]}, vphi = m[12];
    if (!(vphi > 0.0) || !(var[0] > 0.0) || !(var[1] > 0.0) || !(var[2] > 0.0)) return;
    const double s[3] = {sqrt(var[0]), sqrt(var[1]), sqrt(var[2])}, sphi = sqrt(vphi);
    const double cuv = m[7], cuw = m[8], cvw = m[9];
    const double A[3][3] = {{1.0, cuv / (s[0] * s[1]), cuw / (s[0] * s[2])},
                            {cuv / (s[0] * s[1]), 1.0, cvw / (s[1] * s[2])},
                            {cuw / (s[0] * s[2]), cvw / (s[1] * s[2]), 1.0}};
    const double b[3] = {uphi[0] / (s[0] * sphi), uphi[1] / (s[1] * sphi), uphi[2] / (s[2] * sphi)};
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
                     - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
                     + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(fabs(det) > 1e-12)) return;
    for (int i = 0; i < 3; ++i) {
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int col = 0; col < 3; ++col) M[r][col] = col == i ? b[r] : A[r][col];
        const double di = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                        - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                        + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        alpha_over_s[i] = (di / det) / s[i];
    }
}

static void fox_conditional_means(orc_ctx *c, const int32_t *off, int32_t *res)
{
    double *key = (double *)malloc(sizeof(double) * (size_t)(c->np > 0 ? c->np : 1));
    for (int e = 0; e < c->ne; ++e) {
        const int N = c->count[e];
        const double *m = c->emom + (size_t)NS * e;
        int Nc = c->p.fox_bins;
        int cap = N / c->p.min_per_bin;
        if (cap < Nc) Nc = cap;
        if (Nc < 1) Nc = 1;
        c->gbin[3 * e] = Nc; c->gbin[3 * e + 1] = 1; c->gbin[3 * e + 2] = 1;
        if (N == 0) continue;
        double f[3];
        fox_alpha(m, c->uphi + 3 * e, f);
        int32_t *par = res + off[e];
        for (int n = 0; n < N; ++n) {
            const int p = par[n];
            key[p] = f[0] * (c->u[p] - m[1]) + f[1] * (c->v[p] - m[2]) + f[2] * (c->w[p] - m[3]);
        }
        g_sort_key = key;
        qsort(par, (size_t)N, sizeof(int32_t), cmp_by_key);
        double *vc = c->vcce + (size_t)e * c->G;
        int np_bin[256];
        for (int i = 0; i < Nc; ++i) { np_bin[i] = 0; vc[i] = 0.0; }
        for (int n = 0; n < N; ++n) {
            const int i = (int)(((long long)Nc * n) / N);
            np_bin[i] += 1;
            vc[i] += c->psi[par[n]];
            c->cp[par[n]] = (uint8_t)i;
        }
        for (int i = 0; i < Nc; ++i) vc[i] = vc[i] / np_bin[i];
    }
    free(key);
}

int orc_statistics(orc_ctx *c)
{
    const int ne = c->ne, nn = c->nn;
    int32_t *off = (int32_t *)calloc(ne + 1, sizeof(int32_t));
    memset(c->count, 0, sizeof(int32_t) * ne);
    for (int p = 0; p < c->np; ++p) c->count[c->elem[p]]++;
    for (int e = 0; e < ne; ++e) off[e + 1] = off[e] + c->count[e];
    int32_t *res = (int32_t *)malloc(sizeof(int32_t) * (c->np > 0 ? c->np : 1));
    int32_t *fillc = (int32_t *)calloc(ne, sizeof(int32_t));
    for (int p = 0; p < c->np; ++p) res[off[c->elem[p]] + fillc[c->elem[p]]++] = p;
    free(fillc);

    /* Element moments: first pass means (Eq. 35), second pass central moments (Eq. 36).
     * Layout: N, <U>, <V>, <W>, <uu>, <vv>, <ww>, <uv>, <uw>, <vw>, <omega>, <phi>, <phi'^2> */
    for (int e = 0; e < ne; ++e) {
        double *m = c->emom + (size_t)NS * e;
        for (int i = 0; i < NS; ++i) m[i] = 0.0;
        int N = c->count[e];
        m[0] = (double)N;
        if (N == 0) continue;
        double su = 0, sv = 0, sw = 0, so = 0, sp = 0;
        for (int i = off[e]; i < off[e + 1]; ++i) {
            int p = res[i];
            su += c->u[p]; sv += c->v[p]; sw += c->w[p]; so += c->om[p]; sp += c->psi[p];
        }
        double mu = su / N, mv = sv / N, mw = sw / N, mo = so / N, mp = sp / N;
        double suu = 0, svv = 0, sww = 0, suv = 0, suw = 0, svw = 0, spp = 0;
        double sup = 0, svp = 0, swp = 0;
        for (int i = off[e]; i < off[e + 1]; ++i) {
            int p = res[i];
            double du = c->u[p] - mu, dv = c->v[p] - mv, dw = c->w[p] - mw, dp = c->psi[p] - mp;
            suu += du * du; svv += dv * dv; sww += dw * dw;
            suv += du * dv; suw += du * dw; svw += dv * dw;
            spp += dp * dp;
            sup += du * dp; svp += dv * dp; swp += dw * dp;
        }
        c->uphi[3 * e] = sup / N; c->uphi[3 * e + 1] = svp / N; c->uphi[3 * e + 2] = swp / N;
        m[1] = mu; m[2] = mv; m[3] = mw;
        m[4] = suu / N; m[5] = svv / N; m[6] = sww / N;
        m[7] = suv / N; m[8] = suw / N; m[9] = svw / N;
        m[10] = mo; m[11] = mp; m[12] = spp / N;
    }
    /* Node values: average over the surrounding elements (Sect. 3.3).  Reading: plain
     * average over the surrounding elements that hold particles; column 0 is the mean
     * particle count of those elements; a node with none gets zeros. */
    for (int n = 0; n < nn; ++n) {
        double *m = c->nmom + (size_t)NS * n;
        for (int i = 0; i < NS; ++i) m[i] = 0.0;
        int cntn = 0;
        for (int i = c->ne_off[n]; i < c->ne_off[n + 1]; ++i) {
            int e = c->ne_list[i];
            if (c->count[e] < 1) continue;
            const double *em = c->emom + (size_t)NS * e;
            for (int s = 0; s < NS; ++s) m[s] += em[s];
            cntn++;
        }
        if (cntn > 0)
            for (int s = 0; s < NS; ++s) m[s] /= cntn;
    }
    /* Conditional means (Sect. 3.5, Appendix A) */
    const double *keys[3] = {c->u, c->v, c->w};
    memset(c->vcce, 0, sizeof(double) * (size_t)ne * c->G);
    if (c->p.cond_mode == 1) {
        fox_conditional_means(c, off, res);
        free(res);
        free(off);
        return 0;
    }
    for (int e = 0; e < ne; ++e) {
        int N = c->count[e];
        int g[3];
        effective_bins(&c->p, N, g);
        c->gbin[3 * e] = g[0]; c->gbin[3 * e + 1] = g[1]; c->gbin[3 * e + 2] = g[2];
        if (N == 0) continue;
        int32_t *par = res + off[e];                 /* parid[] of Appendix A */
        /* sort & divide: level l sorts each group of the previous level */
        int Gprev = 1;
        for (int l = 0; l < 3; ++l) {
            if (g[l] > 1) {
                g_sort_key = keys[l];
                int start = 0;
                while (start < N) {
                    /* group of position n at the previous level: floor(Gprev n / N) */
                    int grp = (int)(((long long)Gprev * start) / N);
                    int end = start;
                    while (end < N && (int)(((long long)Gprev * end) / N) == grp) end++;
                    qsort(par + start, (size_t)(end - start), sizeof(int32_t), cmp_by_key);
                    start = end;
                }
            }
            Gprev *= g[l];
        }
        /* Appendix A: i = CNBI * n / npel[e] */
        const int CNBI = g[0] * g[1] * g[2];
        int np_bin[256];
        double *vc = c->vcce + (size_t)e * c->G;
        for (int i = 0; i < CNBI; ++i) { np_bin[i] = 0; vc[i] = 0.0; }
        for (int n = 0; n < N; ++n) {
            int i = (int)(((long long)CNBI * n) / N);
            np_bin[i] += 1;
            vc[i] += c->psi[par[n]];
            c->cp[par[n]] = (uint8_t)i;
        }
        for (int i = 0; i < CNBI; ++i) vc[i] = vc[i] / np_bin[i];
    }
    free(res);
    free(off);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Initial particles (Sect. 3.7) and the whole step.                                    */
/* ------------------------------------------------------------------------------------ */

static void alloc_particles(orc_ctx *c, int np)
{
    free(c->x); free(c->y); free(c->u); free(c->v); free(c->w); free(c->om); free(c->psi);
    free(c->elem); free(c->cp); free(c->pid);
    c->pid = NULL;
    c->np = np;
    size_t n = (size_t)(np > 0 ? np : 1);
    c->x = (double *)calloc(n, sizeof(double));
    c->y = (double *)calloc(n, sizeof(double));
    c->u = (double *)calloc(n, sizeof(double));
    c->v = (double *)calloc(n, sizeof(double));
    c->w = (double *)calloc(n, sizeof(double));
    c->om = (double *)calloc(n, sizeof(double));
    c->psi = (double *)calloc(n, sizeof(double));
    c->elem = (int32_t *)calloc(n, sizeof(int32_t));
    c->cp = (uint8_t *)calloc(n, 1);
}

/* Sect. 3.7: an equal number of particles per element, uniform in the element; velocity
 * Gaussian about the local mean with variance 2k/3; frequency gamma with the local mean
 * and variance C4 <omega>^2; psi from the source disc.  Particle id = e * ppe + k.
 * Draws: purpose 1 block 0 (position words 0-1, Gaussians from words 2-3), block 1
 * (third Gaussian from words 0-1); gamma attempts on purpose 4. */
/* Sect. 3.7 initial state of the particle at index p, element e, id id. */
static void init_one(orc_ctx *c, int p, int e, uint32_t id)
{
    uint32_t r0[4], r1[4];
    philox_draw(c->p.seed, c->p.instance, id, 0, PUR_INIT, 0, r0);
    philox_draw(c->p.seed, c->p.instance, id, 0, PUR_INIT, 1, r1);
    double s = sqrt(orc_uniform(r0[0]));
    double t = orc_uniform(r0[1]);
    double px = c->ax[e] + s * (1.0 - t) * c->bx[e] + s * t * c->cx[e];
    double py = c->ay[e] + s * (1.0 - t) * c->by[e] + s * t * c->cy[e];
    double lam[3], q[NF];
    if (c->p.interp_mode == 1) lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
    else orc_lambda(c, e, px, py, lam);
    orc_interp(c, e, lam, q);
    double k2 = 0.5 * (q[23] + q[24] + q[25]);
    if (k2 < 0.0) k2 = 0.0;
    double sd = sqrt(2.0 * k2 / 3.0);
    double g0, g1, g2, gdum;
    orc_box_muller(r0[2], r0[3], &g0, &g1);
    orc_box_muller(r1[0], r1[1], &g2, &gdum);
    int ex = 0;
    double om = orc_gamma_draw(c->p.seed, c->p.instance, id, 0, PUR_INIT_GAMMA,
                               1.0 / c->p.C4, c->p.C4 * q[29], &ex);
    if (ex) c->diag.gamma_exhausted++;
    px = wrap_x(px, c->p.period_x);
    c->x[p] = px; c->y[p] = py;
    c->u[p] = q[0] + sd * g0;
    c->v[p] = q[1] + sd * g1;
    c->w[p] = q[2] + sd * g2;
    c->om[p] = om;
    c->psi[p] = in_source(c, px, py) ? 1.0 : 0.0;
    c->elem[p] = e;
}

int orc_init_particles(orc_ctx *c, int ppe)
{
    if (ppe <= 0) return -1;
    long long np = (long long)ppe * c->ne;
    if (np > 2147483647LL) return -1;
    alloc_particles(c, (int)np);
    c->step = 0;
    memset(&c->diag, 0, sizeof(c->diag));
    for (int e = 0; e < c->ne; ++e)
        for (int k = 0; k < ppe; ++k) init_one(c, e * ppe + k, e, (uint32_t)(e * ppe + k));
    return orc_statistics(c);
}

/* The particles of a run initialised with ppe per element, for the listed elements only
 * (ascending): the same ids (e * ppe + k) and draws, so the oracle can follow a sample of a
 * run too large for it. */
int orc_init_elements(orc_ctx *c, int ppe, int n, const int32_t *elems)
{
    if (ppe <= 0 || n < 0) return -1;
    for (int i = 0; i < n; ++i)
        if (elems[i] < 0 || elems[i] >= c->ne || (i > 0 && elems[i] <= elems[i - 1])) return -2;
    if ((long long)ppe * c->ne > 4294967295LL) return -1;
    alloc_particles(c, n * ppe);
    c->pid = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n * ppe > 0 ? n * ppe : 1));
    c->step = 0;
    memset(&c->diag, 0, sizeof(c->diag));
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < ppe; ++k) {
            const int p = i * ppe + k;
            c->pid[p] = (uint32_t)elems[i] * (uint32_t)ppe + (uint32_t)k;
            init_one(c, p, elems[i], c->pid[p]);
        }
    return orc_statistics(c);
}

/* As orc_set_particles with explicit, strictly ascending particle ids. */
int orc_set_particles_ids(orc_ctx *c, int np, const double *x, const double *y, const double *u,
                          const double *v, const double *w, const double *om, const double *psi,
                          const int32_t *elem, const uint32_t *pid, uint32_t step)
{
    for (int p = 1; p < np; ++p)
        if (pid[p] <= pid[p - 1]) return -3;
    int rc = orc_set_particles(c, np, x, y, u, v, w, om, psi, elem, step);
    if (rc) return rc;
    c->pid = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(np > 0 ? np : 1));
    memcpy(c->pid, pid, sizeof(uint32_t) * (size_t)np);
    return orc_statistics(c);
}

int orc_get_pids(const orc_ctx *c, uint32_t *out)
{
    for (int p = 0; p < c->np; ++p) out[p] = pid_of(c, p);
    return 0;
}

int orc_set_particles(orc_ctx *c, int np, const double *x, const double *y, const double *u,
                      const double *v, const double *w, const double *om, const double *psi,
                      const int32_t *elem, uint32_t step)
{
    if (np < 0) return -1;
    for (int p = 0; p < np; ++p)
        if (elem[p] < 0 || elem[p] >= c->ne) return -2;
    alloc_particles(c, np);
    memcpy(c->x, x, sizeof(double) * np);
    memcpy(c->y, y, sizeof(double) * np);
    memcpy(c->u, u, sizeof(double) * np);
    memcpy(c->v, v, sizeof(double) * np);
    memcpy(c->w, w, sizeof(double) * np);
    memcpy(c->om, om, sizeof(double) * np);
    memcpy(c->psi, psi, sizeof(double) * np);
    memcpy(c->elem, elem, sizeof(int32_t) * np);
    c->step = step;
    return orc_statistics(c);
}

int orc_get_particles(const orc_ctx *c, double *x, double *y, double *u, double *v, double *w,
                      double *om, double *psi, int32_t *elem, uint8_t *cp)
{
    size_t n = (size_t)c->np;
    if (x) memcpy(x, c->x, sizeof(double) * n);
    if (y) memcpy(y, c->y, sizeof(double) * n);
    if (u) memcpy(u, c->u, sizeof(double) * n);
    if (v) memcpy(v, c->v, sizeof(double) * n);
    if (w) memcpy(w, c->w, sizeof(double) * n);
    if (om) memcpy(om, c->om, sizeof(double) * n);
    if (psi) memcpy(psi, c->psi, sizeof(double) * n);
    if (elem) memcpy(elem, c->elem, sizeof(int32_t) * n);
    if (cp) memcpy(cp, c->cp, n);
    return 0;
}

int orc_num_particles(const orc_ctx *c) { return c->np; }
uint32_t orc_step_index(const orc_ctx *c) { return c->step; }

/* Eq. 26: dt = CFL min_n sqrt(A_n) / max_n ||<Z>_n||_2, A_n the average area of the
 * elements around node n and <Z>_n = (<U>, <V>, <W>, <omega>, <psi>) the nodal means of the
 * last statistics pass.  Reading: the norm is taken literally, omega and psi included;
 * nodes that no element holding particles surrounds have zero means and take part; the
 * step cannot be derived (returns -1) when every nodal mean vector is zero. */
int orc_cfl_dt(const orc_ctx *c, double *dt)
{
    double min_sqrt_a = INFINITY, max_norm = 0.0;
    for (int n = 0; n < c->nn; ++n) {
        const int m = c->ne_off[n + 1] - c->ne_off[n];
        if (m > 0) {
            double a = 0.0;
            for (int i = c->ne_off[n]; i < c->ne_off[n + 1]; ++i) a += 0.5 * fabs(c->area2[c->ne_list[i]]);
            const double s = sqrt(a / m);
            if (s < min_sqrt_a) min_sqrt_a = s;
        }
        const double *z = c->nmom + (size_t)NS * n;
        const double norm = sqrt(z[1] * z[1] + z[2] * z[2] + z[3] * z[3] + z[10] * z[10] + z[11] * z[11]);
        if (norm > max_norm) max_norm = norm;
    }
    if (!(max_norm > 0.0) || !isfinite(min_sqrt_a)) return -1;
    *dt = c->p.cfl * min_sqrt_a / max_norm;
    return 0;
}

double orc_last_dt(const orc_ctx *c) { return c->last_dt; }

/* Sect. 3.4.  Eq. 39 with the shapefunction derivatives of Eq. 40 (constant over the
 * element, from its vertices in the element's frame, x_CA = x_C - x_A and so on, and twice
 * its area): dQ/dx = sum_j dN^j/dx Q_j.  The element values are then transferred to the
 * nodes as the plain mean over the elements around each node. */
void orc_node_gradient(const orc_ctx *c, const double *q, double *grad)
{
    for (int n = 0; n < c->nn; ++n) {
        double gx = 0.0, gy = 0.0;
        const int m = c->ne_off[n + 1] - c->ne_off[n];
        for (int i = c->ne_off[n]; i < c->ne_off[n + 1]; ++i) {
            const int e = c->ne_list[i];
            const double *vx = c->vx + 3 * e, *vy = c->vy + 3 * e;
            const double xBA = vx[1] - vx[0], yBA = vy[1] - vy[0];
            const double xCA = vx[2] - vx[0], yCA = vy[2] - vy[0];
            const double inv = 1.0 / c->area2[e];
            const double dNx[3] = {(-yCA + yBA) * inv, yCA * inv, -yBA * inv};
            const double dNy[3] = {(xCA - xBA) * inv, -xCA * inv, xBA * inv};
            const int32_t *t = c->tri + 3 * e;
            gx += dNx[0] * q[t[0]] + dNx[1] * q[t[1]] + dNx[2] * q[t[2]];
            gy += dNy[0] * q[t[0]] + dNy[1] * q[t[1]] + dNy[2] * q[t[2]];
        }
        grad[2 * n] = m > 0 ? gx / m : 0.0;
        grad[2 * n + 1] = m > 0 ? gy / m : 0.0;
    }
}

/* The nodal fields that the particles' own statistics provide (the non-hybrid coupling of
 * Sect. 3.3-3.4): <U_i> (slots 0-2) = the nodal means; d<U_i>/dx_j (slots 5-10, i-major)
 * = their node-transferred gradients; the laplacian of <U_i> (slots 11-13) =
 * d/dx (d<U_i>/dx) + d/dy (d<U_i>/dy) by the same procedure applied to the nodal first
 * derivatives (the two-pass second derivatives of Sect. 3.4); <u_i u_j> (slots 23-28) and
 * <omega> (slot 29) = the nodal moments.  The mean-pressure gradient, the
 * elliptic-relaxation tensor and the wall frequency (slots 3-4, 14-22, 30) come from the
 * Eulerian solves and are kept. */
/* Sect. 3.2, Eq. 31: the mean-velocity correction <U>^{n+1} = <U>* - dt grad(<P>^{n+1} -
 * <P>^n) / rho applied to every particle (the velocity field is the particles', rho = 1),
 * the gradient of the nodal pressure change being constant over the particle's element
 * (Eq. 39 with Eq. 40's derivatives).  The third velocity component has no gradient in the
 * plane and is unchanged. */
int orc_correct_velocity(orc_ctx *c, const double *dp, double dt)
{
    if (!c->x) return -1;
    for (int p = 0; p < c->np; ++p) {
        const int e = c->elem[p];
        const double *vx = c->vx + 3 * e, *vy = c->vy + 3 * e;
        const double xBA = vx[1] - vx[0], yBA = vy[1] - vy[0];
        const double xCA = vx[2] - vx[0], yCA = vy[2] - vy[0];
        const double inv = 1.0 / c->area2[e];
        const int32_t *t = c->tri + 3 * e;
        const double gx = (-yCA + yBA) * inv * dp[t[0]] + yCA * inv * dp[t[1]] - yBA * inv * dp[t[2]];
        const double gy = (xCA - xBA) * inv * dp[t[0]] - xCA * inv * dp[t[1]] + xBA * inv * dp[t[2]];
        c->u[p] -= dt * gx;
        c->v[p] -= dt * gy;
    }
    return 0;
}

int orc_get_fields(const orc_ctx *c, double *out)
{
    memcpy(out, c->fields, sizeof(double) * (size_t)NF * c->nn);
    return 0;
}

int orc_derive_fields(orc_ctx *c)
{
    const int nn = c->nn;
    double *q = (double *)malloc(sizeof(double) * (size_t)nn);
    double *g1 = (double *)malloc(sizeof(double) * 2 * (size_t)nn);
    double *g2 = (double *)malloc(sizeof(double) * 2 * (size_t)nn);
    double *first = (double *)malloc(sizeof(double) * 6 * (size_t)nn);
    double *lap = (double *)calloc(3 * (size_t)nn, sizeof(double));
    for (int i = 0; i < 3; ++i) {
        for (int n = 0; n < nn; ++n) q[n] = c->nmom[(size_t)NS * n + 1 + i];
        orc_node_gradient(c, q, g1);
        for (int n = 0; n < nn; ++n) {
            first[6 * n + 2 * i] = g1[2 * n];
            first[6 * n + 2 * i + 1] = g1[2 * n + 1];
        }
        for (int j = 0; j < 2; ++j) {
            for (int n = 0; n < nn; ++n) q[n] = g1[2 * n + j];
            orc_node_gradient(c, q, g2);
            for (int n = 0; n < nn; ++n) lap[3 * n + i] += g2[2 * n + j];
        }
    }
    for (int n = 0; n < nn; ++n) {
        double *f = c->fields + (size_t)NF * n;
        const double *m = c->nmom + (size_t)NS * n;
        for (int i = 0; i < 3; ++i) f[i] = m[1 + i];
        for (int k = 0; k < 6; ++k) f[5 + k] = first[6 * n + k];
        for (int i = 0; i < 3; ++i) f[11 + i] = lap[3 * n + i];
        for (int k = 0; k < 6; ++k) f[23 + k] = m[4 + k];
        f[29] = m[10];
    }
    free(q); free(g1); free(g2); free(first); free(lap);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Elliptic relaxation (Sect. 2, Eqs. 12-18; Sect. 3.2; Eq. 59).                          */
/* ------------------------------------------------------------------------------------ */

/* Boundary class of every node: 1 where a no-slip edge (tag 1) ends, else 2 where a
 * free-slip edge (tag 2) ends, else 0.  For class-1 nodes (onx, ony) is the unit outward
 * normal: the normalised sum of the outward unit normals of the node's no-slip edges (one
 * edge's normal on a straight wall; the bisector at a corner). */
static void node_boundary(const orc_ctx *c, int8_t *cls, double *onx, double *ony)
{
    for (int n = 0; n < c->nn; ++n) { cls[n] = 0; onx[n] = 0.0; ony[n] = 0.0; }
    for (int e = 0; e < c->ne; ++e) {
        for (int k = 0; k < 3; ++k) {
            const int t = c->tag[3 * e + k];
            if (t != 1 && t != 2) continue;
            double px, py, mx, my;
            edge_line(c, e, k, &px, &py, &mx, &my);   /* (mx, my) points into the domain */
            const int ends[2] = {c->tri[3 * e + (k + 1) % 3], c->tri[3 * e + (k + 2) % 3]};
            for (int s = 0; s < 2; ++s) {
                const int n = ends[s];
                if (t == 1) {
                    cls[n] = 1;
                    onx[n] -= mx;
                    ony[n] -= my;
                } else if (cls[n] == 0) {
                    cls[n] = 2;
                }
            }
        }
    }
    for (int n = 0; n < c->nn; ++n) {
        if (cls[n] != 1) continue;
        const double len = sqrt(onx[n] * onx[n] + ony[n] * ony[n]);
        if (len > 0.0) { onx[n] /= len; ony[n] /= len; }
    }
}

/* Eq. 17's n_i: the unit outward normal of the no-slip edge nearest to the point (x, y)
 * (point-to-segment distance, minimum image in x; the first edge in element and local edge
 * order wins a tie).  Returns 0 and n = 0 when the grid has no no-slip edge. */
static int nearest_wall_normal(const orc_ctx *c, double x, double y, double *nx, double *ny)
{
    double best = INFINITY;
    *nx = 0.0; *ny = 0.0;
    for (int e = 0; e < c->ne; ++e) {
        for (int k = 0; k < 3; ++k) {
            if (c->tag[3 * e + k] != 1) continue;
            const double *vx = c->vx + 3 * e, *vy = c->vy + 3 * e;
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            /* segment in the frame of the point */
            const double ax = x + min_image(vx[a] - x, c->p.period_x), ay = vy[a];
            const double bx = ax + (vx[b] - vx[a]), by = vy[b];
            const double tx = bx - ax, ty = by - ay;
            double s = ((x - ax) * tx + (y - ay) * ty) / (tx * tx + ty * ty);
            s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
            const double dx = x - (ax + s * tx), dy = y - (ay + s * ty);
            const double d = sqrt(dx * dx + dy * dy);
            if (d < best) {
                double px, py, mx, my;
                edge_line(c, e, k, &px, &py, &mx, &my);
                best = d;
                *nx = -mx;
                *ny = -my;
            }
        }
    }
    return isfinite(best);
}

/* Eqs. 12-18 at every node, from the context's nodal fields: the local right-hand side of
 * Eq. 12,
 *     rhs_ij = (1 - C1)/2 k <omega> delta_ij + k H_ijkl d<U_k>/dx_l,
 * with H_ijkl of Eq. 13, A_v of Eq. 14 and b_ij of Eq. 15, and the length scale L of
 * Eq. 16 with C_xi of Eq. 17 and eps of Eq. 18.  Inputs: d<U_k>/dx_l (slots 5-10, k-major,
 * l = x, y; d/dz = 0 in the plane), <u_i u_j> (slots 23-28), <omega> (slot 29); nu and the
 * constants of Table 4 from the parameters.  Readings: b_ij = 0 where <u_k u_k> = 0 and
 * A_v = 0 where k = 0 (every term of the right-hand side carries the factor k there, so
 * neither choice shows); A_v is min[1, .] as printed, with no lower bound; C_xi takes the
 * printed n_i n_i of a unit normal, which is 1 wherever a no-slip wall exists (C_xi = 2.3)
 * and 0 on a grid without one (C_xi = 1).  A node with eps <= 0 has no length scale:
 * the call fails.  rhs[nn][9] is row-major (i, j); L[nn]. */
int orc_wp_rhs(const orc_ctx *c, double *rhs, double *L)
{
    const orc_params *p = &c->p;
    for (int n = 0; n < c->nn; ++n) {
        const double *f = c->fields + (size_t)NF * n;
        const double R[3][3] = {{f[23], f[26], f[27]}, {f[26], f[24], f[28]}, {f[27], f[28], f[25]}};
        const double G[3][3] = {{f[5], f[6], 0.0}, {f[7], f[8], 0.0}, {f[9], f[10], 0.0}};
        const double om = f[29];
        const double ukuk = R[0][0] + R[1][1] + R[2][2];
        const double k = 0.5 * ukuk;
        double b[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                b[i][j] = ukuk > 0.0 ? R[i][j] / ukuk - (i == j ? 1.0 / 3.0 : 0.0) : 0.0;   /* Eq. 15 */
        const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1])
                         - R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0])
                         + R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
        const double k23 = 2.0 * k / 3.0;
        const double Av = k > 0.0 ? fmin(1.0, p->Cv * det / (k23 * k23 * k23)) : 0.0;   /* Eq. 14 */
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int kk = 0; kk < 3; ++kk) {
                    for (int l = 0; l < 3; ++l) {
                        const double d_ik = i == kk, d_jl = j == l, d_il = i == l, d_jk = j == kk;
                        const double H = (p->C2 * Av + p->gamma5 / 3.0) * d_ik * d_jl       /* Eq. 13 */
                                       - (p->gamma5 / 3.0) * d_il * d_jk
                                       + p->gamma5 * b[i][kk] * d_jl
                                       - p->gamma5 * b[i][l] * d_jk;
                        s += H * G[kk][l];
                    }
                }
                rhs[(size_t)9 * n + 3 * i + j] =
                    (i == j ? 0.5 * (1.0 - p->C1) * k * om : 0.0) + k * s;            /* Eq. 12 */
            }
        }
        const double eps = om * (k + p->nu * p->CT * p->CT * om);                    /* Eq. 18 */
        if (!(eps > 0.0)) return -1;
        double nx, ny;
        nearest_wall_normal(c, c->node_xy[2 * n], c->node_xy[2 * n + 1], &nx, &ny);
        const double Cxi = 1.0 + 1.3 * (nx * nx + ny * ny);                           /* Eq. 17 */
        L[n] = p->CL * fmax(Cxi * pow(k, 1.5) / eps,
                            p->Ceta * pow(p->nu * p->nu * p->nu / eps, 0.25));         /* Eq. 16 */
    }
    return 0;
}

/* y = (M + K) x for one component: the Galerkin matrices of Eq. 12's operator with linear
 * triangles (Sect. 3.2), the consistent mass matrix M_e = A_e/12 (1 + delta_ab) and the
 * stiffness K_e = L_e^2 A_e grad N_a . grad N_b with Eq. 40's derivatives; L_e^2 is the mean
 * of the element's three nodal L^2.  Reading: the paper solves Eq. 12 by conjugate
 * gradients, whose matrix must be symmetric, so the operator is div(L_e^2 grad) with L^2
 * constant over each element (the L^2 grad(N_a) . grad(wp) weak form without the
 * non-symmetric N_a grad(L^2) . grad(wp) term).  Elements use their vertices in the
 * element's frame, so a periodic seam needs nothing else. */
static void wp_operator(const orc_ctx *c, const double *L, const double *x, double *y, double *diag)
{
    for (int n = 0; n < c->nn; ++n) y[n] = 0.0;
    if (diag) for (int n = 0; n < c->nn; ++n) diag[n] = 0.0;
    for (int e = 0; e < c->ne; ++e) {
        const double *vx = c->vx + 3 * e, *vy = c->vy + 3 * e;
        const double xBA = vx[1] - vx[0], yBA = vy[1] - vy[0];
        const double xCA = vx[2] - vx[0], yCA = vy[2] - vy[0];
        const double A = 0.5 * c->area2[e];
        const double inv = 1.0 / c->area2[e];
        const double dNx[3] = {(-yCA + yBA) * inv, yCA * inv, -yBA * inv};   /* Eq. 40 */
        const double dNy[3] = {(xCA - xBA) * inv, -xCA * inv, xBA * inv};
        const int32_t *t = c->tri + 3 * e;
        const double L2 = (L[t[0]] * L[t[0]] + L[t[1]] * L[t[1]] + L[t[2]] * L[t[2]]) / 3.0;
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) {
                const double m = A / 12.0 * (a == b ? 2.0 : 1.0);
                const double kab = L2 * A * (dNx[a] * dNx[b] + dNy[a] * dNy[b]);
                y[t[a]] += (m + kab) * x[t[b]];
                if (diag && a == b) diag[t[a]] += m + kab;
            }
        }
    }
}

/* y = M x with the consistent mass matrix (the Galerkin load of a linearly interpolated
 * right-hand side). */
static void mass_apply(const orc_ctx *c, const double *x, double *y)
{
    for (int n = 0; n < c->nn; ++n) y[n] = 0.0;
    for (int e = 0; e < c->ne; ++e) {
        const double A = 0.5 * c->area2[e];
        const int32_t *t = c->tri + 3 * e;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) y[t[a]] += A / 12.0 * (a == b ? 2.0 : 1.0) * x[t[b]];
    }
}

/* The Galerkin operators as plain functions (test access): which = 0 the consistent mass
 * matrix, 1 the laplacian stiffness. */
static void stiffness_apply(const orc_ctx *c, const double *x, double *y, double *diag);
void orc_fem_apply(const orc_ctx *c, int which, const double *x, double *y)
{
    if (which == 0) mass_apply(c, x, y);
    else stiffness_apply(c, x, y, NULL);
}

/* y = (M + K_L) x, Eq. 12's Galerkin operator with the nodal length scale L (test access). */
void orc_wp_apply(const orc_ctx *c, const double *L, const double *x, double *y)
{
    wp_operator(c, L, x, y, NULL);
}

static double dot_free(const double *a, const double *b, const int8_t *fixed, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        if (!fixed[i]) s += a[i] * b[i];
    return s;
}

/* Eq. 12 solved for the nine components of wp_ij (Sect. 3.2: Galerkin FEM with linear
 * triangles, conjugate gradients with a Jacobi preconditioner started from the previous
 * solution).  Boundary conditions: at no-slip nodes wp_ij = -4.5 eps n_i n_j (Eq. 59; eps of
 * Eq. 18 from the node's fields, n the node's outward unit normal, n_z = 0); at free-slip
 * nodes the symmetry conditions of Sect. 4.1, homogeneous Dirichlet for i != j and the
 * natural (zero normal derivative) condition for i == j; a node on both kinds takes the
 * no-slip condition.  rhs[nn][9], L[nn]; wp[nn][9] holds the initial guess on entry and the
 * solution on exit.  Each component iterates until the preconditioned residual's
 * 2-norm over the free nodes is at most tol times that of its reduced load (the load minus
 * the Dirichlet columns), a zero reduced load giving the zero solution on the free nodes
 * at once; *iters returns the largest count.  Fails (-2) if a component
 * needs more than max_iter iterations, (-1) if an eps needed at a wall is not positive. */
int orc_wp_solve(const orc_ctx *c, const double *rhs, const double *L, double *wp, double tol,
                 int max_iter, int *iters)
{
    const int nn = c->nn;
    int8_t *cls = (int8_t *)malloc((size_t)nn);
    int8_t *fixed = (int8_t *)malloc((size_t)nn);
    double *onx = (double *)malloc(sizeof(double) * nn), *ony = (double *)malloc(sizeof(double) * nn);
    double *f = (double *)malloc(sizeof(double) * nn), *bl = (double *)malloc(sizeof(double) * nn);
    double *x = (double *)malloc(sizeof(double) * nn), *r = (double *)malloc(sizeof(double) * nn);
    double *z = (double *)malloc(sizeof(double) * nn), *d = (double *)malloc(sizeof(double) * nn);
    double *q = (double *)malloc(sizeof(double) * nn), *dg = (double *)malloc(sizeof(double) * nn);
    double *x0 = (double *)malloc(sizeof(double) * nn);
    int rc = 0, worst = 0;
    node_boundary(c, cls, onx, ony);
    for (int comp = 0; comp < 9 && rc == 0; ++comp) {
        const int i = comp / 3, j = comp % 3;
        for (int n = 0; n < nn; ++n) {
            f[n] = rhs[(size_t)9 * n + comp];
            x[n] = wp[(size_t)9 * n + comp];
            fixed[n] = 0;
            if (cls[n] == 1) {
                const double *fl = c->fields + (size_t)NF * n;
                const double k = 0.5 * (fl[23] + fl[24] + fl[25]), om = fl[29];
                const double eps = om * (k + c->p.nu * c->p.CT * c->p.CT * om);
                if (!(eps > 0.0)) { rc = -1; break; }
                const double nv[3] = {onx[n], ony[n], 0.0};
                x[n] = -4.5 * eps * nv[i] * nv[j];                                      /* Eq. 59 */
                fixed[n] = 1;
            } else if (cls[n] == 2 && i != j) {
                x[n] = 0.0;
                fixed[n] = 1;
            }
        }
        if (rc) break;
        mass_apply(c, f, bl);
        /* reduced load: bl - A (Dirichlet values, zero elsewhere), on the free nodes */
        for (int n = 0; n < nn; ++n) x0[n] = fixed[n] ? x[n] : 0.0;
        wp_operator(c, L, x0, q, dg);
        for (int n = 0; n < nn; ++n) q[n] = bl[n] - q[n];
        for (int n = 0; n < nn; ++n) z[n] = fixed[n] ? 0.0 : q[n] / dg[n];
        const double bnorm = sqrt(dot_free(z, z, fixed, nn));
        if (bnorm == 0.0)   /* a zero reduced load: the free nodes' solution is zero */
            for (int n = 0; n < nn; ++n)
                if (!fixed[n]) x[n] = 0.0;
        /* r = bl - A x on the free nodes */
        wp_operator(c, L, x, q, NULL);
        for (int n = 0; n < nn; ++n) r[n] = fixed[n] ? 0.0 : bl[n] - q[n];
        for (int n = 0; n < nn; ++n) z[n] = fixed[n] ? 0.0 : r[n] / dg[n];
        for (int n = 0; n < nn; ++n) d[n] = z[n];
        double rz = dot_free(r, z, fixed, nn);
        int it = 0;
        while (sqrt(dot_free(z, z, fixed, nn)) > tol * bnorm) {
            if (it == max_iter) { rc = -2; break; }
            wp_operator(c, L, d, q, NULL);
            for (int n = 0; n < nn; ++n) if (fixed[n]) q[n] = 0.0;
            const double alpha = rz / dot_free(d, q, fixed, nn);
            for (int n = 0; n < nn; ++n) {
                if (fixed[n]) continue;
                x[n] += alpha * d[n];
                r[n] -= alpha * q[n];
                z[n] = r[n] / dg[n];
            }
            const double rz1 = dot_free(r, z, fixed, nn);
            const double beta = rz1 / rz;
            rz = rz1;
            for (int n = 0; n < nn; ++n) d[n] = fixed[n] ? 0.0 : z[n] + beta * d[n];
            ++it;
        }
        if (it > worst) worst = it;
        for (int n = 0; n < nn; ++n) wp[(size_t)9 * n + comp] = x[n];
    }
    if (iters) *iters = worst;
    free(cls); free(fixed); free(onx); free(ony); free(f); free(bl); free(x); free(r);
    free(z); free(d); free(q); free(dg); free(x0);
    return rc;
}

/* The elliptic-relaxation update of the coupled loop: Eq. 12's right-hand side and length
 * scale from the current nodal fields, solved from the fields' wp_ij (slots 14-22) as the
 * initial guess, the solution written back to slots 14-22. */
int orc_update_wp(orc_ctx *c, double tol, int max_iter, int *iters)
{
    const int nn = c->nn;
    double *rhs = (double *)malloc(sizeof(double) * 9 * (size_t)nn);
    double *L = (double *)malloc(sizeof(double) * (size_t)nn);
    double *wp = (double *)malloc(sizeof(double) * 9 * (size_t)nn);
    int rc = orc_wp_rhs(c, rhs, L);
    if (rc == 0) {
        for (int n = 0; n < nn; ++n)
            for (int m = 0; m < 9; ++m) wp[(size_t)9 * n + m] = c->fields[(size_t)NF * n + 14 + m];
        rc = orc_wp_solve(c, rhs, L, wp, tol, max_iter, iters);
        if (rc == 0)
            for (int n = 0; n < nn; ++n)
                for (int m = 0; m < 9; ++m) c->fields[(size_t)NF * n + 14 + m] = wp[(size_t)9 * n + m];
    }
    free(rhs); free(L); free(wp);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Pressure projection (Sect. 3.2, Eqs. 28-33; Eqs. 60-61) and the coupled step.          */
/* ------------------------------------------------------------------------------------ */

/* The nodal right-hand side of Eq. 33 with rho = 1,
 *     src = (div <U>* - C_p lap <P>^n) / dt,
 * with div <U>* from the node-transferred gradients of the nodal means ustar[nn][3] and
 * lap <P>^n by the two passes of Sect. 3.4 applied to P[nn]; and the normal derivative of
 * the pressure increment at no-slip nodes (zero elsewhere), flux[nn].  Reading: Eq. 61
 * fixes the outward normal derivative of <P>^{n+1}; with the current nodal fields (the
 * laplacian of <U_i>, slots 11-12, and the node-transferred gradients of <u_i u_j>, slots
 * 23, 24 and 26) it is nu lap<U_i> n_i - d<u_i u_j>/dx_j n_i, and the increment's is that
 * value minus n . grad <P>^n (the node-transferred gradient of P); n is the node's outward
 * unit normal (the bisector at a corner).  Free-slip rows are symmetry lines, where the
 * normal derivative is zero. */
int orc_pressure_rhs(const orc_ctx *c, const double *ustar, const double *P, double dt, double Cp,
                     double *src, double *flux)
{
    const int nn = c->nn;
    if (!(dt > 0.0)) return -1;
    double *q = (double *)calloc((size_t)nn, sizeof(double));
    double *gu = (double *)malloc(sizeof(double) * 2 * nn), *gv = (double *)malloc(sizeof(double) * 2 * nn);
    double *gp = (double *)malloc(sizeof(double) * 2 * nn), *g2 = (double *)malloc(sizeof(double) * 2 * nn);
    double *lapP = (double *)calloc((size_t)nn, sizeof(double));
    double *guu = (double *)malloc(sizeof(double) * 2 * nn), *gvv = (double *)malloc(sizeof(double) * 2 * nn);
    double *guv = (double *)malloc(sizeof(double) * 2 * nn);
    double *onx = (double *)malloc(sizeof(double) * nn), *ony = (double *)malloc(sizeof(double) * nn);
    int8_t *cls = (int8_t *)malloc((size_t)nn);
    for (int n = 0; n < nn; ++n) q[n] = ustar[3 * n];
    orc_node_gradient(c, q, gu);
    for (int n = 0; n < nn; ++n) q[n] = ustar[3 * n + 1];
    orc_node_gradient(c, q, gv);
    orc_node_gradient(c, P, gp);
    for (int j = 0; j < 2; ++j) {
        for (int n = 0; n < nn; ++n) q[n] = gp[2 * n + j];
        orc_node_gradient(c, q, g2);
        for (int n = 0; n < nn; ++n) lapP[n] += g2[2 * n + j];
    }
    for (int n = 0; n < nn; ++n) src[n] = (gu[2 * n] + gv[2 * n + 1] - Cp * lapP[n]) / dt;   /* Eq. 33 */
    const int slots[3] = {23, 24, 26};                 /* <uu>, <vv>, <uv> */
    double *gs[3] = {guu, gvv, guv};
    for (int s = 0; s < 3; ++s) {
        for (int n = 0; n < nn; ++n) q[n] = c->fields[(size_t)NF * n + slots[s]];
        orc_node_gradient(c, q, gs[s]);
    }
    node_boundary(c, cls, onx, ony);
    for (int n = 0; n < nn; ++n) {
        flux[n] = 0.0;
        if (cls[n] != 1) continue;
        const double *f = c->fields + (size_t)NF * n;
        const double divx = guu[2 * n] + guv[2 * n + 1];   /* d<u u_j>/dx_j */
        const double divy = guv[2 * n] + gvv[2 * n + 1];   /* d<v u_j>/dx_j */
        const double eq61 = c->p.nu * (f[11] * onx[n] + f[12] * ony[n]) - (divx * onx[n] + divy * ony[n]);
        flux[n] = eq61 - (gp[2 * n] * onx[n] + gp[2 * n + 1] * ony[n]);
    }
    free(q); free(gu); free(gv); free(gp); free(g2); free(lapP); free(guu); free(gvv); free(guv);
    free(onx); free(ony); free(cls);
    return 0;
}

/* y = K x, the Galerkin stiffness of the laplacian with linear triangles (Eq. 40). */
static void stiffness_apply(const orc_ctx *c, const double *x, double *y, double *diag)
{
    for (int n = 0; n < c->nn; ++n) y[n] = 0.0;
    if (diag) for (int n = 0; n < c->nn; ++n) diag[n] = 0.0;
    for (int e = 0; e < c->ne; ++e) {
        const double *vx = c->vx + 3 * e, *vy = c->vy + 3 * e;
        const double xBA = vx[1] - vx[0], yBA = vy[1] - vy[0];
        const double xCA = vx[2] - vx[0], yCA = vy[2] - vy[0];
        const double A = 0.5 * c->area2[e];
        const double inv = 1.0 / c->area2[e];
        const double dNx[3] = {(-yCA + yBA) * inv, yCA * inv, -yBA * inv};
        const double dNy[3] = {(xCA - xBA) * inv, -xCA * inv, xBA * inv};
        const int32_t *t = c->tri + 3 * e;
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) {
                const double kab = A * (dNx[a] * dNx[b] + dNy[a] * dNy[b]);
                y[t[a]] += kab * x[t[b]];
                if (diag && a == b) diag[t[a]] += kab;
            }
        }
    }
}

/* Eq. 33 by Galerkin FEM with linear triangles (Sect. 3.2): the weak form
 *     int grad N_a . grad dP = int_boundary N_a dP/dn - int N_a src
 * with src[nn] interpolated linearly (consistent mass matrix) and the normal derivative
 * flux[nn] interpolated linearly along each no-slip edge (edge length l: l/6 (2 g_a + g_b)
 * to node a).  The matrix is singular (periodic and Neumann boundaries only: constants
 * are its null space).  Readings: the load's component along the constants (the
 * statistical defect of the compatibility condition) is removed by subtracting its nodal
 * mean; conjugate gradients with the Jacobi preconditioner, started from dP, then solve
 * the consistent system, and the solution is shifted to zero integral over the domain.
 * Stopping rule and iteration limit as in orc_wp_solve. */
int orc_pressure_solve(const orc_ctx *c, const double *src, const double *flux, double *dP,
                       double tol, int max_iter, int *iters)
{
    const int nn = c->nn;
    double *b = (double *)malloc(sizeof(double) * nn), *r = (double *)malloc(sizeof(double) * nn);
    double *z = (double *)malloc(sizeof(double) * nn), *d = (double *)malloc(sizeof(double) * nn);
    double *q = (double *)malloc(sizeof(double) * nn), *dg = (double *)malloc(sizeof(double) * nn);
    int8_t *none = (int8_t *)calloc((size_t)nn, 1);
    int rc = 0;
    mass_apply(c, src, b);
    for (int n = 0; n < nn; ++n) b[n] = -b[n];
    for (int e = 0; e < c->ne; ++e) {
        for (int k = 0; k < 3; ++k) {
            if (c->tag[3 * e + k] != 1) continue;
            const int ia = (k + 1) % 3, ib = (k + 2) % 3;
            const int na = c->tri[3 * e + ia], nb = c->tri[3 * e + ib];
            const double ex = c->vx[3 * e + ib] - c->vx[3 * e + ia], ey = c->vy[3 * e + ib] - c->vy[3 * e + ia];
            const double l = sqrt(ex * ex + ey * ey);
            b[na] += l / 6.0 * (2.0 * flux[na] + flux[nb]);
            b[nb] += l / 6.0 * (flux[na] + 2.0 * flux[nb]);
        }
    }
    double mean = 0.0;
    for (int n = 0; n < nn; ++n) mean += b[n];
    mean /= nn;
    for (int n = 0; n < nn; ++n) b[n] -= mean;
    stiffness_apply(c, dP, q, dg);
    for (int n = 0; n < nn; ++n) z[n] = b[n] / dg[n];
    const double bnorm = sqrt(dot_free(z, z, none, nn));
    if (bnorm == 0.0)   /* a zero load: the solution is zero */
        for (int n = 0; n < nn; ++n) { dP[n] = 0.0; q[n] = 0.0; }
    for (int n = 0; n < nn; ++n) r[n] = b[n] - q[n];
    for (int n = 0; n < nn; ++n) { z[n] = r[n] / dg[n]; d[n] = z[n]; }
    double rz = dot_free(r, z, none, nn);
    int it = 0;
    while (sqrt(dot_free(z, z, none, nn)) > tol * bnorm) {
        if (it == max_iter) { rc = -2; break; }
        stiffness_apply(c, d, q, NULL);
        const double alpha = rz / dot_free(d, q, none, nn);
        for (int n = 0; n < nn; ++n) {
            dP[n] += alpha * d[n];
            r[n] -= alpha * q[n];
            z[n] = r[n] / dg[n];
        }
        const double rz1 = dot_free(r, z, none, nn);
        const double beta = rz1 / rz;
        rz = rz1;
        for (int n = 0; n < nn; ++n) d[n] = z[n] + beta * d[n];
        ++it;
    }
    /* zero integral: the integral of the linear interpolant is sum_a dP_a (sum_e A_e / 3) */
    double num = 0.0, den = 0.0;
    for (int e = 0; e < c->ne; ++e) {
        const double A3 = 0.5 * c->area2[e] / 3.0;
        for (int a = 0; a < 3; ++a) { num += A3 * dP[c->tri[3 * e + a]]; den += A3; }
    }
    for (int n = 0; n < nn; ++n) dP[n] -= num / den;
    if (iters) *iters = it;
    free(b); free(r); free(z); free(d); free(q); free(dg); free(none);
    return rc;
}

/* One timestep of the coupled loop in the order of Table 1: the time step (Eq. 26, for
 * dt <= 0), the elliptic relaxation (Eq. 12, slots 14-22), the particle advance (velocity
 * prediction, Eq. 27, with the other particle equations, walls and tracking) and the
 * particle-number control, the pressure projection (Eq. 33 from the nodal means <U>* of
 * the predicted particles, two-pass as in Sect. 3.3) and the mean-velocity correction
 * (Eq. 31), then the statistics.  P[nn] (the nodal mean pressure, rho = 1) is advanced by
 * the increment, which dP[nn] returns (its value on entry is the initial guess); the
 * fields the particles provide and the pressure gradient (slots 3-4, Sect. 3.4) are then
 * derived from the new state.  Reading: the redistribution of Appendix B, which Table 1
 * does not list, follows the advance as in the particle-path step. */
int orc_coupled_step(orc_ctx *c, double dt, double Cp, double *P, double *dP, double tol,
                     int max_iter, int *wp_iters, int *p_iters)
{
    const int nn = c->nn;
    if (!(dt > 0.0)) {
        if (orc_cfl_dt(c, &dt)) return -1;
    }
    c->last_dt = dt;
    int rc = orc_update_wp(c, tol, max_iter, wp_iters);
    if (rc) return rc;
    rc = orc_advance(c, dt);
    if (rc) return rc;
    orc_redistribute(c);
    rc = orc_statistics(c);
    if (rc) return rc;
    double *ustar = (double *)malloc(sizeof(double) * 3 * nn);
    double *src = (double *)malloc(sizeof(double) * nn), *flux = (double *)malloc(sizeof(double) * nn);
    double *gp = (double *)malloc(sizeof(double) * 2 * nn);
    for (int n = 0; n < nn; ++n)
        for (int i = 0; i < 3; ++i) ustar[3 * n + i] = c->nmom[(size_t)NS * n + 1 + i];
    rc = orc_pressure_rhs(c, ustar, P, dt, Cp, src, flux);
    if (rc == 0) rc = orc_pressure_solve(c, src, flux, dP, tol, max_iter, p_iters);
    if (rc == 0) {
        orc_correct_velocity(c, dP, dt);
        rc = orc_statistics(c);
    }
    if (rc == 0) {
        for (int n = 0; n < nn; ++n) P[n] += dP[n];
        orc_derive_fields(c);
        orc_node_gradient(c, P, gp);
        for (int n = 0; n < nn; ++n) {
            c->fields[(size_t)NF * n + 3] = gp[2 * n];
            c->fields[(size_t)NF * n + 4] = gp[2 * n + 1];
        }
        orc_finish_step(c);
    }
    free(ustar); free(src); free(flux); free(gp);
    return rc;
}

/* One timestep (Table 1 order restricted to the particle path): advance and track,
 * particle-number control, then statistics and conditional means for the next step; with
 * dt <= 0 the step of Eq. 26 from the current nodal means. */
int orc_step(orc_ctx *c, double dt)
{
    if (!(dt > 0.0)) {
        if (orc_cfl_dt(c, &dt)) return -1;
    }
    c->last_dt = dt;
    int rc = orc_advance(c, dt);
    if (rc) return rc;
    orc_redistribute(c);
    rc = orc_statistics(c);
    orc_finish_step(c);
    return rc;
}

int orc_get_element_stats(const orc_ctx *c, double *out, int32_t *counts)
{
    if (out) memcpy(out, c->emom, sizeof(double) * (size_t)c->ne * NS);
    if (counts) memcpy(counts, c->count, sizeof(int32_t) * (size_t)c->ne);
    return 0;
}

int orc_get_nodal_stats(const orc_ctx *c, double *out)
{
    memcpy(out, c->nmom, sizeof(double) * (size_t)c->nn * NS);
    return 0;
}

int orc_get_bins(const orc_ctx *c, double *vcce, int32_t *g)
{
    if (vcce) memcpy(vcce, c->vcce, sizeof(double) * (size_t)c->ne * c->G);
    if (g) memcpy(g, c->gbin, sizeof(int32_t) * 3 * (size_t)c->ne);
    return 0;
}

int orc_bins_capacity(const orc_ctx *c) { return c->G; }

/* Scalar statistics of the particles of each probe element e = elems[j] (Sect. 4.1.2,
 * Figs. 12-15), with the state's conditioning pointers and conditional means:
 *   bin of psi: b = floor(psi nb) clamped to 0..nb-1 (nb equal bins of [0, 1], dpsi = 1/nb);
 *   count[j][b]  particles in bin b;
 *   phit[j][b]   Eq. 68: the mean of <phi|V> (the particle's conditional mean) over the
 *                particles of bin b (Reading: the integral over the conditional PDF is the
 *                bin average, as the paper computes it);
 *   cdiff[j][b]  t_m <Gamma lap phi | psi>: under IECM (Eq. 24) the conditional diffusion
 *                is the conditional mean of (<phi|V> - psi) / t_m; per unit 1/t_m (Reading:
 *                t_m is a local constant; the paper shows these curves normalised by the mean
 *                dissipation, where it cancels);
 *   cdiss[j][b]  t_m <2 Gamma (grad phi)^2 | psi> by Eq. 67 at the bin centre, with f~ the
 *                empirical PDF: the integral up to psi is (1/N) sum over particles below it
 *                of (psi_p - phit(psi_p)), which over whole bins is (1/N) sum (psi_p - c_p)
 *                (c_p the particle's <phi|V>, whose bin average phit is); half of bin b is
 *                counted; divided by f~ = count / (N dpsi); 0 for an empty bin;
 *   mom[j][0..5] <phi>, <phi'^2>, <phi'^3>, <phi'^4> (1/N central moments), psi_min, psi_max
 *                (zeros for an empty element).                                            */
int orc_scalar_stats(const orc_ctx *c, int n, const int32_t *elems, int nb, int32_t *count,
                     double *phit, double *cdiff, double *cdiss, double *mom)
{
    if (n < 0 || nb < 1 || !c->x) return -1;
    const double dpsi = 1.0 / nb;
    double *sc = (double *)calloc((size_t)nb, sizeof(double));
    double *sd = (double *)calloc((size_t)nb, sizeof(double));
    for (int j = 0; j < n; ++j) {
        const int e = elems[j];
        if (e < 0 || e >= c->ne) { free(sc); free(sd); return -1; }
        int32_t *cnt = count + (size_t)j * nb;
        for (int b = 0; b < nb; ++b) { cnt[b] = 0; sc[b] = 0.0; sd[b] = 0.0; }
        int N = 0;
        double s1 = 0.0, lo = 0.0, hi = 0.0;
        for (int p = 0; p < c->np; ++p) {
            if (c->elem[p] != e) continue;
            const double psi = c->psi[p];
            const double cp = c->vcce[(size_t)e * c->G + c->cp[p]];
            int b = (int)floor(psi * nb);
            if (b < 0) b = 0;
            if (b > nb - 1) b = nb - 1;
            cnt[b]++;
            sc[b] += cp;
            sd[b] += psi - cp;
            if (N == 0 || psi < lo) lo = psi;
            if (N == 0 || psi > hi) hi = psi;
            s1 += psi;
            N++;
        }
        double *m = mom + (size_t)j * 6;
        for (int k = 0; k < 6; ++k) m[k] = 0.0;
        if (N > 0) {
            const double mean = s1 / N;
            double s2 = 0.0, s3 = 0.0, s4 = 0.0;
            for (int p = 0; p < c->np; ++p) {
                if (c->elem[p] != e) continue;
                const double d = c->psi[p] - mean;
                s2 += d * d;
                s3 += d * d * d;
                s4 += d * d * d * d;
            }
            m[0] = mean; m[1] = s2 / N; m[2] = s3 / N; m[3] = s4 / N; m[4] = lo; m[5] = hi;
        }
        double cum = 0.0;
        for (int b = 0; b < nb; ++b) {
            const size_t o = (size_t)j * nb + b;
            if (cnt[b] > 0) {
                phit[o] = sc[b] / cnt[b];
                cdiff[o] = -sd[b] / cnt[b];
                cdiss[o] = -2.0 * dpsi * (cum + 0.5 * sd[b]) / cnt[b];
            } else {
                phit[o] = cdiff[o] = cdiss[o] = 0.0;
            }
            cum += sd[b];
        }
    }
    free(sc);
    free(sd);
    return 0;
}
void orc_get_diag(const orc_ctx *c, orc_diag *d) { *d = c->diag; }
void orc_reset_diag(orc_ctx *c) { memset(&c->diag, 0, sizeof(c->diag)); }
