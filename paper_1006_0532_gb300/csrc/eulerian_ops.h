// Per-node and per-element arithmetic of the coupled loop's kernels (k_eulerian.cu), as
// inline functions that compile for the device and, without CUDA, for the host.  Each
// kernel thread calls one of them; a test harness calls them in plain loops over a grid.
// FP64 throughout; T is the precision the nodal fields are stored in.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#if defined(__CUDACC__)
#define PDFX_HD __host__ __device__ __forceinline__
#else
#define PDFX_HD inline
#endif

namespace pdfx {

struct WpConst {             // constants of Eqs. 12-18 and Eq. 59
  double C1, C2, Cv, gamma5, CL, Ceta, CT, nu;
  double cxi;                // Eq. 17: 1 + 1.3 n_i n_i (2.3 with a no-slip wall, else 1)
};

namespace eops {

// Eqs. 12-18 at one node from its 32 field slots f: the right-hand side of Eq. 12 into
// rhs[c * stride] (c = 3 i + j) and the length scale of Eq. 16 into *L.  H_ijkl of Eq. 13
// is applied in contracted form,
//     H_ijkl G_kl = (C2 A_v + g5/3) G_ij - (g5/3) G_ji + g5 (b G)_ij - g5 (b G^T)_ij,
// with G_kl = d<U_k>/dx_l (zero for l = z).  Returns false when eps <= 0 (no length scale;
// *L = 0 then).
template <typename T>
PDFX_HD bool wp_rhs_node(const T* f, const WpConst& k, double* rhs, size_t stride, double* L) {
  double R[3][3];
  R[0][0] = f[23]; R[1][1] = f[24]; R[2][2] = f[25];
  R[0][1] = R[1][0] = f[26];
  R[0][2] = R[2][0] = f[27];
  R[1][2] = R[2][1] = f[28];
  double G[3][3];
  for (int i = 0; i < 3; ++i) {
    G[i][0] = f[5 + 2 * i];
    G[i][1] = f[6 + 2 * i];
    G[i][2] = 0.0;
  }
  const double om = f[29];
  const double tr = R[0][0] + R[1][1] + R[2][2];
  const double kk = 0.5 * tr;
  double b[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) b[i][j] = tr > 0.0 ? R[i][j] / tr - (i == j ? 1.0 / 3.0 : 0.0) : 0.0;
  const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                     R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                     R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
  const double k23 = 2.0 * kk / 3.0;
  const double Av = kk > 0.0 ? fmin(1.0, k.Cv * det / (k23 * k23 * k23)) : 0.0;   // Eq. 14
  const double c1 = k.C2 * Av + k.gamma5 / 3.0, c2 = k.gamma5 / 3.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      double bG = 0.0, bGt = 0.0;
      for (int m = 0; m < 3; ++m) {
        bG += b[i][m] * G[m][j];
        bGt += b[i][m] * G[j][m];
      }
      const double h = c1 * G[i][j] - c2 * G[j][i] + k.gamma5 * (bG - bGt);
      rhs[static_cast<size_t>(3 * i + j) * stride] = (i == j ? 0.5 * (1.0 - k.C1) * kk * om : 0.0) + kk * h;
    }
  }
  const double eps = om * (kk + k.nu * k.CT * k.CT * om);   // Eq. 18
  if (!(eps > 0.0)) {
    *L = 0.0;
    return false;
  }
  const double lt = k.cxi * kk * sqrt(kk) / eps;
  const double lk = k.Ceta * sqrt(sqrt(k.nu * k.nu * k.nu / eps));
  *L = k.CL * fmax(lt, lk);                                   // Eq. 16
  return true;
}

// Dirichlet conditions of the nine components at one node of class cls (1 no-slip with
// outward unit normal (nx, ny), 2 free-slip): Eq. 59's -4.5 eps n_i n_j, or zero for the
// off-diagonal components at a free-slip node.  x[c * stride] holds the initial guess and
// is overwritten where the component is fixed.  Returns false when a no-slip node has
// eps <= 0.
template <typename T>
PDFX_HD bool wp_bc_node(const T* f, const WpConst& k, int cls, double nx, double ny, uint8_t* fixed,
                        double* x, size_t stride) {
  double eps = 0.0;
  bool ok = true;
  if (cls == 1) {
    const double kk = 0.5 * (static_cast<double>(f[23]) + f[24] + f[25]);
    const double om = f[29];
    eps = om * (kk + k.nu * k.CT * k.CT * om);
    ok = eps > 0.0;
  }
  const double nv[3] = {nx, ny, 0.0};
  for (int c = 0; c < 9; ++c) {
    const int i = c / 3, j = c % 3;
    const size_t o = static_cast<size_t>(c) * stride;
    if (cls == 1) {
      x[o] = -4.5 * eps * nv[i] * nv[j];   // Eq. 59
      fixed[o] = 1;
    } else if (cls == 2 && i != j) {
      x[o] = 0.0;
      fixed[o] = 1;
    } else {
      fixed[o] = 0;
    }
  }
  return ok;
}

// One CSR entry of M + L_e^2 K from its element contributions clist[jb, je) (codes
// 9 e + 3 a + b); fe[e][7] holds Eq. 40's derivatives and the area; L_e^2 is the mean of
// the element's nodal L^2.
PDFX_HD double wp_entry(int jb, int je, const int32_t* clist, const double* fe, const int32_t* tri,
                        const double* L) {
  double s = 0.0;
  for (int j = jb; j < je; ++j) {
    const int cc = clist[j];
    const int e = cc / 9, a = (cc % 9) / 3, b = cc % 3;
    const double* g = fe + 7 * static_cast<size_t>(e);
    const int32_t* t = tri + 3 * static_cast<size_t>(e);
    const double l0 = L[t[0]], l1 = L[t[1]], l2 = L[t[2]];
    const double L2 = (l0 * l0 + l1 * l1 + l2 * l2) / 3.0;
    const double A = g[6];
    s += A / 12.0 * (a == b ? 2.0 : 1.0) + L2 * A * (g[a] * g[b] + g[3 + a] * g[3 + b]);
  }
  return s;
}

// Row n of a CSR matrix times x.
PDFX_HD double csr_row(int n, const int32_t* row, const int32_t* col, const double* val, const double* x) {
  double s = 0.0;
  for (int k = row[n]; k < row[n + 1]; ++k) s += val[k] * x[col[k]];
  return s;
}

// Element gradient (Eq. 39 with Eq. 40's derivatives) of the nodal quantity q at element e.
PDFX_HD void elem_gradient(int e, const double* fe, const int32_t* tri, const double* q, double* gx, double* gy) {
  const double* g = fe + 7 * static_cast<size_t>(e);
  const int32_t* t = tri + 3 * static_cast<size_t>(e);
  const double v0 = q[t[0]], v1 = q[t[1]], v2 = q[t[2]];
  *gx = g[0] * v0 + g[1] * v1 + g[2] * v2;
  *gy = g[3] * v0 + g[4] * v1 + g[5] * v2;
}

// Node transfer (Sect. 3.4): the mean of eg[e][2] over the elements around node n.
PDFX_HD void node_mean(int n, const int32_t* ne_off, const int32_t* ne_list, const double* eg, double* gx, double* gy) {
  double sx = 0.0, sy = 0.0;
  const int m = ne_off[n + 1] - ne_off[n];
  for (int k = ne_off[n]; k < ne_off[n + 1]; ++k) {
    const int e = ne_list[k];
    sx += eg[2 * e];
    sy += eg[2 * e + 1];
  }
  *gx = m > 0 ? sx / m : 0.0;
  *gy = m > 0 ? sy / m : 0.0;
}

// Eq. 33's source at one node, (div <U>* - C_p lap P) / dt with rho = 1, from the node's
// gradients of <U>* and <V>* and its two-pass laplacian of P; and at a no-slip node (cls 1,
// outward normal (nx, ny)) the increment's normal derivative: Eq. 61's value from the
// node's fields (laplacian slots 11-12) and gradients of <uu>, <vv>, <uv>, minus n . grad P.
template <typename T>
PDFX_HD void pressure_node(const double* gu, const double* gv, const double* gp, const double* guu,
                           const double* gvv, const double* guv, double lapP, const T* f, int cls, double nx,
                           double ny, double nu, double dt, double Cp, double* src, double* flux) {
  *src = (gu[0] + gv[1] - Cp * lapP) / dt;
  double fl = 0.0;
  if (cls == 1) {
    const double divx = guu[0] + guv[1];
    const double divy = guv[0] + gvv[1];
    const double eq61 = nu * (static_cast<double>(f[11]) * nx + static_cast<double>(f[12]) * ny) -
                        (divx * nx + divy * ny);
    fl = eq61 - (gp[0] * nx + gp[1] * ny);
  }
  *flux = fl;
}

// The Galerkin load of Eq. 33 at node n: -M src plus the no-slip edge integrals of the
// normal derivative (linear along each edge).
PDFX_HD double pressure_load_node(int n, const int32_t* row, const int32_t* col, const double* mval,
                                  const double* src, const double* flux, const int32_t* boff,
                                  const int32_t* bnb, const double* blen) {
  const double s = csr_row(n, row, col, mval, src);
  double e = 0.0;
  for (int k = boff[n]; k < boff[n + 1]; ++k) e += blen[k] / 6.0 * (2.0 * flux[n] + flux[bnb[k]]);
  return e - s;
}

// Conjugate gradients with the Jacobi preconditioner over C systems (Sect. 3.2): the work
// of one free or fixed node per pass, and the scalars of one component.  Scalars of a
// component: s[kPcgScalars] = rz, |b|, zz, alpha, beta, active, iterations.
constexpr int kPcgScalars = 8;
enum { S_RZ = 0, S_BNORM = 1, S_ZZ = 2, S_ALPHA = 3, S_BETA = 4, S_ACTIVE = 5, S_ITERS = 6 };

// One node of a pass (fr: the node is free for this component; q holds A times the vector
// the pass needs).  mode 0: the preconditioned reduced load, sums zb^2; mode 1: initial
// residual r = b - q, z = r / diag, d = z, sums r z and z z; mode 2: q masked, sums d q;
// mode 3: x += alpha d, r -= alpha q, z = r / diag, sums r z and z z.
PDFX_HD void pcg_node(int mode, bool fr, double diag, double alpha, const double* b, double* x, double* r,
                      double* z, double* d, double* q, double* s0, double* s1) {
  if (mode == 0) {
    const double zb = fr ? (*b - *q) / diag : 0.0;
    *s0 += zb * zb;
  } else if (mode == 1) {
    const double rr = fr ? *b - *q : 0.0;
    const double zz = fr ? rr / diag : 0.0;
    *r = rr;
    *z = zz;
    *d = zz;
    *s0 += rr * zz;
    *s1 += zz * zz;
  } else if (mode == 2) {
    const double qq = fr ? *q : 0.0;
    *q = qq;
    *s0 += *d * qq;
  } else {
    if (fr) {
      *x += alpha * *d;
      *r -= alpha * *q;
    }
    const double zz = fr ? *r / diag : 0.0;
    *z = zz;
    *s0 += *r * zz;
    *s1 += zz * zz;
  }
}

// The scalars of one component from a pass's sums t0, t1.  step 0: |b|; step 1: rz, zz,
// the stopping test, iterations = 0; step 2: alpha (0 once converged); step 3: beta, rz, zz,
// iterations + 1 and the stopping test, for a component still iterating.
PDFX_HD void pcg_scalars(int step, double t0, double t1, double tol, double* s) {
  if (step == 0) {
    s[S_BNORM] = sqrt(t0);
  } else if (step == 1) {
    s[S_RZ] = t0;
    s[S_ZZ] = t1;
    s[S_ITERS] = 0.0;
    s[S_ACTIVE] = sqrt(t1) > tol * s[S_BNORM] ? 1.0 : 0.0;
    s[S_ALPHA] = 0.0;
    s[S_BETA] = 0.0;
  } else if (step == 2) {
    s[S_ALPHA] = s[S_ACTIVE] != 0.0 ? s[S_RZ] / t0 : 0.0;
  } else {
    if (s[S_ACTIVE] != 0.0) {
      s[S_BETA] = t0 / s[S_RZ];
      s[S_RZ] = t0;
      s[S_ZZ] = t1;
      s[S_ITERS] += 1.0;
      s[S_ACTIVE] = sqrt(t1) > tol * s[S_BNORM] ? 1.0 : 0.0;
    } else {
      s[S_BETA] = 0.0;
    }
  }
}

// The new direction d = z + beta d of a free node of a component still iterating.
PDFX_HD void pcg_direction(bool fr, const double* s, double z, double* d) {
  if (s[S_ACTIVE] == 0.0) return;
  *d = fr ? z + s[S_BETA] * *d : 0.0;
}

// A component with a zero reduced load has the zero solution on its free nodes.
PDFX_HD void pcg_trivial(bool fr, const double* s, double* x) {
  if (s[S_BNORM] == 0.0 && fr) *x = 0.0;
}

}  // namespace eops
}  // namespace pdfx
