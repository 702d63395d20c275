// Eulerian solves of the coupled loop (Sect. 3.2), FP64 throughout.  The per-node and
// per-element arithmetic lives in eulerian_ops.h; these kernels map threads onto it and
// carry the reductions.
//
// * The local right-hand side of the elliptic relaxation and its length scale (Eqs. 12-18),
//   one thread per node.  H_ijkl of Eq. 13 is applied in contracted form:
//       H_ijkl G_kl = (C2 A_v + g5/3) G_ij - (g5/3) G_ji + g5 (b G)_ij - g5 (b G^T)_ij
//   with G_kl = d<U_k>/dx_l (zero for l = z).
// * Galerkin matrices of linear triangles in CSR.  Fixed matrices (consistent mass,
//   laplacian stiffness) come from the host.  The elliptic-relaxation matrix M + L_e^2 K
//   changes with L every call, so each CSR entry sums its element contributions in
//   ascending element order.
// * Conjugate gradients with the Jacobi preconditioner for C right-hand sides at once
//   (vectors [C][nn]), with per-component Dirichlet masks.  Every reduction is two-stage:
//   block partials, then one block per component summing them in a fixed order.  Results
//   therefore repeat bit for bit.
// * The pressure projection's source (Eq. 33), the increment's normal derivative (Eq. 61),
//   node-transferred gradients (Sect. 3.4) and the Galerkin load.
#include "pdfx_device.cuh"
#include "pdfx_internal.h"

namespace pdfx {
namespace {

constexpr int kEB = 256;   // threads per block
constexpr int kRowChunk = 8;   // CSR entries whose loads a row issues together

unsigned blocks_for(int64_t n) { return static_cast<unsigned>((n + kEB - 1) / kEB); }

// Sum of v over the block's threads (kEB threads); the result is valid in thread 0.
__device__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int w = kEB / 2; w > 0; w >>= 1) {
    if (t < w) sh[t] += sh[t + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void wp_rhs_kernel(const T* __restrict__ f, int nn, WpConst k, double* __restrict__ rhs,
                              double* __restrict__ L, int* __restrict__ err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  if (!eops::wp_rhs_node(f + static_cast<size_t>(n) * kNF, k, rhs + n, static_cast<size_t>(nn), L + n))
    atomicExch(err, 1);
}

// The fields' wp_ij (slots 14-22) as the initial guess x[9][nn].
template <typename T>
__global__ void read_wp_kernel(int nn, const T* __restrict__ f, double* __restrict__ x) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  for (int c = 0; c < 9; ++c) x[static_cast<size_t>(c) * nn + n] = f[static_cast<size_t>(n) * kNF + 14 + c];
}

// Dirichlet conditions of the nine components (Eq. 59 at no-slip nodes, zero off-diagonal
// components at free-slip nodes) written into x[9][nn], which holds the initial guess.
template <typename T>
__global__ void wp_bc_kernel(const T* __restrict__ f, int nn, WpConst k, const int8_t* __restrict__ ncls,
                             const double* __restrict__ nrm, uint8_t* __restrict__ fixed,
                             double* __restrict__ x, int* __restrict__ err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  if (!eops::wp_bc_node(f + static_cast<size_t>(n) * kNF, k, ncls[n], nrm[2 * n], nrm[2 * n + 1], fixed + n,
                        x + n, static_cast<size_t>(nn)))
    atomicExch(err, 1);
}

__global__ void assemble_wp_kernel(int nnz, const int32_t* __restrict__ cptr, const int32_t* __restrict__ clist,
                                   const double* __restrict__ fe, const int32_t* __restrict__ tri,
                                   const double* __restrict__ L, double* __restrict__ aval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnz) return;
  aval[i] = eops::wp_entry(cptr[i], cptr[i + 1], clist, fe, tri, L);
}

// y[c][n] = sum_k val[k] x[c][col[k]] over row n, for C components.
__global__ void spmv_kernel(int nn, int C, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ x,
                            double* __restrict__ y) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(nn) * C) return;
  const int c = static_cast<int>(i / nn), n = static_cast<int>(i % nn);
  y[i] = eops::csr_row(n, row, col, val, x + static_cast<size_t>(c) * nn);
}

// Scalars of component c: sc[c * kSc + .].
constexpr int kSc = kPcgScalars;
using eops::S_ALPHA;

// Sums over nodes of the block's slice: grid (nblk, C); part[(c * nblk + blk) * 2 + m].
// mode 0: zb = free ? (b - q) / diag : 0, sums zb^2 (the reduced load's norm)
// mode 1: r = free ? b - q : 0, z = r / diag, d = z, sums r z and z z (initial residual)
// mode 2: q = free ? q : 0, sums d q
// mode 3: x += alpha d, r -= alpha q, z = free ? r / diag : 0, sums r z and z z
__global__ void pcg_pass_kernel(int mode, int nn, const uint8_t* __restrict__ fixed, const double* __restrict__ diag,
                                const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r,
                                double* __restrict__ z, double* __restrict__ d, double* __restrict__ q,
                                const double* __restrict__ sc, double* __restrict__ part) {
  __shared__ double sh[kEB];
  const int c = blockIdx.y, nblk = gridDim.x;
  const size_t base = static_cast<size_t>(c) * nn;
  const double alpha = sc[c * kSc + S_ALPHA];
  double s0 = 0.0, s1 = 0.0;
  for (int n = blockIdx.x * kEB + threadIdx.x; n < nn; n += nblk * kEB) {
    const size_t o = base + n;
    const bool fr = !fixed || !fixed[o];
    eops::pcg_node(mode, fr, diag[n], alpha, b + o, x + o, r + o, z + o, d + o, q + o, &s0, &s1);
  }
  const double t0 = block_sum(s0, sh);
  const double t1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[(static_cast<size_t>(c) * nblk + blockIdx.x) * 2] = t0;
    part[(static_cast<size_t>(c) * nblk + blockIdx.x) * 2 + 1] = t1;
  }
}

// One block per component: the partial sums in block order, then the scalars.
// step 0: bnorm; step 1: rz, zz, active, iters = 0; step 2: alpha; step 3: beta, rz, zz,
// iters, active.
__global__ void pcg_scalar_kernel(int step, int nblk, const double* __restrict__ part, double tol,
                                  double* __restrict__ sc) {
  __shared__ double sh[kEB];
  const int c = blockIdx.x;
  double a0 = 0.0, a1 = 0.0;
  for (int j = threadIdx.x; j < nblk; j += kEB) {
    a0 += part[(static_cast<size_t>(c) * nblk + j) * 2];
    a1 += part[(static_cast<size_t>(c) * nblk + j) * 2 + 1];
  }
  const double t0 = block_sum(a0, sh);
  const double t1 = block_sum(a1, sh);
  if (threadIdx.x == 0) eops::pcg_scalars(step, t0, t1, tol, sc + c * kSc);
}

// d = free ? z + beta d : 0 for the components still iterating.
__global__ void pcg_direction_kernel(int nn, int C, const uint8_t* __restrict__ fixed, const double* __restrict__ z,
                                     double* __restrict__ d, const double* __restrict__ sc) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(nn) * C) return;
  const int c = static_cast<int>(i / nn);
  eops::pcg_direction(!fixed || !fixed[i], sc + c * kSc, z[i], d + i);
}

// ---------------------------------------------------------------------------------------
// Two kernels per conjugate-gradient iteration.  Each ends with a block sum per block and,
// in the last block of a component to finish (an atomic ticket after a memory fence), the
// component's scalars from the blocks' partial sums in block order: the sums and scalars
// of the three-kernel passes above, bit for bit.
//   direction_spmv: d1 = the new direction (z + beta d0 on free nodes of a component still
//     iterating; d0 otherwise), q = A d1 masked to the free nodes, sums d1 q; then alpha.
//     A row needs the new direction at its neighbours: it forms z + beta d0 there itself, so
//     the old direction d0 stays untouched and d1 is a second buffer.
//   update: x += alpha d1, r -= alpha q, z = r / diag, sums r z and z z; then beta, the
//     stopping test, the iteration count.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double new_direction(bool fr, const double* sc, double z, double d0) {
  double d = d0;
  eops::pcg_direction(fr, sc, z, &d);
  return d;
}

// The last block of component c (grid.x blocks) to arrive returns true, after a fence that
// makes the other blocks' partial sums visible; it resets the ticket for the next use.
__device__ __forceinline__ bool last_block(unsigned* ticket, int c) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned k = atomicAdd(ticket + c, 1u);
    last = k == gridDim.x - 1;
    if (last) ticket[c] = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sums the component's partials part[(c nblk + j) 2 + m] over j in the order of the scalar
// kernel and applies scalar step `step` (called by a whole block).
__device__ __forceinline__ void finish_scalars(int step, int c, int nblk, const double* part, double tol,
                                               double* sc, double* sh) {
  double a0 = 0.0, a1 = 0.0;
  for (int j = threadIdx.x; j < nblk; j += kEB) {   // other blocks' sums: read past the L1
    a0 += __ldcg(part + (static_cast<size_t>(c) * nblk + j) * 2);
    a1 += __ldcg(part + (static_cast<size_t>(c) * nblk + j) * 2 + 1);
  }
  const double t0 = block_sum(a0, sh);
  const double t1 = block_sum(a1, sh);
  if (threadIdx.x == 0) eops::pcg_scalars(step, t0, t1, tol, sc + c * kSc);
}

__global__ void pcg_direction_spmv_kernel(int nn, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                          const double* __restrict__ val, const uint8_t* __restrict__ fixed,
                                          const double* __restrict__ z, const double* __restrict__ d0,
                                          double* __restrict__ d1, double* __restrict__ q, double tol,
                                          double* __restrict__ sc, double* __restrict__ part,
                                          unsigned* __restrict__ ticket) {
  __shared__ double sh[kEB];
  const int c = blockIdx.y, nblk = gridDim.x;
  const size_t base = static_cast<size_t>(c) * nn;
  const double* scc = sc + c * kSc;
  double s0 = 0.0;
  for (int n = blockIdx.x * kEB + threadIdx.x; n < nn; n += nblk * kEB) {
    // the row in chunks of kRowChunk entries: every load of a chunk is issued before the
    // first product, so that a row costs a few memory round trips instead of two per entry;
    // the products are summed in entry order, as in the loop they replace
    double acc = 0.0;
    const int r0 = row[n], r1 = row[n + 1];
#pragma unroll 1
    for (int k0 = r0; k0 < r1; k0 += kRowChunk) {
      int32_t cj[kRowChunk];
      double vk[kRowChunk];
#pragma unroll
      for (int u = 0; u < kRowChunk; ++u) {
        const bool in = k0 + u < r1;
        cj[u] = in ? col[k0 + u] : 0;
        vk[u] = in ? val[k0 + u] : 0.0;
      }
      double zj[kRowChunk], dj[kRowChunk];
      bool fj[kRowChunk];
#pragma unroll
      for (int u = 0; u < kRowChunk; ++u) {
        const size_t oj = base + cj[u];
        fj[u] = !fixed || !fixed[oj];
        zj[u] = z[oj];
        dj[u] = d0[oj];
      }
#pragma unroll
      for (int u = 0; u < kRowChunk; ++u)
        if (k0 + u < r1) acc += vk[u] * new_direction(fj[u], scc, zj[u], dj[u]);
    }
    const size_t o = base + n;
    const bool fr = !fixed || !fixed[o];
    const double dn = new_direction(fr, scc, z[o], d0[o]);
    double qn = acc, dummy = 0.0;
    d1[o] = dn;
    eops::pcg_node(2, fr, 1.0, 0.0, nullptr, nullptr, nullptr, nullptr, &d1[o], &qn, &s0, &dummy);
    q[o] = qn;
  }
  const double t0 = block_sum(s0, sh);
  if (threadIdx.x == 0) {
    part[(static_cast<size_t>(c) * nblk + blockIdx.x) * 2] = t0;
    part[(static_cast<size_t>(c) * nblk + blockIdx.x) * 2 + 1] = 0.0;
  }
  if (last_block(ticket, c)) finish_scalars(2, c, nblk, part, tol, sc, sh);
}

__global__ void pcg_update_kernel(int nn, const uint8_t* __restrict__ fixed, const double* __restrict__ diag,
                                  double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                                  double* __restrict__ d1, double* __restrict__ q, double tol,
                                  double* __restrict__ sc, double* __restrict__ part, unsigned* __restrict__ ticket) {
  __shared__ double sh[kEB];
  const int c = blockIdx.y, nblk = gridDim.x;
  const size_t base = static_cast<size_t>(c) * nn;
  const double alpha = sc[c * kSc + S_ALPHA];
  double s0 = 0.0, s1 = 0.0;
  for (int n = blockIdx.x * kEB + threadIdx.x; n < nn; n += nblk * kEB) {
    const size_t o = base + n;
    const bool fr = !fixed || !fixed[o];
    eops::pcg_node(3, fr, diag[n], alpha, nullptr, x + o, r + o, z + o, d1 + o, q + o, &s0, &s1);
  }
  const double t0 = block_sum(s0, sh);
  const double t1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[(static_cast<size_t>(c) * nblk + blockIdx.x) * 2] = t0;
    part[(static_cast<size_t>(c) * nblk + blockIdx.x) * 2 + 1] = t1;
  }
  if (last_block(ticket, c)) finish_scalars(3, c, nblk, part, tol, sc, sh);
}

// xD = fixed ? x : 0 (the Dirichlet columns of the reduced load).
__global__ void dirichlet_part_kernel(int64_t n, const uint8_t* __restrict__ fixed, const double* __restrict__ x,
                                      double* __restrict__ xd) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  xd[i] = (fixed && fixed[i]) ? x[i] : 0.0;
}

// A component whose reduced load is zero has the zero solution on its free nodes.
__global__ void trivial_kernel(int nn, int C, const uint8_t* __restrict__ fixed, const double* __restrict__ sc,
                               double* __restrict__ x) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(nn) * C) return;
  const int c = static_cast<int>(i / nn);
  eops::pcg_trivial(!(fixed && fixed[i]), sc + c * kSc, x + i);
}

// Element gradients (Eq. 39 with Eq. 40's derivatives) of nq nodal quantities q[nq][nn]:
// eg[nq][ne][2].
__global__ void egrad_kernel(int ne, int nn, int nq, const double* __restrict__ fe, const int32_t* __restrict__ tri,
                             const double* __restrict__ q, double* __restrict__ eg) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(ne) * nq) return;
  const int j = static_cast<int>(i / ne), e = static_cast<int>(i % ne);
  eops::elem_gradient(e, fe, tri, q + static_cast<size_t>(j) * nn, &eg[2 * i], &eg[2 * i + 1]);
}

// Node transfer (Sect. 3.4): the mean over the elements around each node: gn[nq][nn][2].
__global__ void nmean_kernel(int nn, int ne, int nq, const int32_t* __restrict__ ne_off,
                             const int32_t* __restrict__ ne_list, const double* __restrict__ eg,
                             double* __restrict__ gn) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(nn) * nq) return;
  const int j = static_cast<int>(i / nn), n = static_cast<int>(i % nn);
  eops::node_mean(n, ne_off, ne_list, eg + 2 * static_cast<size_t>(j) * ne, &gn[2 * i], &gn[2 * i + 1]);
}

// Inputs of the first derivative pass: <U>*, <V>* (from nmom or a caller's [nn][3]), P and
// <uu>, <vv>, <uv> from the fields: q6[6][nn].
template <typename T>
__global__ void pressure_inputs_kernel(int nn, const double* __restrict__ ustar, int ustride, int uoff,
                                       const double* __restrict__ P, const T* __restrict__ f,
                                       double* __restrict__ q6) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const T* fn = f + static_cast<size_t>(n) * kNF;
  q6[n] = ustar[static_cast<size_t>(n) * ustride + uoff];
  q6[static_cast<size_t>(nn) + n] = ustar[static_cast<size_t>(n) * ustride + uoff + 1];
  q6[2 * static_cast<size_t>(nn) + n] = P[n];
  q6[3 * static_cast<size_t>(nn) + n] = fn[23];
  q6[4 * static_cast<size_t>(nn) + n] = fn[24];
  q6[5 * static_cast<size_t>(nn) + n] = fn[26];
}

__global__ void second_inputs_kernel(int nn, const double* __restrict__ g6, double* __restrict__ q2) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const double* gp = g6 + 2 * (2 * static_cast<size_t>(nn));   // gradient of P
  q2[n] = gp[2 * n];
  q2[static_cast<size_t>(nn) + n] = gp[2 * n + 1];
}

// Eq. 33's source and the increment's outward normal derivative at no-slip nodes (Eq. 61
// from the fields minus n . grad P).
template <typename T>
__global__ void pressure_src_kernel(int nn, const double* __restrict__ g6, const double* __restrict__ g2,
                                    const T* __restrict__ f, const int8_t* __restrict__ ncls,
                                    const double* __restrict__ nrm, double nu, double dt, double Cp,
                                    double* __restrict__ src, double* __restrict__ flux) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const size_t N2 = 2 * static_cast<size_t>(nn);
  const double lapP = g2[2 * n] + g2[N2 + 2 * n + 1];
  eops::pressure_node(g6 + 2 * n, g6 + N2 + 2 * n, g6 + 2 * N2 + 2 * n, g6 + 3 * N2 + 2 * n,
                      g6 + 4 * N2 + 2 * n, g6 + 5 * N2 + 2 * n, lapP, f + static_cast<size_t>(n) * kNF, ncls[n],
                      nrm[2 * n], nrm[2 * n + 1], nu, dt, Cp, &src[n], &flux[n]);
}

// Galerkin load of Eq. 33: b = -M src + the no-slip edge integrals of the normal derivative.
__global__ void pressure_load_kernel(int nn, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                     const double* __restrict__ mval, const double* __restrict__ src,
                                     const double* __restrict__ flux, const int32_t* __restrict__ boff,
                                     const int32_t* __restrict__ bnb, const double* __restrict__ blen,
                                     double* __restrict__ b) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  b[n] = eops::pressure_load_node(n, row, col, mval, src, flux, boff, bnb, blen);
}

// v -= sum[0] / div (a sum the dot kernels left in device memory).
__global__ void sub_mean_kernel(int nn, const double* __restrict__ sum, double div, double* __restrict__ v) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  v[n] -= sum[0] / div;
}

// part[blk] = sum over the block's slice of w[n] v[n] (w = NULL: 1).
__global__ void dot_part_kernel(int nn, const double* __restrict__ w, const double* __restrict__ v,
                                double* __restrict__ part) {
  __shared__ double sh[kEB];
  double s = 0.0;
  for (int n = blockIdx.x * kEB + threadIdx.x; n < nn; n += gridDim.x * kEB) s += (w ? w[n] : 1.0) * v[n];
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void dot_finish_kernel(int nblk, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[kEB];
  double s = 0.0;
  for (int j = threadIdx.x; j < nblk; j += kEB) s += part[j];
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = t;
}

template <typename T>
__global__ void write_wp_kernel(int nn, const double* __restrict__ x, T* __restrict__ f) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  for (int c = 0; c < 9; ++c) f[static_cast<size_t>(n) * kNF + 14 + c] = static_cast<T>(x[static_cast<size_t>(c) * nn + n]);
}

template <typename T>
__global__ void write_pgrad_kernel(int nn, const double* __restrict__ gp, T* __restrict__ f) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  f[static_cast<size_t>(n) * kNF + 3] = static_cast<T>(gp[2 * n]);
  f[static_cast<size_t>(n) * kNF + 4] = static_cast<T>(gp[2 * n + 1]);
}

__global__ void diag_kernel(int nn, const int32_t* __restrict__ dpos, const double* __restrict__ val,
                            double* __restrict__ diag) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nn) diag[n] = val[dpos[n]];
}

__global__ void add_kernel(int nn, const double* __restrict__ a, double* __restrict__ b) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nn) b[n] += a[n];
}

}  // namespace

// Blocks of the reduction passes: one node per thread up to kRedBlocks blocks (the passes
// are latency-bound at these sizes, so every SM should take part).
int pcg_blocks(int nn) {
  const int nb = static_cast<int>(blocks_for(nn));
  return nb < kRedBlocks ? nb : kRedBlocks;
}

size_t pcg_scratch_doubles(int nn, int C) {
  return static_cast<size_t>(C) * (2 * static_cast<size_t>(pcg_blocks(nn)) + kSc);
}

template <typename T>
void launch_wp_rhs(const T* fields, int nn, const WpConst& k, double* rhs, double* L, int* err, cudaStream_t s) {
  wp_rhs_kernel<T><<<blocks_for(nn), kEB, 0, s>>>(fields, nn, k, rhs, L, err);
}

template <typename T>
void launch_wp_bc(const T* fields, int nn, const WpConst& k, const int8_t* ncls, const double* nrm,
                  uint8_t* fixed, double* x, int* err, cudaStream_t s) {
  wp_bc_kernel<T><<<blocks_for(nn), kEB, 0, s>>>(fields, nn, k, ncls, nrm, fixed, x, err);
}

template <typename T>
void launch_read_wp(int nn, const T* fields, double* x, cudaStream_t s) {
  read_wp_kernel<T><<<blocks_for(nn), kEB, 0, s>>>(nn, fields, x);
}

// The elliptic-relaxation matrix M + L_e^2 K into aval[nnz] and its diagonal into adiag[nn].
void launch_assemble_wp(const FemDev& m, const double* L, double* aval, double* adiag, cudaStream_t s) {
  assemble_wp_kernel<<<blocks_for(m.nnz), kEB, 0, s>>>(m.nnz, m.cptr, m.clist, m.fe, m.tri, L, aval);
  diag_kernel<<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, m.dpos, aval, adiag);
}

void launch_spmv(const FemDev& m, const double* val, int C, const double* x, double* y, cudaStream_t s) {
  spmv_kernel<<<blocks_for(static_cast<int64_t>(m.nn) * C), kEB, 0, s>>>(m.nn, C, m.row, m.col, val, x, y);
}

// Jacobi-PCG setup for C systems sharing one matrix: the reduced load's norm, the zero
// solution of components with a zero reduced load, the initial residual and direction.
void launch_pcg_setup(const FemDev& m, const PcgArgs& a, cudaStream_t s) {
  const int nn = m.nn, C = a.C, nblk = pcg_blocks(nn);
  const int64_t n = static_cast<int64_t>(nn) * C;
  double* part = a.scratch;
  double* sc = a.scratch + 2 * static_cast<size_t>(C) * nblk;
  const dim3 grid(static_cast<unsigned>(nblk), static_cast<unsigned>(C));
  dirichlet_part_kernel<<<blocks_for(n), kEB, 0, s>>>(n, a.fixed, a.x, a.d);
  spmv_kernel<<<blocks_for(n), kEB, 0, s>>>(nn, C, m.row, m.col, a.val, a.d, a.q);
  pcg_pass_kernel<<<grid, kEB, 0, s>>>(0, nn, a.fixed, a.diag, a.b, a.x, a.r, a.z, a.d, a.q, sc, part);
  pcg_scalar_kernel<<<C, kEB, 0, s>>>(0, nblk, part, a.tol, sc);
  trivial_kernel<<<blocks_for(n), kEB, 0, s>>>(nn, C, a.fixed, sc, a.x);
  spmv_kernel<<<blocks_for(n), kEB, 0, s>>>(nn, C, m.row, m.col, a.val, a.x, a.q);
  pcg_pass_kernel<<<grid, kEB, 0, s>>>(1, nn, a.fixed, a.diag, a.b, a.x, a.r, a.z, a.d, a.q, sc, part);
  pcg_scalar_kernel<<<C, kEB, 0, s>>>(1, nblk, part, a.tol, sc);
}

// One conjugate-gradient iteration of every component still iterating.
void launch_pcg_iteration(const FemDev& m, const PcgArgs& a, cudaStream_t s) {
  const int nn = m.nn, C = a.C, nblk = pcg_blocks(nn);
  const int64_t n = static_cast<int64_t>(nn) * C;
  double* part = a.scratch;
  double* sc = a.scratch + 2 * static_cast<size_t>(C) * nblk;
  const dim3 grid(static_cast<unsigned>(nblk), static_cast<unsigned>(C));
  spmv_kernel<<<blocks_for(n), kEB, 0, s>>>(nn, C, m.row, m.col, a.val, a.d, a.q);
  pcg_pass_kernel<<<grid, kEB, 0, s>>>(2, nn, a.fixed, a.diag, a.b, a.x, a.r, a.z, a.d, a.q, sc, part);
  pcg_scalar_kernel<<<C, kEB, 0, s>>>(2, nblk, part, a.tol, sc);
  pcg_pass_kernel<<<grid, kEB, 0, s>>>(3, nn, a.fixed, a.diag, a.b, a.x, a.r, a.z, a.d, a.q, sc, part);
  pcg_scalar_kernel<<<C, kEB, 0, s>>>(3, nblk, part, a.tol, sc);
  pcg_direction_kernel<<<blocks_for(n), kEB, 0, s>>>(nn, C, a.fixed, a.z, a.d, sc);
}

const double* pcg_scalars(const PcgArgs& a, int nn) {
  return a.scratch + 2 * static_cast<size_t>(a.C) * pcg_blocks(nn);
}

// Two iterations of every component still iterating, in two kernels each; the direction
// alternates between a.d and a.q2 (a second direction buffer), so that after an even number
// of iterations it is back in a.d.  a.ticket: C zeroed counters.
void launch_pcg_two_iterations(const FemDev& m, const PcgArgs& a, cudaStream_t s) {
  const int nn = m.nn, C = a.C, nblk = pcg_blocks(nn);
  double* part = a.scratch;
  double* sc = a.scratch + 2 * static_cast<size_t>(C) * nblk;
  const dim3 grid(static_cast<unsigned>(nblk), static_cast<unsigned>(C));
  double* dirs[2] = {a.d, a.d2};
  for (int it = 0; it < 2; ++it) {
    pcg_direction_spmv_kernel<<<grid, kEB, 0, s>>>(nn, m.row, m.col, a.val, a.fixed, a.z, dirs[it],
                                                   dirs[1 - it], a.q, a.tol, sc, part, a.ticket);
    pcg_update_kernel<<<grid, kEB, 0, s>>>(nn, a.fixed, a.diag, a.x, a.r, a.z, dirs[1 - it], a.q, a.tol,
                                           sc, part, a.ticket);
  }
}

// Node-transferred gradients (Sect. 3.4) of nq quantities q[nq][nn] into gn[nq][nn][2];
// eg is scratch of 2 nq ne doubles.
void launch_node_gradients(const FemDev& m, const int32_t* ne_off, const int32_t* ne_list, int nq,
                           const double* q, double* eg, double* gn, cudaStream_t s) {
  egrad_kernel<<<blocks_for(static_cast<int64_t>(m.ne) * nq), kEB, 0, s>>>(m.ne, m.nn, nq, m.fe, m.tri, q, eg);
  nmean_kernel<<<blocks_for(static_cast<int64_t>(m.nn) * nq), kEB, 0, s>>>(m.nn, m.ne, nq, ne_off, ne_list, eg, gn);
}

template <typename T>
void launch_pressure_rhs(const FemDev& m, const int32_t* ne_off, const int32_t* ne_list, const double* ustar,
                         int ustride, int uoff, const double* P, const T* fields, double nu, double dt,
                         double Cp, double* work, double* src, double* flux, cudaStream_t s) {
  const size_t nn = static_cast<size_t>(m.nn), ne = static_cast<size_t>(m.ne);
  double* q6 = work;                 // 6 nn
  double* g6 = q6 + 6 * nn;          // 12 nn
  double* q2 = g6 + 12 * nn;         // 2 nn
  double* g2 = q2 + 2 * nn;          // 4 nn
  double* eg = g2 + 4 * nn;          // 12 ne
  pressure_inputs_kernel<T><<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, ustar, ustride, uoff, P, fields, q6);
  launch_node_gradients(m, ne_off, ne_list, 6, q6, eg, g6, s);
  second_inputs_kernel<<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, g6, q2);
  launch_node_gradients(m, ne_off, ne_list, 2, q2, eg, g2, s);
  pressure_src_kernel<T><<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, g6, g2, fields, m.ncls, m.nrm, nu, dt, Cp, src, flux);
  (void)ne;
}

size_t pressure_rhs_scratch_doubles(int nn, int ne) {
  return 24 * static_cast<size_t>(nn) + 12 * static_cast<size_t>(ne);
}

// The Galerkin load of Eq. 33 with its nodal mean removed; red holds kRedBlocks + 1 doubles.
void launch_pressure_load(const FemDev& m, const double* src, const double* flux, double* b, double* red,
                          cudaStream_t s) {
  pressure_load_kernel<<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, m.row, m.col, m.mval, src, flux, m.boff, m.bnb,
                                                        m.blen, b);
  const int nblk = pcg_blocks(m.nn);
  dot_part_kernel<<<nblk, kEB, 0, s>>>(m.nn, nullptr, b, red);
  dot_finish_kernel<<<1, kEB, 0, s>>>(nblk, red, red + kRedBlocks);
  sub_mean_kernel<<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, red + kRedBlocks, static_cast<double>(m.nn), b);
}

// Zero integral: x -= (sum_n mlump_n x_n) / (domain area).
void launch_zero_mean(const FemDev& m, double* x, double* red, cudaStream_t s) {
  const int nblk = pcg_blocks(m.nn);
  dot_part_kernel<<<nblk, kEB, 0, s>>>(m.nn, m.mlump, x, red);
  dot_finish_kernel<<<1, kEB, 0, s>>>(nblk, red, red + kRedBlocks);
  sub_mean_kernel<<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, red + kRedBlocks, m.area, x);
}

template <typename T>
void launch_write_wp(int nn, const double* x, T* fields, cudaStream_t s) {
  write_wp_kernel<T><<<blocks_for(nn), kEB, 0, s>>>(nn, x, fields);
}

template <typename T>
void launch_write_pgrad(const FemDev& m, const int32_t* ne_off, const int32_t* ne_list, const double* P,
                        double* eg, double* gp, T* fields, cudaStream_t s) {
  launch_node_gradients(m, ne_off, ne_list, 1, P, eg, gp, s);
  write_pgrad_kernel<T><<<blocks_for(m.nn), kEB, 0, s>>>(m.nn, gp, fields);
}

void launch_add(int nn, const double* a, double* b, cudaStream_t s) {
  add_kernel<<<blocks_for(nn), kEB, 0, s>>>(nn, a, b);
}

#define PDFX_INSTANTIATE(T)                                                                         \
  template void launch_wp_rhs<T>(const T*, int, const WpConst&, double*, double*, int*, cudaStream_t); \
  template void launch_wp_bc<T>(const T*, int, const WpConst&, const int8_t*, const double*, uint8_t*, \
                                double*, int*, cudaStream_t);                                        \
  template void launch_pressure_rhs<T>(const FemDev&, const int32_t*, const int32_t*, const double*,  \
                                       int, int, const double*, const T*, double, double, double,     \
                                       double*, double*, double*, cudaStream_t);                      \
  template void launch_write_wp<T>(int, const double*, T*, cudaStream_t);                             \
  template void launch_read_wp<T>(int, const T*, double*, cudaStream_t);                              \
  template void launch_write_pgrad<T>(const FemDev&, const int32_t*, const int32_t*, const double*,   \
                                      double*, double*, T*, cudaStream_t);
PDFX_INSTANTIATE(float)
PDFX_INSTANTIATE(double)
#undef PDFX_INSTANTIATE

}  // namespace pdfx
