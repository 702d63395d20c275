// Particle advance (one thread per particle slot) and particle initialisation.
//
// Per particle, in the order of one explicit Euler-Maruyama step (Sect. 3.1):
//   area coordinates at X^n in the host element (Eqs. 44-45) and interpolation of the 31
//   nodal fields (Eq. 37); k, eps (Eq. 18), G_ij and C0 (Eq. 11), production and S_omega
//   (Eq. 20), t_m (Eq. 25); six Gaussians and one uniform (Sect. 3.9); velocity (Eq. 27),
//   position (Eq. 7), frequency (Eq. 19), scalar (Eq. 24); wall conditions (Eqs. 53-58)
//   and free-slip reflection; periodic wrap; source disc (Sect. 4.1.2); neighbour walk to
//   the new host element (Sect. 3.6).  Counts per new element are aggregated per warp.
// The simplified model of the particle-redistribution test (Eqs. 46-47, model 1) has its
// own kernel and shares the end of the update (reflection, wrap, walk, store, counts).
#include "pdfx_internal.h"

namespace pdfx {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ bool inside(const ElemGeo<T>& g, const ElemTopo& t, const Pos<T>& P, T L) {
  T na, nb, nc;
  area_cross(g, t.n0, t.n1, t.n2, P, L, na, nb, nc);
  return na >= T(0) && nb >= T(0) && nc >= T(0);
}

// Sect. 3.6: walk to the neighbour opposite the lowest area coordinate (ties: lowest local
// vertex).  Across a free-slip boundary edge (Sect. 4.2) the particle is reflected across
// that edge's line, its normal velocity reversed (*refl set), and the walk goes on from the
// same element; each reflection counts as a hop.  After kHopLimit hops, at any other
// boundary edge, or when the point is not strictly behind the free-slip line, search the
// elements around the nodes of the old host element (lowest containing id), then all
// elements.
template <typename T>
__device__ int walk(const AdvanceArgs<T>& a, int e0, Pos<T>& P, T (&U)[3], T L, int& hops,
                    int& fb, int& brute, int& refl) {
  int e = e0;
  hops = 0;
  for (;;) {
    const ElemGeo<T> g = a.geo[e];
    const ElemTopo t = a.topo[e];
    T la, lb, lc;   // 2 N^k: signs and order of the area coordinates
    area_cross(g, t.n0, t.n1, t.n2, P, L, la, lb, lc);
    if (la >= T(0) && lb >= T(0) && lc >= T(0)) return e;
    if (hops >= kHopLimit) break;
    int k = 0;
    T mn = la;
    if (lb < mn) { k = 1; mn = lb; }
    if (lc < mn) k = 2;
    const int nb = k == 0 ? t.nb0 : (k == 1 ? t.nb1 : t.nb2);
    if (nb < 0) {
      if (nb == -1) break;
      const Line<T> ln = a.fsedges[-2 - nb];
      const T d = line_dist(ln, P, L);
      if (!(d < T(0))) break;
      pos_reflect(P, d, ln.nx, ln.ny);
      const T un = U[0] * ln.nx + U[1] * ln.ny;
      U[0] -= T(2) * un * ln.nx;
      U[1] -= T(2) * un * ln.ny;
      refl = 1;
      ++hops;
      continue;
    }
    e = nb;
    ++hops;
  }
  fb = 1;
  const ElemTopo t0 = a.topo[e0];
  int best = -1;
#pragma unroll
  for (int kv = 0; kv < 3; ++kv) {
    const int nd = kv == 0 ? t0.n0 : (kv == 1 ? t0.n1 : t0.n2);
    for (int i = a.ne_off[nd]; i < a.ne_off[nd + 1]; ++i) {
      const int f = a.ne_list[i];
      if (best >= 0 && f >= best) continue;
      if (inside(a.geo[f], a.topo[f], P, L)) best = f;
    }
  }
  if (best >= 0) return best;
  brute = 1;       // searched over all elements by brute_search_kernel
  return -1;
}

// q = lambda_A f_A + lambda_B f_B + lambda_C f_C for the 31 used field slots.
__device__ __forceinline__ void interp_fields(const double* __restrict__ F, int na, int nb, int nc,
                                              double la, double lb, double lc, double* q) {
  const double2* A = reinterpret_cast<const double2*>(F + (size_t)kNF * na);
  const double2* B = reinterpret_cast<const double2*>(F + (size_t)kNF * nb);
  const double2* C = reinterpret_cast<const double2*>(F + (size_t)kNF * nc);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const double2 a = __ldg(A + i), b = __ldg(B + i), c = __ldg(C + i);
    q[2 * i] = la * a.x + lb * b.x + lc * c.x;
    q[2 * i + 1] = la * a.y + lb * b.y + lc * c.y;
  }
}
__device__ __forceinline__ void interp_fields(const float* __restrict__ F, int na, int nb, int nc,
                                              float la, float lb, float lc, float* q) {
  const float4* A = reinterpret_cast<const float4*>(F + (size_t)kNF * na);
  const float4* B = reinterpret_cast<const float4*>(F + (size_t)kNF * nb);
  const float4* C = reinterpret_cast<const float4*>(F + (size_t)kNF * nc);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 a = __ldg(A + i), b = __ldg(B + i), c = __ldg(C + i);
    q[4 * i] = la * a.x + lb * b.x + lc * c.x;
    q[4 * i + 1] = la * a.y + lb * b.y + lc * c.y;
    q[4 * i + 2] = la * a.z + lb * b.z + lc * c.z;
    q[4 * i + 3] = la * a.w + lb * b.w + lc * c.w;
  }
}

// Reciprocal, square root and cube root of the closure (Eqs. 11, 18, 25).  FP64 form: the
// correctly rounded functions.  FP32 form: the hardware approximations (a few units in the
// last place; the state tolerance of this form is 1e-5) called through CUDA's intrinsics;
// arguments are positive or zero.
__device__ __forceinline__ double trcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float trcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double tsqrt_ratio(double a, double b) { return sqrt(a / b); }
__device__ __forceinline__ float tsqrt_ratio(float a, float b) { return tsqrt(a * trcp(b)); }
__device__ __forceinline__ double tcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float tcbrt(float x) { return exp2f(__log2f(x) * (1.0f / 3.0f)); }

// Box & Muller (1958) for the step's six Gaussians: FP64 form as everywhere; FP32 form with
// the hardware logarithm, square root and sine/cosine (CUDA intrinsics), the angle taken in
// (-pi, pi) where they are most accurate: (cos, sin)(2 pi u) = -(cos, sin)(2 pi (u - 1/2)).
__device__ __forceinline__ void step_gaussians(uint32_t w1, uint32_t w2, double& g1, double& g2) {
  box_muller(w1, w2, g1, g2);
}
__device__ __forceinline__ void step_gaussians(uint32_t w1, uint32_t w2, float& g1, float& g2) {
  const float r = tsqrt(-2.0f * __logf(uniform01(w1, 0.0f)));
  float sn, cs;
  __sincosf(6.2831853071795865f * (uniform01(w2, 0.0f) - 0.5f), &sn, &cs);
  g1 = -r * cs;
  g2 = -r * sn;
}
__device__ __forceinline__ double texp(double x) { return exp(x); }
__device__ __forceinline__ float texp(float x) { return expf(x); }

template <typename T>
__device__ __forceinline__ bool finite(T v) { return isfinite(v); }
__device__ __forceinline__ double pos_lead(const Pos<double>& P) { return P.x + P.y; }
__device__ __forceinline__ float pos_lead(const Pos<float>& P) { return P.xh + P.yh; }

__device__ __forceinline__ void warp_count(unsigned long long* diag, int slot, int v) {
  const unsigned s = __reduce_add_sync(kFull, static_cast<unsigned>(v));
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(diag + slot, static_cast<unsigned long long>(s));
}
// The same per warp into the block's counters in shared memory.
__device__ __forceinline__ void warp_count(unsigned* bc, int slot, int v) {
  const unsigned s = __reduce_add_sync(kFull, static_cast<unsigned>(v));
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(bc + slot, s);
}
// Block counters: cleared at the start of a kernel, added to the diagnostics at its end (one
// global atomic per block and counter instead of one per warp on the same address).
__device__ __forceinline__ void block_counts_clear(unsigned* bc) {
  for (int k = threadIdx.x; k < kDiagCount; k += blockDim.x) bc[k] = 0u;
  __syncthreads();
}
__device__ __forceinline__ void block_counts_flush(unsigned* bc, unsigned long long* diag) {
  __syncthreads();
  for (int k = threadIdx.x; k < kDiagCount; k += blockDim.x)
    if (bc[k]) atomicAdd(diag + k, static_cast<unsigned long long>(bc[k]));
}

// Per-particle event flags of one update, summed per warp into the diagnostics.
struct StepFlags {
  int hops = 0, fb = 0, brute = 0, lost = 0, wall = 0, fs = 0, oref = 0, c0 = 0, gex = 0,
      src = 0, nf = 0;
  int hop_bin = -1;
};

// The end of one particle update, common to both models: free-slip reflection with reversal
// of the normal velocity (Sect. 4.2), periodic wrap, finiteness, neighbour walk to the new
// host element (Sect. 3.6, with the reflections of a particle that crosses a free-slip edge
// further on), source disc (Sect. 4.1.2) and the store of the new state.  Returns the new
// element.
template <typename T>
__device__ __forceinline__ int finish_update(const AdvanceArgs<T>& a, const Model<T>& M, int64_t i,
                                             int e, const ElemTopo& tp, Pos<T> Pn, T (&Un)[3],
                                             T wn, T psin, StepFlags& f) {
  const T L = M.period_x;
  if (tp.fslip >= 0) {
    const Line<T> ln = a.fslines[tp.fslip];
    const T d1 = line_dist(ln, Pn, L);
    if (d1 < T(0)) {
      f.fs = 1;
      pos_reflect(Pn, d1, ln.nx, ln.ny);
      const T un = Un[0] * ln.nx + Un[1] * ln.ny;
      Un[0] -= T(2) * un * ln.nx;
      Un[1] -= T(2) * un * ln.ny;
    }
  }
  pos_wrap(Pn, L);
  // a sum of finite terms of this size is finite; a NaN or infinity anywhere is not
  if (!finite(pos_lead(Pn) + Un[0] + Un[1] + Un[2] + wn + psin)) f.nf = 1;

  int hops = 0, fb = 0, brute = 0, refl = 0;
  int e_new = walk(a, e, Pn, Un, L, hops, fb, brute, refl);
  f.hops = hops;
  f.fb = fb;
  f.brute = brute;
  f.hop_bin = hops < 7 ? hops : 7;
  if (refl) {
    f.fs = 1;
    pos_wrap(Pn, L);
  }
  if (M.source_on) {
    const T sx = rel_x(Pn, M.src_x, M.src_xl, L), sy = rel_y(Pn, M.src_y, M.src_yl);
    if (sx * sx + sy * sy <= M.src_r * M.src_r) { psin = T(1); f.src = 1; }
  }
  if (e_new < 0) {
    // counted in the old element for now; the brute-force kernel moves it (or flags it)
    e_new = e;
    const int at = atomicAdd(a.brute_count, 1);
    if (at < a.brute_cap) a.brute_list[at] = static_cast<int32_t>(i);
    else f.lost = 1;
  }

  store_pos(a.p, i, Pn);
  a.p.u[i] = Un[0];
  a.p.v[i] = Un[1];
  a.p.w[i] = Un[2];
  a.p.om[i] = wn;
  a.p.psi[i] = psin;
  a.p.elem[i] = e_new;
  return e_new;
}

// Counts per new element, aggregated over the lanes of a warp that share it (one atomic when
// the whole warp shares one element, the common case in element-ordered storage), and the
// diagnostics counters (into the block's counters bc) and error word.  Every lane of the
// warp takes part.
template <typename T>
__device__ __forceinline__ void count_update(const AdvanceArgs<T>& a, bool valid, int e_new,
                                             const StepFlags& f, unsigned* bc) {
  const unsigned active = __ballot_sync(kFull, valid);
  if (valid) {
    const int lead = __ffs(active) - 1;
    const int e_lead = __shfl_sync(active, e_new, lead);
    if (__all_sync(active, e_new == e_lead)) {
      if ((threadIdx.x & 31) == lead) atomicAdd(a.cnt + e_lead, __popc(active));
    } else {
      const unsigned peers = __match_any_sync(active, e_new);
      if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(a.cnt + e_new, __popc(peers));
    }
  }
  // hops: the few lanes that hopped add to the block's counters themselves
  if (f.hops > 0) atomicAdd(bc + kDiagHops, static_cast<unsigned>(f.hops));
  if (__any_sync(kFull, f.fb | f.brute | f.lost | f.nf | f.gex | f.c0)) {
    warp_count(bc, kDiagFallback, f.fb);
    warp_count(bc, kDiagBrute, f.brute);
    warp_count(bc, kDiagLost, f.lost);
    warp_count(bc, kDiagNonFinite, f.nf);
    warp_count(bc, kDiagGammaExhausted, f.gex);
    warp_count(bc, kDiagC0Clamp, f.c0);
  }
  if (__any_sync(kFull, f.lost) && (threadIdx.x & 31) == 0) atomicCAS(a.err, 0, PDFX_ERR_LOST_PARTICLE);
  if (__any_sync(kFull, f.nf) && (threadIdx.x & 31) == 0) atomicCAS(a.err, 0, PDFX_ERR_NONFINITE);
  if (__any_sync(kFull, f.wall | f.fs | f.oref | f.src)) {
    warp_count(bc, kDiagWall, f.wall);
    warp_count(bc, kDiagFreeSlip, f.fs);
    warp_count(bc, kDiagOmegaReflect, f.oref);
    warp_count(bc, kDiagSource, f.src);
  }
  if (f.hop_bin > 0) atomicAdd(bc + kDiagHopHist0 + f.hop_bin, 1u);
}

// FP32: 4 blocks of 256 per SM (64 registers); FP64: 2 blocks.  BATCH: model constants and
// Philox key of the particle's instance (that of its element) instead of a.m, a.k0, a.k1.
// Tiles of blockDim.x particles, one particle per thread: block b takes the consecutive tiles
// [b per, (b + 1) per), per = ceil(tiles / gridDim.x), so that its particles, stored by
// element, reuse one another's element, geometry and nodal-field lines in L1; the block's
// counters are flushed once, after its last tile.
template <typename T, bool BATCH>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) advance_kernel(const AdvanceArgs<T> a) {
  __shared__ unsigned bc[kDiagCount];
  block_counts_clear(bc);
  const int64_t ntiles = (a.np + blockDim.x - 1) / blockDim.x;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * per;
  const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
#pragma unroll 1
  for (int64_t tile = t0; tile < t1; ++tile) {
    const int64_t i = tile * blockDim.x + threadIdx.x;
    const bool valid = i < a.np;
    StepFlags f;
    int e_new = -1;
    if (valid) {
      const int e = a.p.elem[i];
      const int ki = BATCH ? a.einst[e] : 0;
      const Model<T>& M = BATCH ? a.inst[ki].m : a.m;
      const uint32_t k0 = BATCH ? a.inst[ki].k0 : a.k0, k1 = BATCH ? a.inst[ki].k1 : a.k1;
      const T L = M.period_x;
      const Pos<T> P0 = load_pos(a.p, i);
      T U0[3] = {a.p.u[i], a.p.v[i], a.p.w[i]};
      if (a.corr) {   // Eq. 31 of the last coupled step, applied as the velocity is read
        U0[0] = static_cast<T>(static_cast<double>(U0[0]) - a.corr[2 * static_cast<size_t>(e)]);
        U0[1] = static_cast<T>(static_cast<double>(U0[1]) - a.corr[2 * static_cast<size_t>(e) + 1]);
      }
      const T w0 = a.p.om[i], psi0 = a.p.psi[i];
      const uint32_t pid = a.p.pid[i];
      const int cpi = a.p.cp[i];
      const ElemGeo<T> g = a.geo[e];
      const ElemTopo tp = a.topo[e];

      // Eqs. 37-38, 44-45 at X^n (interp_mode 1: element average)
      T la, lb, lc;
      if (M.interp_mode == 1) {
        la = lb = lc = T(1) / T(3);
      } else {
        area_coords(g, tp.n0, tp.n1, tp.n2, P0, L, la, lb, lc);
      }
      T q[kNF];
      interp_fields(a.fields, tp.n0, tp.n1, tp.n2, la, lb, lc, q);
      const T Um[3] = {q[0], q[1], q[2]};
      const T dP[3] = {q[3], q[4], T(0)};
      T R[3][3];
      R[0][0] = q[23]; R[1][1] = q[24]; R[2][2] = q[25];
      R[0][1] = R[1][0] = q[26];
      R[0][2] = R[2][0] = q[27];
      R[1][2] = R[2][1] = q[28];
      const T Om = q[29];

      // k and Eq. 18 (floored at 1e-30 so a particle on a wall keeps finite coefficients)
      T k = T(0.5) * (R[0][0] + R[1][1] + R[2][2]);
      if (k < T(1e-30)) k = T(1e-30);
      T eps = Om * (k + M.nuCT2 * Om);
      if (eps < T(1e-30)) eps = T(1e-30);
      const T ik = trcp(k), ieps = trcp(eps);
      // Eq. 11
      T C0;
      if (M.c0_mode == 1) {
        C0 = M.C0;
      } else {
        T s = T(0);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) s += q[14 + 3 * r + c] * R[r][c];
        C0 = T(-2) / T(3) * s * ik * ieps;
      }
      // production P = -<u_i u_j> d<U_i>/dx_j (x, y) and Eq. 20
      T prod = T(0);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) prod -= R[r][c] * q[5 + 2 * r + c];
      const T Somega = M.Cw2 - M.Cw1 * prod * ieps;
      // 1 / t_m: Eq. 25, or the IEM time scale t_m = 2k / (C_phi eps)
      T itm;
      if (M.tm_mode == 1) {
        itm = T(0.5) * M.Cphi * eps * ik;
      } else {
        const T kt = k * ieps, kol = M.CT * tsqrt(M.nu * ieps);
        const T a2 = kt > kol ? kt : kol;
        const T ddx = rel_x(P0, M.src_x, M.src_xl, L), ddy = rel_y(P0, M.src_y, M.src_yl);
        const T Uc2 = Um[0] * Um[0] + Um[1] * Um[1] + Um[2] * Um[2];
        T tm = a2;
        if (Uc2 > T(0)) {
          const T a1 = M.cs_r2 * tcbrt(ieps) + M.Ct * tsqrt_ratio(ddx * ddx + ddy * ddy, Uc2);
          tm = a1 < a2 ? a1 : a2;
        }
        itm = trcp(tm);
      }

      // Sect. 3.9: six Gaussians and eta
      const uint32_t step = *a.stepc;
      const uint4 r0 = philox(make_uint4(pid, step, kPurStep, 0u), k0, k1);
      const uint4 r1 = philox(make_uint4(pid, step, kPurStep, 1u), k0, k1);
      T xi[6];
      step_gaussians(r0.x, r0.y, xi[0], xi[1]);
      step_gaussians(r0.z, r0.w, xi[2], xi[3]);
      step_gaussians(r1.x, r1.y, xi[4], xi[5]);
      const T eta = uniform01(r1.z, T(0));     // first wall line
      const T eta2 = uniform01(r1.w, T(0));    // second wall line (a corner element)
      const T dt = a.dt;
      const T sdt = a.sdt;
      const T dWx = sdt * xi[0], dWy = sdt * xi[1];
      const T s2nu = M.s2nu;

      // Eq. 27 (C0 eps < 0 is clamped under the root and counted);
      // G_ij (U_j - <U_j>) = (wp_ij (U_j - <U_j>) - eps/2 (U_i - <U_i>)) / k  (Eq. 11)
      T c0e = C0 * eps;
      if (c0e < T(0)) { c0e = T(0); f.c0 = 1; }
      const T sc0e = tsqrt(c0e) * sdt;
      const T dU[3] = {U0[0] - Um[0], U0[1] - Um[1], U0[2] - Um[2]};
      T Un[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const T base = U0[r] - dP[r] * dt + T(2) * M.nu * q[11 + r] * dt +
                       s2nu * (q[5 + 2 * r] * dWx + q[6 + 2 * r] * dWy);
        T gsum = -T(0.5) * eps * dU[r];
#pragma unroll
        for (int c = 0; c < 3; ++c) gsum += q[14 + 3 * r + c] * dU[c];
        Un[r] = base + gsum * ik * dt + sc0e * xi[2 + r];
      }
      // Eq. 7 (same dW as Eq. 27)
      Pos<T> Pn = P0;
      pos_move(Pn, U0[0], U0[1], dt, s2nu, dWx, dWy);
      // Eq. 19, reflected at zero
      const T wpos = w0 > T(0) ? w0 : T(0);
      T wn = w0 - M.C3 * Om * (w0 - Om) * dt - Somega * Om * w0 * dt +
             tsqrt(T(2) * M.C3 * M.C4 * Om * Om * wpos) * (sdt * xi[5]);
      if (wn < T(0)) { wn = -wn; f.oref = 1; }
      // Eq. 24 with the conditional mean of the particle's bin
      const T phic = static_cast<T>(a.vcce[(size_t)e * a.G + cpi]);
      T psin = psi0 - (psi0 - phic) * dt * itm;

      // Sect. 3.8: wall elements only; each wall line in turn (a corner element has two),
      // the second from the position after the first's reflection
      if (tp.wall >= 0) {
        const int lines[2] = {tp.wall, a.wall2[e]};
        bool any_hit = false;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (lines[j] < 0) break;
          const Line<T> ln = a.walls[lines[j]];
          const T d0 = line_dist(ln, P0, L);
          const T d1 = line_dist(ln, Pn, L);
          bool hit;
          if (d1 < T(0)) {
            hit = true;
          } else {
            const T dd0 = d0 > T(0) ? d0 : T(0);
            hit = (j == 0 ? eta : eta2) < texp(-dd0 * d1 / (M.nu * dt));   // Eqs. 53, 55
          }
          if (hit) {
            any_hit = true;
            if (d1 < T(0)) pos_reflect(Pn, d1, ln.nx, ln.ny);
          }
        }
        if (any_hit) {
          f.wall = 1;
          Un[0] = Un[1] = Un[2] = T(0);                  // Eq. 56
          int ex = 0;                                    // Eq. 58
          wn = gamma_draw<T>(k0, k1, pid, step, kPurWallGamma, T(1) / M.C4, M.C4 * q[30], &ex);
          f.gex = ex;
        }
      }
      e_new = finish_update(a, M, i, e, tp, Pn, Un, wn, psin, f);
    }
    count_update(a, valid, e_new, f, bc);
  }
  block_counts_flush(bc, a.diag);
}

// Eqs. 46-47 (model 1), the particle-redistribution test of Sect. 3.7: one thread per
// particle slot.  The mean velocity is the particles' own, the nodal means of the previous
// statistics pass interpolated at X^n (Eq. 37; interp_mode 1: element average);
// U^{n+1} = U - (U - alpha <U>) dt + sqrt(2 dt) xi (xi the first three Gaussians of the
// step's first Philox block), X^{n+1} = X + U dt; omega and psi are kept.  The grid has no
// no-slip walls; free-slip reflection, wrap, source and walk as in the full model.
template <typename T, bool BATCH>
__global__ void __launch_bounds__(256) simple_advance_kernel(const AdvanceArgs<T> a) {
  __shared__ unsigned bc[kDiagCount];
  block_counts_clear(bc);
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool valid = i < a.np;
  StepFlags f;
  int e_new = -1;
  if (valid) {
    const int e = a.p.elem[i];
    const int ki = BATCH ? a.einst[e] : 0;
    const Model<T>& M = BATCH ? a.inst[ki].m : a.m;
    const uint32_t k0 = BATCH ? a.inst[ki].k0 : a.k0, k1 = BATCH ? a.inst[ki].k1 : a.k1;
    const Pos<T> P0 = load_pos(a.p, i);
    T U0[3] = {a.p.u[i], a.p.v[i], a.p.w[i]};
    if (a.corr) {
      U0[0] = static_cast<T>(static_cast<double>(U0[0]) - a.corr[2 * static_cast<size_t>(e)]);
      U0[1] = static_cast<T>(static_cast<double>(U0[1]) - a.corr[2 * static_cast<size_t>(e) + 1]);
    }
    const ElemTopo tp = a.topo[e];
    T la, lb, lc;
    if (M.interp_mode == 1) {
      la = lb = lc = T(1) / T(3);
    } else {
      area_coords(a.geo[e], tp.n0, tp.n1, tp.n2, P0, M.period_x, la, lb, lc);
    }
    const double* m0 = a.nmom + static_cast<size_t>(kNS) * tp.n0;
    const double* m1 = a.nmom + static_cast<size_t>(kNS) * tp.n1;
    const double* m2 = a.nmom + static_cast<size_t>(kNS) * tp.n2;
    const uint4 r0 = philox(make_uint4(a.p.pid[i], *a.stepc, kPurStep, 0u), k0, k1);
    T xi[4];
    box_muller(r0.x, r0.y, xi[0], xi[1]);
    box_muller(r0.z, r0.w, xi[2], xi[3]);
    const T dt = a.dt;
    const T s2dt = sqrt(T(2) * dt);
    T Un[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T Um = la * T(m0[1 + r]) + lb * T(m1[1 + r]) + lc * T(m2[1 + r]);
      Un[r] = U0[r] - (U0[r] - M.alpha * Um) * dt + s2dt * xi[r];
    }
    Pos<T> Pn = P0;
    pos_add(Pn, U0[0] * dt, U0[1] * dt);
    e_new = finish_update(a, M, i, e, tp, Pn, Un, a.p.om[i], a.p.psi[i], f);
  }
  count_update(a, valid, e_new, f, bc);
  block_counts_flush(bc, a.diag);
}

// Last resort of Sect. 3.6 for particles neither the walk nor the fall-back located: one
// block per particle tests every element (of the particle's instance); the lowest
// containing id wins.  The particle's count moves from its old element to the found one; a
// particle in no element is flagged.
template <typename T, bool BATCH>
__global__ void __launch_bounds__(256) brute_search_kernel(AdvanceArgs<T> a) {
  __shared__ int best_s[8];
  const int n = min(*a.brute_count, a.brute_cap);
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const int32_t i = a.brute_list[j];
    const Pos<T> P = load_pos(a.p, i);
    const int ki = BATCH ? a.einst[a.p.elem[i]] : 0;
    const int f0 = BATCH ? a.inst[ki].e0 : 0, f1 = BATCH ? a.inst[ki].e1 : a.ne;
    const T L = BATCH ? a.inst[ki].m.period_x : a.m.period_x;
    int best = 0x7fffffff;
    for (int f = f0 + threadIdx.x; f < f1; f += blockDim.x)
      if (f < best && inside(a.geo[f], a.topo[f], P, L)) best = f;
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0) best_s[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (blockDim.x >> 5); ++w) best = min(best, best_s[w]);
      const int32_t e0 = a.p.elem[i];
      if (best < f1) {
        if (best != e0) {
          atomicSub(a.cnt + e0, 1);
          atomicAdd(a.cnt + best, 1);
          a.p.elem[i] = best;
        }
      } else {
        atomicAdd(a.diag + kDiagLost, 1ull);
        atomicCAS(a.err, 0, PDFX_ERR_LOST_PARTICLE);
        const unsigned long long k = atomicAdd(a.diag + kDiagLostRecord, 1ull);
        if (k < kLostRecords) {
          double* rec = a.lost_rec + 4 * k;
          rec[0] = pos_x(P);
          rec[1] = pos_y(P);
          rec[2] = static_cast<double>(e0);
          rec[3] = static_cast<double>(a.p.pid[i]);
        }
      }
    }
    __syncthreads();
  }
}

// Sect. 3.7: particle id e * ppe + k, uniform in element e (square-root method of Osada
// et al.), velocity N(<U>, 2k/3 I), frequency Gamma(1/C4, C4 <omega>), scalar from the
// source disc.
template <typename T>
__device__ __forceinline__ int init_one(Particles<T> p, int64_t i, int e, uint32_t pid,
                                        const ElemGeo<T>* geo, const ElemTopo* topo,
                                        const T* fields, const Model<T>& m, uint32_t k0,
                                        uint32_t k1) {
  int c_gex = 0;
  {
    const uint4 r0 = philox(make_uint4(pid, 0u, kPurInit, 0u), k0, k1);
    const uint4 r1 = philox(make_uint4(pid, 0u, kPurInit, 1u), k0, k1);
    const ElemGeo<T> g = geo[e];
    const ElemTopo tp = topo[e];
    const T s = sqrt(uniform01(r0.x, T(0)));
    const T t = uniform01(r0.y, T(0));
    Pos<T> P = triangle_point(g, s, t, m.period_x);
    T la, lb, lc;
    if (m.interp_mode == 1) {
      la = lb = lc = T(1) / T(3);
    } else {
      area_coords(g, tp.n0, tp.n1, tp.n2, P, m.period_x, la, lb, lc);
    }
    T q[kNF];
    interp_fields(fields, tp.n0, tp.n1, tp.n2, la, lb, lc, q);
    T k2 = T(0.5) * (q[23] + q[24] + q[25]);
    if (k2 < T(0)) k2 = T(0);
    const T sd = sqrt(T(2) * k2 / T(3));
    T g0, g1, g2, gd;
    box_muller(r0.z, r0.w, g0, g1);
    box_muller(r1.x, r1.y, g2, gd);
    int ex = 0;
    const T om = gamma_draw<T>(k0, k1, pid, 0u, kPurInitGamma, T(1) / m.C4, m.C4 * q[29], &ex);
    c_gex = ex;
    pos_wrap(P, m.period_x);
    bool src = false;
    if (m.source_on) {
      const T sx = rel_x(P, m.src_x, m.src_xl, m.period_x), sy = rel_y(P, m.src_y, m.src_yl);
      src = sx * sx + sy * sy <= m.src_r * m.src_r;
    }
    store_pos(p, i, P);
    p.u[i] = q[0] + sd * g0;
    p.v[i] = q[1] + sd * g1;
    p.w[i] = q[2] + sd * g2;
    p.om[i] = om;
    p.psi[i] = src ? T(1) : T(0);
    p.pid[i] = pid;
    p.elem[i] = e;
    p.cp[i] = 0;
  }
  return c_gex;
}

template <typename T>
__global__ void init_kernel(Particles<T> p, int32_t ne, int32_t ppe, const ElemGeo<T>* geo,
                            const ElemTopo* topo, const T* fields, Model<T> m, uint32_t k0,
                            uint32_t k1, unsigned long long* diag) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t np = static_cast<int64_t>(ne) * ppe;
  int c_gex = 0;
  if (i < np)
    c_gex = init_one(p, i, static_cast<int>(i / ppe), static_cast<uint32_t>(i), geo, topo, fields,
                     m, k0, k1);
  warp_count(diag, kDiagGammaExhausted, c_gex);
}

// Batches: slot i belongs to the instance k with p0_k <= i < p0_{k+1}; id i - p0_k, element
// e0_k + (i - p0_k) / ppe_k (the numbering of a run of that instance alone).
template <typename T>
__global__ void init_batch_kernel(Particles<T> p, int64_t np, int K, const InstDev<T>* inst,
                                  const int64_t* ip0, const ElemGeo<T>* geo, const ElemTopo* topo,
                                  const T* fields, unsigned long long* diag) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int c_gex = 0;
  if (i < np) {
    int lo = 0, hi = K - 1;   // largest k with ip0[k] <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ip0[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const InstDev<T>& I = inst[lo];
    const int64_t loc = i - I.p0;
    c_gex = init_one(p, i, I.e0 + static_cast<int>(loc / I.ppe), static_cast<uint32_t>(loc), geo,
                     topo, fields, I.m, I.k0, I.k1);
  }
  warp_count(diag, kDiagGammaExhausted, c_gex);
}

// Counts per element of a state whose element ids may come from the caller: an id outside
// 0 .. ne - 1 is not counted (the particle is in no element list), is counted in the
// diagnostics and sets the error word to PDFX_ERR_ELEMENT.
__global__ void count_kernel(const int32_t* __restrict__ elem, int64_t np, int32_t ne, int32_t* cnt,
                             unsigned long long* diag, int* err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int e = i < np ? elem[i] : -1;
  const bool bad = i < np && (e < 0 || e >= ne);
  const bool valid = i < np && !bad;
  const unsigned active = __ballot_sync(kFull, valid);
  if (valid) {
    const unsigned peers = __match_any_sync(active, e);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + e, __popc(peers));
  }
  if (__any_sync(kFull, bad)) {
    warp_count(diag, kDiagBadElement, bad ? 1 : 0);
    if ((threadIdx.x & 31) == 0) atomicCAS(err, 0, PDFX_ERR_ELEMENT);
  }
}

template <typename T>
__global__ void gather_by_pid_kernel(Particles<T> p, int64_t np, const int32_t* einst,
                                     const int64_t* ip0, double* x, double* y, double* u,
                                     double* v, double* w, double* om, double* psi,
                                     int32_t* elem, uint8_t* cp) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int64_t id = (einst ? ip0[einst[p.elem[i]]] : 0) + p.pid[i];
  const Pos<T> P = load_pos(p, i);
  if (x) x[id] = pos_x(P);
  if (y) y[id] = pos_y(P);
  if (u) u[id] = p.u[i];
  if (v) v[id] = p.v[i];
  if (w) w[id] = p.w[i];
  if (om) om[id] = p.om[i];
  if (psi) psi[id] = p.psi[i];
  if (elem) elem[id] = p.elem[i];
  if (cp) cp[id] = p.cp[i];
}

template <typename T>
__global__ void load_state_kernel(Particles<T> p, int64_t np, const int32_t* einst,
                                  const int64_t* ip0, const double* x, const double* y,
                                  const double* u, const double* v, const double* w,
                                  const double* om, const double* psi, const int32_t* elem,
                                  int32_t ne, unsigned long long* diag, int* err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= np) return;
  store_pos(p, i, pos_of(x[i], y[i], T(0)));
  p.u[i] = static_cast<T>(u[i]);
  p.v[i] = static_cast<T>(v[i]);
  p.w[i] = static_cast<T>(w[i]);
  p.om[i] = static_cast<T>(om[i]);
  p.psi[i] = static_cast<T>(psi[i]);
  // an element id outside the grid (device input is not checked on the host) is replaced
  // by element 0, whose walk relocates the particle at the next step, and raises
  // PDFX_ERR_ELEMENT; every later index stays within the grid
  int32_t e = elem[i];
  if (e < 0 || e >= ne) {
    atomicAdd(diag + kDiagBadElement, 1ull);
    atomicCAS(err, 0, PDFX_ERR_ELEMENT);
    e = 0;
  }
  p.elem[i] = e;
  p.pid[i] = static_cast<uint32_t>(i - (einst ? ip0[einst[e]] : 0));
  p.cp[i] = 0;
}

__global__ void convert_fields_kernel(const double* in, float* out, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = static_cast<float>(in[i]);
}

inline unsigned blocks_for(int64_t n, int threads) {
  return static_cast<unsigned>((n + threads - 1) / threads);
}

}  // namespace

template <typename T>
void launch_advance(const AdvanceArgs<T>& a, int num_sms, int block, cudaStream_t s) {
  if (a.np <= 0) return;
  cudaMemsetAsync(a.brute_count, 0, sizeof(int), s);
  const unsigned bgrid = static_cast<unsigned>(num_sms > 0 ? num_sms : 1);
  const unsigned grid = blocks_for(a.np, block);
  // FP32 advance_kernel: 16 waves of resident blocks, each block over a run of consecutive
  // tiles (at 25M particles: 4 waves 1.07 ms, 8 1.03, 16 1.01, 32 1.02, one tile per block
  // 1.14).  The FP64 form, bound by its FP64 pipe, keeps one tile per block (1.5% faster).
  const unsigned resident = bgrid * static_cast<unsigned>(1024 / block);
  const unsigned agrid = sizeof(T) == 4 && grid > 16u * resident ? 16u * resident : grid;
  if (a.einst) {
    if (a.m.model == 1) simple_advance_kernel<T, true><<<grid, block, 0, s>>>(a);
    else advance_kernel<T, true><<<agrid, block, 0, s>>>(a);
    brute_search_kernel<T, true><<<bgrid, 256, 0, s>>>(a);
  } else {
    if (a.m.model == 1) simple_advance_kernel<T, false><<<grid, block, 0, s>>>(a);
    else advance_kernel<T, false><<<agrid, block, 0, s>>>(a);
    brute_search_kernel<T, false><<<bgrid, 256, 0, s>>>(a);
  }
}

template <typename T>
void launch_init(Particles<T> p, int32_t ne, int32_t ppe, const ElemGeo<T>* geo,
                 const ElemTopo* topo, const T* fields, Model<T> m, uint32_t k0, uint32_t k1,
                 unsigned long long* diag, cudaStream_t s) {
  const int64_t np = static_cast<int64_t>(ne) * ppe;
  if (np <= 0) return;
  init_kernel<T><<<blocks_for(np, 256), 256, 0, s>>>(p, ne, ppe, geo, topo, fields, m, k0, k1, diag);
}

template <typename T>
void launch_init_batch(Particles<T> p, int64_t np, int K, const InstDev<T>* inst,
                       const int64_t* ip0, const ElemGeo<T>* geo, const ElemTopo* topo,
                       const T* fields, unsigned long long* diag, cudaStream_t s) {
  if (np <= 0) return;
  init_batch_kernel<T><<<blocks_for(np, 256), 256, 0, s>>>(p, np, K, inst, ip0, geo, topo, fields, diag);
}

void launch_count(const int32_t* elem, int64_t np, int32_t ne, int32_t* cnt, unsigned long long* diag,
                  int* err, cudaStream_t s) {
  if (np <= 0) return;
  count_kernel<<<blocks_for(np, 256), 256, 0, s>>>(elem, np, ne, cnt, diag, err);
}

template <typename T>
void launch_gather_by_pid(Particles<T> p, int64_t np, const int32_t* einst, const int64_t* ip0,
                          double* x, double* y, double* u, double* v, double* w, double* om,
                          double* psi, int32_t* elem, uint8_t* cp, cudaStream_t s) {
  if (np <= 0) return;
  gather_by_pid_kernel<T><<<blocks_for(np, 256), 256, 0, s>>>(p, np, einst, ip0, x, y, u, v, w, om,
                                                              psi, elem, cp);
}

template <typename T>
void launch_load_state(Particles<T> p, int64_t np, const int32_t* einst, const int64_t* ip0,
                       const double* x, const double* y, const double* u, const double* v,
                       const double* w, const double* om, const double* psi, const int32_t* elem,
                       int32_t ne, unsigned long long* diag, int* err, cudaStream_t s) {
  if (np <= 0) return;
  load_state_kernel<T><<<blocks_for(np, 256), 256, 0, s>>>(p, np, einst, ip0, x, y, u, v, w, om,
                                                           psi, elem, ne, diag, err);
}

void launch_convert_fields(const double* in, float* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  convert_fields_kernel<<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
}

#define PDFX_INSTANTIATE(T)                                                                    \
  template void launch_advance<T>(const AdvanceArgs<T>&, int, int, cudaStream_t);              \
  template void launch_init<T>(Particles<T>, int32_t, int32_t, const ElemGeo<T>*,              \
                               const ElemTopo*, const T*, Model<T>, uint32_t, uint32_t,        \
                               unsigned long long*, cudaStream_t);                             \
  template void launch_init_batch<T>(Particles<T>, int64_t, int, const InstDev<T>*,            \
                                     const int64_t*, const ElemGeo<T>*, const ElemTopo*,       \
                                     const T*, unsigned long long*, cudaStream_t);             \
  template void launch_gather_by_pid<T>(Particles<T>, int64_t, const int32_t*, const int64_t*, \
                                        double*, double*, double*, double*, double*, double*,  \
                                        double*, int32_t*, uint8_t*, cudaStream_t);            \
  template void launch_load_state<T>(Particles<T>, int64_t, const int32_t*, const int64_t*,    \
                                     const double*, const double*, const double*,              \
                                     const double*, const double*, const double*,              \
                                     const double*, const int32_t*, int32_t,                   \
                                     unsigned long long*, int*, cudaStream_t);
PDFX_INSTANTIATE(double)
PDFX_INSTANTIATE(float)
#undef PDFX_INSTANTIATE

}  // namespace pdfx
