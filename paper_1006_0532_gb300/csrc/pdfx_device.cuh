// Device building blocks shared by the pdfx kernels: counter-based random numbers,
// Gaussian and gamma sampling, and the per-element data layout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pdfx {

constexpr int kNF = 32;            // nodal field slots
constexpr int kNS = 13;            // statistics per element / node
constexpr int kHopLimit = 64;      // neighbour-walk hops before the fall-back search
constexpr int kGammaAttempts = 32; // Marsaglia-Tsang attempts before falling back to the mean

// Philox counter word 2 ("purpose"): independent streams per use.
enum Purpose : uint32_t { kPurStep = 0, kPurInit = 1, kPurWallGamma = 2, kPurRedist = 3,
                          kPurInitGamma = 4 };

// Diagnostic counter slots (int64 each).
enum Diag : int {
  kDiagHops = 0, kDiagFallback, kDiagBrute, kDiagLost, kDiagWall, kDiagFreeSlip,
  kDiagOmegaReflect, kDiagC0Clamp, kDiagGammaExhausted, kDiagMoves, kDiagSource,
  kDiagCapacity, kDiagNonFinite, kDiagHopHist0, kDiagLostRecord = kDiagHopHist0 + 8,
  kDiagBadElement, kDiagCount
};
constexpr int kLostRecords = 4;    // (x, y, old element, particle id) of the first lost particles
constexpr int kBruteCap = 4096;    // particles per step that may need the brute-force search

// Per-element geometry: the coordinates of the three nodes (x in [0, period)) and
// 1 / (2 A_e).
template <typename T>
struct __align__(sizeof(T) * 8) ElemGeo {
  T x0, y0, x1, y1, x2, y2, inv2a, pad;
};

// Per-element topology: node ids, neighbour across the edge opposite each vertex (-1 = a
// boundary edge; -2 - j = a free-slip boundary edge whose own line is entry j of the
// free-slip edge table), index into the no-slip and free-slip line tables (-1 = none).
struct __align__(16) ElemTopo {
  int n0, n1, n2, wall;
  int nb0, nb1, nb2, fslip;
};

// A boundary line: a point on it and the unit normal pointing into the domain.
template <typename T>
struct __align__(sizeof(T) * 4) Line {
  T px, py, nx, ny;
};

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  Counter = (particle id, step,
// purpose, block); key = (seed low word, seed high word ^ instance).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k0, static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k1, static_cast<uint32_t>(p0));
  }
  return c;
}

// Uniform on (0, 1) from one 32-bit word: (w + 1/2) 2^-32.  The FP32 form keeps relative
// precision for small words (the Gaussian tail) and may round the top words up to 1.
__device__ __forceinline__ double uniform01(uint32_t w, double) {
  return (static_cast<double>(w) + 0.5) * 2.3283064365386963e-10;
}
__device__ __forceinline__ float uniform01(uint32_t w, float) {
  return fmaf(__uint2float_rn(w), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

// Box & Muller (1958): two independent N(0, 1) from two uniform words.
__device__ __forceinline__ void box_muller(uint32_t w1, uint32_t w2, double& g1, double& g2) {
  const double r = sqrt(-2.0 * log(uniform01(w1, 0.0)));
  double s, c;
  sincospi(2.0 * uniform01(w2, 0.0), &s, &c);
  g1 = r * c;
  g2 = r * s;
}
__device__ __forceinline__ void box_muller(uint32_t w1, uint32_t w2, float& g1, float& g2) {
  const float r = sqrtf(-2.0f * logf(uniform01(w1, 0.0f)));
  float s, c;
  sincospif(2.0f * uniform01(w2, 0.0f), &s, &c);
  g1 = r * c;
  g2 = r * s;
}

template <typename T>
__device__ __forceinline__ T dlog(T x);
template <>
__device__ __forceinline__ double dlog<double>(double x) { return log(x); }
template <>
__device__ __forceinline__ float dlog<float>(float x) { return logf(x); }

// Gamma(shape >= 1, scale) by Marsaglia & Tsang (2000).  Attempt j uses Philox block j:
// one Gaussian from words 0-1 (cosine branch) and one uniform from word 2.  After
// kGammaAttempts rejections the mean is returned and *exhausted is set.
template <typename T>
__device__ T gamma_draw(uint32_t k0, uint32_t k1, uint32_t pid, uint32_t step, uint32_t purpose,
                        T shape, T scale, int* exhausted) {
  const T d = shape - T(1) / T(3);
  const T c = T(1) / sqrt(T(9) * d);
  for (uint32_t j = 0; j < kGammaAttempts; ++j) {
    const uint4 r = philox(make_uint4(pid, step, purpose, j), k0, k1);
    T xg, dummy;
    box_muller(r.x, r.y, xg, dummy);
    const T uu = uniform01(r.z, T(0));
    const T t = T(1) + c * xg;
    if (t <= T(0)) continue;
    const T vv = t * t * t;
    if (dlog(uu) < T(0.5) * xg * xg + d - d * vv + d * dlog(vv)) return d * vv * scale;
  }
  *exhausted = 1;
  return shape * scale;
}

template <typename T>
__device__ __forceinline__ T min_image(T d, T L) {
  if (L > T(0)) {
    if (d > T(0.5) * L) return d - L;
    if (d < T(-0.5) * L) return d + L;
  }
  return d;
}

template <typename T>
__device__ __forceinline__ T wrap_period(T x, T L) {
  if (L > T(0)) {
    if (x < T(0)) x += L;
    if (x >= L) x -= L;
  }
  return x;
}

// Separately rounded products (no fused multiply-add).  Every evaluation of an edge's
// cross product then rounds identically, whichever element and slot it is computed for,
// so the two elements sharing an edge always see exactly opposite values (a point on the
// edge is in both), and the FP64 form matches host arithmetic bit for bit.
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }

// (r_b - r_a) x (r_P - r_a) for the edge a -> b (minimum image in x).
template <typename T>
__device__ __forceinline__ T edge_cross(T xa, T ya, T xb, T yb, T x, T y, T L) {
  return xmul(min_image(xb - xa, L), y - ya) - xmul(yb - ya, min_image(x - xa, L));
}

// Twice the signed areas N^A, N^B, N^C (Eqs. 44-45, Fig. 1): for each vertex, the cross
// product of the opposite edge with the vector from one end of that edge to the particle.
// Each edge is pivoted at its lower-numbered node, so the two elements sharing an edge
// evaluate it with identical rounding and opposite signs (watertight point location).
template <typename T>
__device__ __forceinline__ void area_cross(const ElemGeo<T>& g, int na, int nb, int nc, T x, T y,
                                           T L, T& n0, T& n1, T& n2) {
  // edge opposite A: B -> C
  n0 = nb < nc ? edge_cross(g.x1, g.y1, g.x2, g.y2, x, y, L)
               : -edge_cross(g.x2, g.y2, g.x1, g.y1, x, y, L);
  // edge opposite B: C -> A
  n1 = nc < na ? edge_cross(g.x2, g.y2, g.x0, g.y0, x, y, L)
               : -edge_cross(g.x0, g.y0, g.x2, g.y2, x, y, L);
  // edge opposite C: A -> B
  n2 = na < nb ? edge_cross(g.x0, g.y0, g.x1, g.y1, x, y, L)
               : -edge_cross(g.x1, g.y1, g.x0, g.y0, x, y, L);
}

// Area coordinates lambda_k = N^k / A_e (Eqs. 37-38 shapefunction values at the particle).
template <typename T>
__device__ __forceinline__ void area_coords(const ElemGeo<T>& g, int na, int nb, int nc, T x, T y,
                                            T L, T& la, T& lb, T& lc) {
  area_cross(g, na, nb, nc, x, y, L, la, lb, lc);
  la *= g.inv2a;
  lb *= g.inv2a;
  lc *= g.inv2a;
}

// Point in the triangle with weights (1 - s) A + s (1 - t) B + s t C (Osada et al.).
template <typename T>
__device__ __forceinline__ void triangle_point(const ElemGeo<T>& g, T s, T t, T L, T& px, T& py) {
  px = g.x0 + s * (T(1) - t) * min_image(g.x1 - g.x0, L) + s * t * min_image(g.x2 - g.x0, L);
  py = g.y0 + s * (T(1) - t) * (g.y1 - g.y0) + s * t * (g.y2 - g.y0);
}

}  // namespace pdfx

namespace pdfx {

// Fox's projection (Eqs. 64-66): from the element's moments em (layout of the element
// statistics: 4-6 variances, 7-9 <uv>, <uw>, <vw>, 12 scalar variance) and its scalar-
// velocity covariances uphi[3], the factors f_a = alpha_a / s_a of the projected velocity
// U_rho = sum_a f_a (U_a - <U_a>), alpha solving rho_ab alpha_b = rho_a by Cramer's rule;
// all zero when the scalar or a velocity component has no variance or |det| <= 1e-12.
__host__ __device__ inline void fox_factors(const double* em, const double* uphi, double f[3]) {
  f[0] = f[1] = f[2] = 0.0;
  const double var0 = em[4], var1 = em[5], var2 = em[6], vphi = em[12];
  if (!(vphi > 0.0) || !(var0 > 0.0) || !(var1 > 0.0) || !(var2 > 0.0)) return;
  const double s[3] = {sqrt(var0), sqrt(var1), sqrt(var2)}, sphi = sqrt(vphi);
  const double cuv = em[7], cuw = em[8], cvw = em[9];
  const double A[3][3] = {{1.0, cuv / (s[0] * s[1]), cuw / (s[0] * s[2])},
                          {cuv / (s[0] * s[1]), 1.0, cvw / (s[1] * s[2])},
                          {cuw / (s[0] * s[2]), cvw / (s[1] * s[2]), 1.0}};
  const double b[3] = {uphi[0] / (s[0] * sphi), uphi[1] / (s[1] * sphi), uphi[2] / (s[2] * sphi)};
  auto det3 = [](const double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  };
  const double det = det3(A);
  if (!(fabs(det) > 1e-12)) return;
  for (int i = 0; i < 3; ++i) {
    double M[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[r][c] = c == i ? b[r] : A[r][c];
    f[i] = (det3(M) / det) / s[i];
  }
}

}  // namespace pdfx
