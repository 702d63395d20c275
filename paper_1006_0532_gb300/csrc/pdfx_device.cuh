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
  kDiagCapacity, kDiagNonFinite, kDiagHopHist0, kDiagCount = kDiagHopHist0 + 8
};

// Per-element geometry in the element's own frame: vertex A at its node, B and C as
// offsets from A (minimum image across a periodic seam), and 1 / (2 A_e).
template <typename T>
struct __align__(sizeof(T) * 8) ElemGeo {
  T ax, ay, bx, by, cx, cy, inv2a, pad;
};

// Per-element topology: node ids, neighbour across the edge opposite each vertex (-1 =
// boundary), index into the no-slip and free-slip line tables (-1 = none).
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
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
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

// Area coordinates (Eqs. 44-45): N^A and N^C are half the signed cross products pivoted
// at vertex B, lambda = N / A_e, and lambda_B = 1 - lambda_A - lambda_C.
template <typename T>
__device__ __forceinline__ void area_coords(const ElemGeo<T>& g, T x, T y, T L, T& la, T& lb,
                                            T& lc) {
  const T dx = min_image(x - g.ax, L);
  const T dy = y - g.ay;
  const T nA2 = (g.cx - g.bx) * (dy - g.by) - (g.cy - g.by) * (dx - g.bx);
  const T nC2 = (dx - g.bx) * (-g.by) - (dy - g.by) * (-g.bx);
  la = nA2 * g.inv2a;
  lc = nC2 * g.inv2a;
  lb = T(1) - la - lc;
}

}  // namespace pdfx
