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

// Per-element geometry: the coordinates of the three nodes (x in [0, period), the canonical
// image) and 1 / (2 A_e).  FP64 form: plain FP64.  FP32 form: each coordinate as an
// unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits), so that a
// particle's offset from a node, and with it the area coordinates, keep FP32 precision
// relative to the cell rather than to the domain (a first cell 4.6e-5 high at y = 1 is 770
// FP32 spacings of y).
template <typename T>
struct ElemGeo;
template <>
struct __align__(64) ElemGeo<double> {
  double x[3], y[3], inv2a, pad;
};
// The FP32 form also keeps each edge's vector in FP32, from the edge's lower-numbered node
// (its pivot) to the other, computed once in FP64 from the nodes' coordinates: the same
// numbers for both elements of the edge.  code holds, for the edge opposite local vertex k,
// the pivot's local index (bits 3k, 3k + 1) and whether the pivot is the edge's second
// node in counter-clockwise order (bit 3k + 2, the cross product's sign flips).
template <>
struct __align__(16) ElemGeo<float> {
  float xh[3], yh[3], xl[3], yl[3];
  float ex[3], ey[3];
  float inv2a;
  uint32_t code;
  float pad[2];
};

// Per-element topology: node ids, neighbour across the edge opposite each vertex (-1 = a
// boundary edge; -2 - j = a free-slip boundary edge whose own line is entry j of the
// free-slip edge table), index into the no-slip and free-slip line tables (-1 = none).
struct __align__(16) ElemTopo {
  int n0, n1, n2, wall;
  int nb0, nb1, nb2, fslip;
};

// A boundary line: a point on it and the unit normal pointing into the domain (FP32 form:
// the point as hi + lo pairs).
template <typename T>
struct Line;
template <>
struct __align__(32) Line<double> {
  double px, py, nx, ny;
};
template <>
struct __align__(16) Line<float> {
  float px, py, nx, ny, pxl, pyl, pad0, pad1;
};

// A particle position: FP64, or (FP32 form) each coordinate as hi + lo.
template <typename T>
struct Pos;
template <>
struct Pos<double> {
  double x, y;
};
template <>
struct Pos<float> {
  float xh, xl, yh, yl;
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
__host__ __device__ __forceinline__ T min_image(T d, T L) {
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

// (h, l) += d for an FP32 pair: an exact two-sum of the leading parts (Knuth), the error
// added to the trailing part, then renormalised (Dekker's fast two-sum), every operation
// rounded on its own.
__device__ __forceinline__ void pair_add(float& h, float& l, float d) {
  const float s = __fadd_rn(h, d);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  const float t = __fadd_rn(l, e);
  h = __fadd_rn(s, t);
  l = __fsub_rn(t, __fsub_rn(h, s));
}
// The FP32 pair nearest a double (hi = its FP32 rounding, lo = the FP32 rounding of the rest).
__host__ __device__ __forceinline__ void pair_of(double v, float& h, float& l) {
  h = static_cast<float>(v);
  l = static_cast<float>(v - static_cast<double>(h));
}
__host__ __device__ __forceinline__ double pair_value(float h, float l) {
  return static_cast<double>(h) + static_cast<double>(l);
}

// Node k's coordinates as FP64 (the FP32 form's pairs summed).
__device__ __forceinline__ double node_x(const ElemGeo<double>& g, int k) { return g.x[k]; }
__device__ __forceinline__ double node_y(const ElemGeo<double>& g, int k) { return g.y[k]; }
__device__ __forceinline__ double node_x(const ElemGeo<float>& g, int k) { return pair_value(g.xh[k], g.xl[k]); }
__device__ __forceinline__ double node_y(const ElemGeo<float>& g, int k) { return pair_value(g.yh[k], g.yl[k]); }

// Node m minus node k (minimum image in x), in the working precision.
__device__ __forceinline__ void node_vec(const ElemGeo<double>& g, int k, int m, double L, double& ex,
                                         double& ey) {
  ex = min_image(g.x[m] - g.x[k], L);
  ey = g.y[m] - g.y[k];
}
__device__ __forceinline__ void node_vec(const ElemGeo<float>& g, int k, int m, float L, float& ex,
                                         float& ey) {
  ex = __fadd_rn(min_image(__fsub_rn(g.xh[m], g.xh[k]), L), __fsub_rn(g.xl[m], g.xl[k]));
  ey = __fadd_rn(__fsub_rn(g.yh[m], g.yh[k]), __fsub_rn(g.yl[m], g.yl[k]));
}
// Particle minus node k (minimum image in x), in the working precision.
__device__ __forceinline__ void node_rel(const ElemGeo<double>& g, int k, const Pos<double>& P, double L,
                                         double& dx, double& dy) {
  dx = min_image(P.x - g.x[k], L);
  dy = P.y - g.y[k];
}
__device__ __forceinline__ void node_rel(const ElemGeo<float>& g, int k, const Pos<float>& P, float L,
                                         float& dx, float& dy) {
  dx = __fadd_rn(min_image(__fsub_rn(P.xh, g.xh[k]), L), __fsub_rn(P.xl, g.xl[k]));
  dy = __fadd_rn(__fsub_rn(P.yh, g.yh[k]), __fsub_rn(P.yl, g.yl[k]));
}

// Particle minus a point given in FP64 (FP32 form: as the pair (ph, pl)), minimum image in x.
__device__ __forceinline__ double rel_x(const Pos<double>& P, double px, double, double L) {
  return min_image(P.x - px, L);
}
__device__ __forceinline__ double rel_y(const Pos<double>& P, double py, double) { return P.y - py; }
__device__ __forceinline__ float rel_x(const Pos<float>& P, float ph, float pl, float L) {
  return __fadd_rn(min_image(__fsub_rn(P.xh, ph), L), __fsub_rn(P.xl, pl));
}
__device__ __forceinline__ float rel_y(const Pos<float>& P, float ph, float pl) {
  return __fadd_rn(__fsub_rn(P.yh, ph), __fsub_rn(P.yl, pl));
}

// Signed distance of a particle from a boundary line (positive on the domain side).
__device__ __forceinline__ double line_dist(const Line<double>& ln, const Pos<double>& P, double L) {
  return min_image(P.x - ln.px, L) * ln.nx + (P.y - ln.py) * ln.ny;
}
__device__ __forceinline__ float line_dist(const Line<float>& ln, const Pos<float>& P, float L) {
  return rel_x(P, ln.px, ln.pxl, L) * ln.nx + rel_y(P, ln.py, ln.pyl) * ln.ny;
}

// P += (dx, dy): plain FP64, or pair additions.
__device__ __forceinline__ void pos_add(Pos<double>& P, double dx, double dy) {
  P.x += dx;
  P.y += dy;
}
__device__ __forceinline__ void pos_add(Pos<float>& P, float dx, float dy) {
  pair_add(P.xh, P.xl, dx);
  pair_add(P.yh, P.yl, dy);
}
// Eq. 7's move X + U dt + sqrt(2 nu) dW per coordinate (FP64: one expression, as the
// oracle writes it; FP32: the increment added to the pair).
__device__ __forceinline__ void pos_move(Pos<double>& P, double ux, double uy, double dt, double s2nu,
                                         double dWx, double dWy) {
  P.x = P.x + ux * dt + s2nu * dWx;
  P.y = P.y + uy * dt + s2nu * dWy;
}
__device__ __forceinline__ void pos_move(Pos<float>& P, float ux, float uy, float dt, float s2nu,
                                         float dWx, float dWy) {
  pair_add(P.xh, P.xl, ux * dt + s2nu * dWx);
  pair_add(P.yh, P.yl, uy * dt + s2nu * dWy);
}
// Reflection across a line at signed distance d < 0: P -= 2 d n.
__device__ __forceinline__ void pos_reflect(Pos<double>& P, double d, double nx, double ny) {
  P.x -= 2.0 * d * nx;
  P.y -= 2.0 * d * ny;
}
__device__ __forceinline__ void pos_reflect(Pos<float>& P, float d, float nx, float ny) {
  pair_add(P.xh, P.xl, -(2.0f * d * nx));
  pair_add(P.yh, P.yl, -(2.0f * d * ny));
}
// Periodic wrap of x into [0, L).
__device__ __forceinline__ void pos_wrap(Pos<double>& P, double L) { P.x = wrap_period(P.x, L); }
__device__ __forceinline__ void pos_wrap(Pos<float>& P, float L) {
  if (L > 0.0f) {
    if (P.xh < 0.0f) pair_add(P.xh, P.xl, L);
    if (P.xh >= L) pair_add(P.xh, P.xl, -L);
  }
}
__device__ __forceinline__ double pos_x(const Pos<double>& P) { return P.x; }
__device__ __forceinline__ double pos_y(const Pos<double>& P) { return P.y; }
__device__ __forceinline__ double pos_x(const Pos<float>& P) { return pair_value(P.xh, P.xl); }
__device__ __forceinline__ double pos_y(const Pos<float>& P) { return pair_value(P.yh, P.yl); }
__device__ __forceinline__ Pos<double> pos_of(double x, double y, double) { return {x, y}; }
__device__ __forceinline__ Pos<float> pos_of(double x, double y, float) {
  Pos<float> P;
  pair_of(x, P.xh, P.xl);
  pair_of(y, P.yh, P.yl);
  return P;
}

// Separately rounded products (no fused multiply-add).  Every evaluation of an edge's
// cross product then rounds identically, whichever element and slot it is computed for,
// so the two elements sharing an edge always see exactly opposite values (a point on the
// edge is in both), and the FP64 form matches host arithmetic bit for bit.
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }

// (r_b - r_a) x (r_P - r_a) for the edge from local node a to local node b.  Its inputs are
// node b - node a and P - node a, formed from the nodes' own coordinates and the particle's
// alone, so both elements of the edge compute the same value.
template <typename T>
__device__ __forceinline__ T edge_cross(const ElemGeo<T>& g, int a, int b, const Pos<T>& P, T L) {
  T ex, ey, dx, dy;
  node_vec(g, a, b, L, ex, ey);
  node_rel(g, a, P, L, dx, dy);
  return xmul(ex, dy) - xmul(ey, dx);
}

// Twice the signed areas N^A, N^B, N^C (Eqs. 44-45, Fig. 1): for each vertex, the cross
// product of the opposite edge with the vector from one end of that edge to the particle.
// Each edge is pivoted at its lower-numbered node, so the two elements sharing an edge
// evaluate it with identical rounding and opposite signs (watertight point location).
__device__ __forceinline__ void area_cross(const ElemGeo<double>& g, int na, int nb, int nc,
                                           const Pos<double>& P, double L, double& n0, double& n1,
                                           double& n2) {
  n0 = nb < nc ? edge_cross(g, 1, 2, P, L) : -edge_cross(g, 2, 1, P, L);   // edge B -> C
  n1 = nc < na ? edge_cross(g, 2, 0, P, L) : -edge_cross(g, 0, 2, P, L);   // edge C -> A
  n2 = na < nb ? edge_cross(g, 0, 1, P, L) : -edge_cross(g, 1, 0, P, L);   // edge A -> B
}
// FP32 form: the particle's offsets from the three nodes, then each edge's stored vector
// crossed with the offset from its pivot.
__device__ __forceinline__ void area_cross(const ElemGeo<float>& g, int, int, int, const Pos<float>& P,
                                           float L, float& n0, float& n1, float& n2) {
  float dx[3], dy[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) node_rel(g, m, P, L, dx[m], dy[m]);
  float n[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint32_t c = g.code >> (3 * k);
    const int pv = static_cast<int>(c & 3u);
    const float px = pv == 0 ? dx[0] : (pv == 1 ? dx[1] : dx[2]);
    const float py = pv == 0 ? dy[0] : (pv == 1 ? dy[1] : dy[2]);
    const float cr = xmul(g.ex[k], py) - xmul(g.ey[k], px);
    n[k] = (c & 4u) ? -cr : cr;
  }
  n0 = n[0];
  n1 = n[1];
  n2 = n[2];
}

// Area coordinates lambda_k = N^k / A_e (Eqs. 37-38 shapefunction values at the particle).
template <typename T>
__device__ __forceinline__ void area_coords(const ElemGeo<T>& g, int na, int nb, int nc, const Pos<T>& P,
                                            T L, T& la, T& lb, T& lc) {
  area_cross(g, na, nb, nc, P, L, la, lb, lc);
  la *= g.inv2a;
  lb *= g.inv2a;
  lc *= g.inv2a;
}

// Point in the triangle with weights (1 - s) A + s (1 - t) B + s t C (Osada et al.).
__device__ __forceinline__ Pos<double> triangle_point(const ElemGeo<double>& g, double s, double t, double L) {
  Pos<double> P;
  P.x = g.x[0] + s * (1.0 - t) * min_image(g.x[1] - g.x[0], L) + s * t * min_image(g.x[2] - g.x[0], L);
  P.y = g.y[0] + s * (1.0 - t) * (g.y[1] - g.y[0]) + s * t * (g.y[2] - g.y[0]);
  return P;
}
__device__ __forceinline__ Pos<float> triangle_point(const ElemGeo<float>& g, float s, float t, float L) {
  float bx, by, cx, cy;
  node_vec(g, 0, 1, L, bx, by);
  node_vec(g, 0, 2, L, cx, cy);
  Pos<float> P{g.xh[0], g.xl[0], g.yh[0], g.yl[0]};
  pos_add(P, s * (1.0f - t) * bx + s * t * cx, s * (1.0f - t) * by + s * t * cy);
  return P;
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
