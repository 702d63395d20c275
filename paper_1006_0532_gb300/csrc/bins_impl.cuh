// Per-element statistics and conditional means for elements of up to 768 particles, one
// thread block per entry of the plan's tile lists (three size classes, launched as parallel
// stream branches), and of 769..1024 from the plan's large-element list; larger elements go
// through the block kernel in k_stats.cu.  The chunk-sort tile below serves every class of
// Fox's projection; the bucket-rank tile further down every class of the hierarchical
// bins.
//
// Sect. 3.5 / Appendix A: the element's particles are sorted by (u, id); the level-1 groups
// (positions with equal floor(g1 p / N)) are sorted by (v, id), the level-2 groups by
// (w, id), and position p of the final order gets bin floor(G p / N).  One level: every
// group is cut into chunks of 32 consecutive positions, a warp sorts a chunk in registers
// (bitonic network, one key per lane), and a key's rank in its group is its rank in its
// chunk plus, for every other chunk of the group, the number of smaller keys found by a
// binary search of that sorted chunk.  Exact keys are distinct (the particle id is part of
// the key), so the ranks are a permutation and the new order is written by scatter.  A
// level first runs on the value bits alone (32-bit keys in the FP32 form, 64-bit in the
// FP64 form); ties are detected exactly (equal neighbours in a sorted chunk, an equal key
// at the end of a search), and an element with a tie at that level runs it again with the
// exact (value, id) keys, which rewrites every position.
// Sect. 3.3, Eqs. 35-36: element means, then central moments about them, summed by one
// warp in the final order (deterministic); the FP32 form accumulates compensated FP32 per
// lane and combines lanes as FP32 value/error pairs, the FP64 form sums in FP64.  The 13
// outputs are then formed in FP64 one per lane.
// Fox's projection (Eqs. 64-66, cond_mode 1) is a compile-time variant of the kernel: the
// particle-id order fixes the order of the moment sums, the moments give the projection
// factors, and one more level orders the whole element by the projected velocity (pairwise
// merge rounds of sorted runs rank these whole-element levels); an element whose factors
// are all zero keeps the id order, which is then its (U_rho, id) order.  The hierarchical
// variant carries none of its members or code.
#pragma once
#include <initializer_list>

#include "pdfx_internal.h"

namespace pdfx {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------------------
// Keys: (order-preserving value bits, particle id).  Particle ids are below 2^28 (checked
// by the host).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ord_bits(float x) {
  const uint32_t b = __float_as_uint(x + 0.0f);   // -0 -> +0: equal values tie
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint64_t ord_bits(double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x + 0.0));
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

struct K32 {   // FP32 form, value bits
  uint32_t k;
};
struct K64 {   // FP32 form: value (32 bits) << 28 | id (28 bits); FP64 form: value bits
  uint64_t k;
};
struct K96 {   // FP64 form: value, id
  uint64_t hi;
  uint32_t lo;
};

__device__ __forceinline__ bool kless(const K32& a, const K32& b) { return a.k < b.k; }
__device__ __forceinline__ bool kless(const K64& a, const K64& b) { return a.k < b.k; }
__device__ __forceinline__ bool kless(const K96& a, const K96& b) {
  return (a.hi < b.hi) | ((a.hi == b.hi) & (a.lo < b.lo));
}
__device__ __forceinline__ bool keq(const K32& a, const K32& b) { return a.k == b.k; }
__device__ __forceinline__ bool keq(const K64& a, const K64& b) { return a.k == b.k; }
__device__ __forceinline__ bool keq(const K96& a, const K96& b) { return (a.hi == b.hi) & (a.lo == b.lo); }
__device__ __forceinline__ K32 ksel(bool c, const K32& a, const K32& b) { return {c ? a.k : b.k}; }
__device__ __forceinline__ K64 ksel(bool c, const K64& a, const K64& b) { return {c ? a.k : b.k}; }
__device__ __forceinline__ K96 ksel(bool c, const K96& a, const K96& b) {
  return {c ? a.hi : b.hi, c ? a.lo : b.lo};
}
__device__ __forceinline__ K32 kshfl(const K32& a, int m) { return {__shfl_xor_sync(kFull, a.k, m)}; }
__device__ __forceinline__ K64 kshfl(const K64& a, int m) { return {__shfl_xor_sync(kFull, a.k, m)}; }
__device__ __forceinline__ K96 kshfl(const K96& a, int m) {
  return {__shfl_xor_sync(kFull, a.hi, m), __shfl_xor_sync(kFull, a.lo, m)};
}
__device__ __forceinline__ K32 kdown(const K32& a) { return {__shfl_down_sync(kFull, a.k, 1)}; }
__device__ __forceinline__ K64 kdown(const K64& a) { return {__shfl_down_sync(kFull, a.k, 1)}; }
__device__ __forceinline__ K96 kdown(const K96& a) {
  return {__shfl_down_sync(kFull, a.hi, 1), __shfl_down_sync(kFull, a.lo, 1)};
}
__device__ __forceinline__ void pad_key(K32& k) { k.k = ~0u; }
__device__ __forceinline__ void pad_key(K64& k) { k.k = ~0ull; }
__device__ __forceinline__ void pad_key(K96& k) { k.hi = ~0ull; k.lo = ~0u; }

// Key of a particle at one level: value bits only (fast pass) or (value, id) (exact pass).
template <typename T, bool EXACT> struct KeyPolicy;
template <> struct KeyPolicy<float, false> {
  using K = K32;
  __device__ __forceinline__ static K make(float v, const uint32_t*, int32_t) { return {ord_bits(v)}; }
};
template <> struct KeyPolicy<float, true> {
  using K = K64;
  __device__ __forceinline__ static K make(float v, const uint32_t* pid, int32_t q) {
    return {(static_cast<uint64_t>(ord_bits(v)) << 28) | (pid[q] & 0x0fffffffu)};
  }
};
template <> struct KeyPolicy<double, false> {
  using K = K64;
  __device__ __forceinline__ static K make(double v, const uint32_t*, int32_t) { return {ord_bits(v)}; }
};
template <> struct KeyPolicy<double, true> {
  using K = K96;
  __device__ __forceinline__ static K make(double v, const uint32_t* pid, int32_t q) {
    return {ord_bits(v), pid[q]};
  }
};

// Sorted chunk keys in shared memory.
template <typename K, int N> struct KeyArr;
template <int N>
struct KeyArr<K32, N> {
  uint32_t k[N];
  __device__ __forceinline__ K32 get(int i) const { return {k[i]}; }
  __device__ __forceinline__ void set(int i, const K32& v) { k[i] = v.k; }
};
template <int N>
struct KeyArr<K64, N> {
  uint64_t k[N];
  __device__ __forceinline__ K64 get(int i) const { return {k[i]}; }
  __device__ __forceinline__ void set(int i, const K64& v) { k[i] = v.k; }
};
template <int N>
struct KeyArr<K96, N> {
  uint64_t hi[N];
  uint32_t lo[N];
  __device__ __forceinline__ K96 get(int i) const { return {hi[i], lo[i]}; }
  __device__ __forceinline__ void set(int i, const K96& v) { hi[i] = v.hi; lo[i] = v.lo; }
};

// Ascending bitonic sort of one key (and its payload) per lane.  Padding keys are the
// maximum and sort above every real key (ties with them only matter for the fast pass,
// whose tie test looks at real lanes only).
template <typename K>
__device__ __forceinline__ void warp_sort32(K& k, int32_t& v, int lane) {
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const K o = kshfl(k, j);
      const int32_t ov = __shfl_xor_sync(kFull, v, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & kk) == 0);
      const bool take = kless(o, k) == keep_min;
      k = ksel(take, o, k);
      v = take ? ov : v;
    }
  }
}

// Number of keys below k in a sorted, padded chunk of 32 keys starting at base; eq tells
// whether the chunk holds a key equal to k (the first key not below k is the last one read).
template <typename Arr, typename K>
__device__ __forceinline__ int count_below(const Arr& s, int base, const K& k, bool& eq) {
  int pos = 0;
#pragma unroll
  for (int st = 16; st >= 1; st >>= 1) pos += kless(s.get(base + pos + st - 1), k) ? st : 0;
  const K v = s.get(base + pos);
  const bool lt = kless(v, k);
  eq = !lt && keq(v, k);
  return pos + (lt ? 1 : 0);
}

// Compensated (Kahan) accumulation for the FP32 form; plain for FP64.  warp_pair() sums
// the 32 lanes' accumulators into a value/error pair (every lane gets the same pair).
template <typename T>
struct Acc;
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s - c; }
  __device__ __forceinline__ static float err(const Acc& a) { return a.c; }
  // value/error pairs: an exact two-sum of the leading parts, errors added, renormalised.
  // Both lanes of a pair take the lower lane's pair as the first operand, so every lane ends
  // with the same bits.
  __device__ __forceinline__ void warp_pair(float& hv, float& lv) const {
    float h = s, l = -c;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(kFull, h, o), ol = __shfl_xor_sync(kFull, l, o);
      const bool first = (lane & o) == 0;
      const float ah = first ? h : oh, bh = first ? oh : h;
      const float al = first ? l : ol, bl = first ? ol : l;
      const float sh = ah + bh;
      const float bb = sh - ah;
      const float se = (ah - (sh - bb)) + (bh - bb);
      const float lo = se + (al + bl);
      h = sh + lo;
      l = lo - (h - sh);
    }
    hv = h;
    lv = l;
  }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ static double err(const Acc&) { return 0.0; }
  __device__ __forceinline__ void warp_pair(double& hv, double& lv) const {
    double v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    hv = v;
    lv = 0.0;
  }
};

// 1/n in FP64 for the element sizes of the tiles (n <= 1024), correctly rounded at compile
// time: the same bits as a run-time FP64 division, without its long dependent sequence on
// this GPU's narrow FP64 pipe.
struct RecipTable {
  double v[1025];
  constexpr RecipTable() : v() {
    for (int i = 1; i <= 1024; ++i) v[i] = 1.0 / i;
  }
};
__constant__ RecipTable c_recip = RecipTable();
__device__ __forceinline__ double recip_n(int n) { return n > 0 ? c_recip.v[n] : 0.0; }

// floor(x / d) for 0 <= x < 2^18 + 2^8 and 1 <= d <= 1024 with inv = 1/d in FP32: the
// quotient is at most 1025, so the two roundings of (x + 1/2) inv err by at most
// 1025 * 2^-23 < 2^-12 < 1/(2d), the distance from (x + 1/2)/d to the nearest integer.
__device__ __forceinline__ int fdiv(int x, float inv) {
  return __float2int_rz((static_cast<float>(x) + 0.5f) * inv);
}

// First position of group g of G over n positions: ceil(g n / G) = floor((g n + G - 1) / G)
// (g <= G <= 256, n <= 1024), invG = 1/G.
__device__ __forceinline__ int group_start(int g, int n, int G, float invG) {
  return fdiv(g * n + G - 1, invG);
}

// Moment outputs, one per lane: em[c] = X + Y/N - (Z/N)(W/N), X a shift value, Y a sum of
// d or of a product of d, Z and W sums of d; four bits per lane, 15 = term absent.
// Sums 0..4: d of u, v, w, omega, psi; 5..11: uu, vv, ww, uv, uw, vw, psi psi.
// Outputs: 0 N, 1-3 means of u, v, w, 4-6 variances, 7-9 <uv>, <uw>, <vw>, 10 mean omega,
// 11 mean psi, 12 variance of psi.
constexpr uint64_t pack13(std::initializer_list<int> v) {
  uint64_t r = 0;
  int i = 0;
  for (int x : v) r |= static_cast<uint64_t>(x & 15) << (4 * i++);
  return r;
}
constexpr uint64_t kMomX = pack13({15, 0, 1, 2, 15, 15, 15, 15, 15, 15, 3, 4, 15});
constexpr uint64_t kMomY = pack13({15, 0, 1, 2, 5, 6, 7, 8, 9, 10, 3, 4, 11});
constexpr uint64_t kMomZ = pack13({15, 15, 15, 15, 0, 1, 2, 0, 0, 1, 15, 15, 4});
constexpr uint64_t kMomW = pack13({15, 15, 15, 15, 0, 1, 2, 1, 2, 2, 15, 15, 4});
__device__ __forceinline__ int mom_nib(uint64_t tab, int c) {
  return static_cast<int>((tab >> (4 * c)) & 15u);
}

// Source of Fox's projected velocity (Eq. 64): factors f_a, means <U_a>, component arrays.
template <typename T>
struct ProjSrc {
  double f[3], m[3];
  const T* c[3];
};

// Members only Fox's projection uses: an empty base of the hierarchical kernels' tile.
template <typename T, bool FOX>
struct TileFox {};
template <typename T>
struct TileFox<T, true> {
  double mhx[3], mlx[3];            // sums of d_a d_phi (value/error pairs), Eq. 66
  double em[kNS];                   // the element's statistics
  double fox[6];                    // projection factors f_a and means <U_a> (Eqs. 64-66)
  ProjSrc<T> proj;                  // the projected velocity's source
};

// Shared tile of one element.  Chunk tables are needed only when groups exceed 32
// positions: then there are fewer than CAP/32 groups and fewer than 2 CAP/32 chunks.
template <typename T, int CAP, bool FOX>
struct Tile : TileFox<T, FOX> {
  static constexpr int kChunks = 2 * CAP / 32;
  int32_t ord[CAP];                 // particle slots in the current order
  int32_t nord[CAP];                // the next level's order
  union {                           // sorted chunks (padded to 32), fast or exact keys
    KeyArr<typename KeyPolicy<T, false>::K, kChunks * 32> fast;
    KeyArr<typename KeyPolicy<T, true>::K, kChunks * 32> exact;
  } sk;
  int32_t spay[kChunks * 32];       // their slots
  int tie[3];                       // a tie was found at level l (fast pass)
  int32_t gfc[CAP / 32 + 1];        // first chunk of each group
  uint8_t cg[kChunks];              // group of each chunk
  double mh[12], ml[12], msh[5];    // moment sums (value/error pairs) and shift values
  int n_gathered;
};

// Number of keys below k in the sorted run s[base, base + len), len <= R <= RMAX (powers of
// two); eq tells whether the run holds a key equal to k.
template <int RMAX, typename Arr, typename K>
__device__ __forceinline__ int run_count_below(const Arr& s, int base, int len, int R, const K& k,
                                               bool& eq) {
  int pos = 0;
#pragma unroll
  for (int st = RMAX; st >= 1; st >>= 1) {
    if (st > R) continue;
    const int np = pos + st;
    if (np <= len && kless(s.get(base + np - 1), k)) pos = np;
  }
  eq = pos < len && keq(s.get(base + pos), k);
  return pos;
}

// One sorting level: the groups of the current order (Gprev groups over n positions, the
// largest of M) are each ordered by the level's key into nxt.  With M <= 32 a group is one
// warp sort; otherwise chunks of 32 (tables t.gfc, t.cg) are sorted first.  A key's rank
// is its chunk rank plus its count in every other chunk of its group; with MERGE, in groups
// above 256 positions sorted runs (32, 64, 128, ... positions of a group) are merged
// pairwise instead (measured faster only where two whole-element levels are ranked), a key's
// place in the merged run being its place in its own run plus its count in the partner
// run, with the keys at their group positions in one half of sk and spay and written to
// the other half (n <= CAP positions each), the last round into nxt.  The fast pass (EXACT
// false) sets *tie when two real keys of a group are equal; until the first round in which
// two equal keys meet the runs are exact, so that round's search finds the tie.  Its places
// never leave the group or run pair, so every index stays within bounds either way.
template <typename T, int CAP, int THREADS, bool EXACT, bool MERGE, bool FOX, typename Arr,
          typename ValFn>
__device__ void sort_level(const StatsArgs<T>& a, Tile<T, CAP, FOX>& t, Arr& sk, const int32_t* cur,
                           int32_t* nxt, const ValFn& val, int n, int Gprev, int M, float invG,
                           int* tie) {
  using P = KeyPolicy<T, EXACT>;
  using K = typename P::K;
  constexpr int W = THREADS / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool found = false;
  if (M <= 32) {
    for (int c = warp; c < Gprev; c += W) {
      const int gs = group_start(c, n, Gprev, invG), len = group_start(c + 1, n, Gprev, invG) - gs;
      K k;
      int32_t q = -1;
      if (lane < len) {
        q = cur[gs + lane];
        k = P::make(val(q), a.p.pid, q);
      } else {
        pad_key(k);
      }
      warp_sort32(k, q, lane);
      if (!EXACT) {
        const K nk = kdown(k);   // every lane takes part in the shuffle
        found |= (lane + 1 < len) && keq(k, nk);
      }
      if (lane < len) nxt[gs + lane] = q;
    }
  } else if (MERGE && M > 256) {
    const int nchunks = t.gfc[Gprev];
    for (int c = warp; c < nchunks; c += W) {
      const int gi = t.cg[c];
      const int gs = group_start(gi, n, Gprev, invG), ge = group_start(gi + 1, n, Gprev, invG);
      const int cs = gs + 32 * (c - t.gfc[gi]), len = min(32, ge - cs);
      K k;
      int32_t q = -1;
      if (lane < len) {
        q = cur[cs + lane];
        k = P::make(val(q), a.p.pid, q);
      } else {
        pad_key(k);
      }
      warp_sort32(k, q, lane);
      if (!EXACT) {
        const K nk = kdown(k);   // every lane takes part in the shuffle
        found |= (lane + 1 < len) && keq(k, nk);
      }
      if (lane < len) {
        sk.set(cs + lane, k);
        t.spay[cs + lane] = q;
      }
    }
    __syncthreads();
    int src = 0;
    for (int lgR = 5; (1 << lgR) < M; ++lgR) {
      const int R = 1 << lgR;
      const bool last = 2 * R >= M;
      const int dst = CAP - src;
      for (int c = warp; c < nchunks; c += W) {
        const int gi = t.cg[c];
        const int gs = group_start(gi, n, Gprev, invG), ge = group_start(gi + 1, n, Gprev, invG);
        const int li = 32 * (c - t.gfc[gi]) + lane;    // position in the group
        if (li < ge - gs) {
          const int m = li >> lgR, ps = (m ^ 1) << lgR;   // own run, partner run start
          const int plen = min(R, ge - gs - ps);        // <= 0: no partner
          const K k = sk.get(src + gs + li);
          bool eq = false;
          const int cnt = plen > 0 ? run_count_below<CAP / 2>(sk, src + gs + ps, plen, R, k, eq) : 0;
          if (!EXACT) found |= eq;
          const int np = ((m & ~1) << lgR) + (li - (m << lgR)) + cnt;
          const int32_t q = t.spay[src + gs + li];
          if (last) {
            nxt[gs + np] = q;
          } else {
            sk.set(dst + gs + np, k);
            t.spay[dst + gs + np] = q;
          }
        }
      }
      __syncthreads();
      src = dst;
    }
  } else {
    const int nchunks = t.gfc[Gprev];
    for (int c = warp; c < nchunks; c += W) {
      const int gi = t.cg[c];
      const int gs = group_start(gi, n, Gprev, invG), ge = group_start(gi + 1, n, Gprev, invG);
      const int cs = gs + 32 * (c - t.gfc[gi]), len = min(32, ge - cs);
      K k;
      int32_t q = -1;
      if (lane < len) {
        q = cur[cs + lane];
        k = P::make(val(q), a.p.pid, q);
      } else {
        pad_key(k);
      }
      warp_sort32(k, q, lane);
      if (!EXACT) {
        const K nk = kdown(k);   // every lane takes part in the shuffle
        found |= (lane + 1 < len) && keq(k, nk);
      }
      sk.set(c * 32 + lane, k);
      t.spay[c * 32 + lane] = q;
    }
    __syncthreads();
    for (int c = warp; c < nchunks; c += W) {
      const int gi = t.cg[c];
      const int gs = group_start(gi, n, Gprev, invG), ge = group_start(gi + 1, n, Gprev, invG);
      const int c0 = t.gfc[gi], c1 = t.gfc[gi + 1];
      const int cs = gs + 32 * (c - c0), len = min(32, ge - cs);
      const K k = sk.get(c * 32 + lane);
      int r = lane;
      bool eq_any = false;
      // Unroll factors here and in the gather, moment and bin loops are measured: the
      // compiler's default unrolling grows the kernel past what its instruction cache holds
      // (2-5% slower per step).
#pragma unroll 1
      for (int c2 = c0; c2 < c1; ++c2) {
        if (c2 == c) continue;
        bool eq;
        r += count_below(sk, c2 * 32, k, eq);
        eq_any |= eq;
      }
      if (!EXACT) found |= eq_any && lane < len;
      if (lane < len) nxt[gs + r] = t.spay[c * 32 + lane];
    }
  }
  if (!EXACT) {
    const bool any = __any_sync(kFull, found);   // every lane takes part
    if (any && lane == 0) *tie = 1;
  }
}

// Key value of a particle at one level: a velocity component, or Fox's projected velocity
// sum_a f_a (U_a - <U_a>) (Eq. 64, formed in FP64 and rounded to the state precision) from
// the factors, means and component arrays in shared memory.
template <typename T>
struct ArrVal {
  const T* v;
  __device__ __forceinline__ T operator()(int32_t q) const { return v[q]; }
};
// Eq. 64's projected velocity from the factors f_a and the means m_a, summed left to right
// with every operation rounded on its own (no fused multiply-add): in FP64 the oracle's bits.
template <typename T>
__device__ __forceinline__ T fox_key(const double* f, const double* m, T u, T v, T w) {
  const double a = __dmul_rn(f[0], __dsub_rn(static_cast<double>(u), m[0]));
  const double b = __dmul_rn(f[1], __dsub_rn(static_cast<double>(v), m[1]));
  const double c = __dmul_rn(f[2], __dsub_rn(static_cast<double>(w), m[2]));
  return static_cast<T>(__dadd_rn(__dadd_rn(a, b), c));
}
// The sort value of a particle id: a positive normal number whose bits are 2^23 (FP32) or
// 2^52 (FP64) plus the id, so that values are distinct and ordered as the ids.
template <typename T>
struct PidVal;
template <>
struct PidVal<float> {
  const uint32_t* pid;
  __device__ __forceinline__ float operator()(int32_t q) const { return __uint_as_float(0x00800000u + pid[q]); }
};
template <>
struct PidVal<double> {
  const uint32_t* pid;
  __device__ __forceinline__ double operator()(int32_t q) const {
    return __longlong_as_double(static_cast<long long>(0x0010000000000000ull + pid[q]));
  }
};
template <typename T>
struct ProjVal {
  const ProjSrc<T>* s;
  __device__ __forceinline__ T operator()(int32_t q) const {
    return fox_key<T>(s->f, s->m, s->c[0][q], s->c[1][q], s->c[2][q]);
  }
};

// Sect. 3.3, Eqs. 35-36, by warp 0 in the order cur: sums of d = x - x_0 and of products of
// d in precision A (each product rounded on its own, never fused into the sum, so that every
// tile kernel forms the same sums bit for bit), x_0 the first particle of the order; mean = x_0 + S1/N, central =
// S2/N - (S1/N)^2; lanes combine as value/error pairs (FP32) or in FP64, then the 13
// outputs are formed in FP64, one per lane.  Inlined: as an out-of-line call it measured
// slower (its spills and the call outweigh the spills it saves in the sorting loops).
// FOX: also the sums of d_a d_phi, then <u_a phi'> and the factors of Eqs. 65-66.
template <typename A, bool FOX, typename T, typename TileT, typename I>
__device__ __forceinline__ void element_moments(const T* __restrict__ pu, const T* __restrict__ pv,
                                                const T* __restrict__ pw, const T* __restrict__ pom,
                                                const T* __restrict__ ppsi, double* emom_e,
                                                int32_t* gbin_e, TileT& t,
                                                const I* cur, int n, int g0, int g1, int g2) {
  const int lane = threadIdx.x & 31;
  A sh[5] = {A(0), A(0), A(0), A(0), A(0)};
  if (n > 0) {
    const int q0 = cur[0];
    sh[0] = A(pu[q0]); sh[1] = A(pv[q0]); sh[2] = A(pw[q0]);
    sh[3] = A(pom[q0]); sh[4] = A(ppsi[q0]);
  }
  Acc<A> m[12];
  Acc<A> mx[3];   // FOX only
#pragma unroll 2
  for (int p = lane; p < n; p += 32) {
    const int q = cur[p];
    const A du = A(pu[q]) - sh[0], dv = A(pv[q]) - sh[1], dw = A(pw[q]) - sh[2];
    const A dom = A(pom[q]) - sh[3], dp = A(ppsi[q]) - sh[4];
    m[0].add(du); m[1].add(dv); m[2].add(dw); m[3].add(dom); m[4].add(dp);
    m[5].add(xmul(du, du)); m[6].add(xmul(dv, dv)); m[7].add(xmul(dw, dw));
    m[8].add(xmul(du, dv)); m[9].add(xmul(du, dw)); m[10].add(xmul(dv, dw));
    m[11].add(xmul(dp, dp));
    if constexpr (FOX) { mx[0].add(xmul(du, dp)); mx[1].add(xmul(dv, dp)); mx[2].add(xmul(dw, dp)); }
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    A h, l;
    m[c].warp_pair(h, l);
    if (lane == c) { t.mh[c] = h; t.ml[c] = l; }
  }
  if constexpr (FOX) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A h, l;
      mx[c].warp_pair(h, l);
      if (lane == c) { t.mhx[c] = h; t.mlx[c] = l; }
    }
  }
  if (lane < 5)
    t.msh[lane] = lane == 0 ? sh[0] : lane == 1 ? sh[1] : lane == 2 ? sh[2] : lane == 3 ? sh[3] : sh[4];
  __syncwarp();
  if (lane < kNS) {
    const double inv = recip_n(n);
    const int ix = mom_nib(kMomX, lane), iy = mom_nib(kMomY, lane);
    const int iz = mom_nib(kMomZ, lane), iw = mom_nib(kMomW, lane);
    double v = ix < 15 ? t.msh[ix] : 0.0;
    if (iy < 15) v += (t.mh[iy] + t.ml[iy]) * inv;
    if (iz < 15) {
      const double z = (t.mh[iz] + t.ml[iz]) * inv;
      const double w = (t.mh[iw] + t.ml[iw]) * inv;
      v -= z * w;
    }
    if (lane == 0) v = static_cast<double>(n);
    else if (n == 0) v = 0.0;
    emom_e[lane] = v;
    if constexpr (FOX) t.em[lane] = v;
  }
  if (lane < 3) gbin_e[lane] = lane == 0 ? g0 : lane == 1 ? g1 : g2;
  if constexpr (FOX) {
    __syncwarp();
    if (lane == 0) {
      // <u_a phi'> = S(d_a d_phi)/N - (S d_a/N)(S d_phi/N); then Eqs. 65-66
      const double inv = recip_n(n);
      const double sp = (t.mh[4] + t.ml[4]) * inv;
      double uphi[3], f[3];
      for (int k = 0; k < 3; ++k)
        uphi[k] = (t.mhx[k] + t.mlx[k]) * inv - (t.mh[k] + t.ml[k]) * inv * sp;
      fox_factors(t.em, uphi, f);
      for (int k = 0; k < 3; ++k) { t.fox[k] = f[k]; t.fox[3 + k] = t.em[1 + k]; }
    }
  }
}

// Moments in the state precision (FP32 form: compensated) or, with acc64 in the FP32
// form, in FP64.
template <typename T, int CAP, bool FOX>
__device__ __forceinline__ void element_moments_of(const StatsArgs<T>& a, Tile<T, CAP, FOX>& t,
                                                   const int32_t* cur, int n, int e,
                                                   const int (&g)[3]) {
  double* const emom_e = a.emom + static_cast<size_t>(kNS) * e;
  int32_t* const gbin_e = a.gbin + 3 * e;
  if (sizeof(T) == 4 && a.acc64)
    element_moments<double, FOX>(a.p.u, a.p.v, a.p.w, a.p.om, a.p.psi, emom_e, gbin_e, t, cur, n,
                                 g[0], g[1], g[2]);
  else
    element_moments<T, FOX>(a.p.u, a.p.v, a.p.w, a.p.om, a.p.psi, emom_e, gbin_e, t, cur, n,
                            g[0], g[1], g[2]);
}

// Chunk tables of one level (warp 0): the first chunk of each of the Gprev groups over n
// positions (Gprev < n / 32 <= CAP / 32 <= 32 groups, one lane each) and the group of each
// chunk.
template <typename T, int CAP, bool FOX>
__device__ __forceinline__ void chunk_tables(Tile<T, CAP, FOX>& t, int n, int Gprev, float invG, int lane) {
  int nch = 0;
  if (lane < Gprev) nch = (group_start(lane + 1, n, Gprev, invG) - group_start(lane, n, Gprev, invG) + 31) >> 5;
  int incl = nch;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane < Gprev) {
    t.gfc[lane] = incl - nch;
    for (int j = 0; j < nch; ++j) t.cg[incl - nch + j] = static_cast<uint8_t>(lane);
  }
  if (lane == Gprev - 1) t.gfc[Gprev] = incl;
}

// One element of N <= CAP particles (list size after redistribution) by a block of THREADS.
template <typename T, int CAP, int THREADS, bool FOX>
__device__ void element_tile(const StatsArgs<T>& a, Tile<T, CAP, FOX>& t, int e, int N, int moves) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;

  // gather: the element's list minus particles moved out, plus those moved in
  if (threadIdx.x == 0) t.n_gathered = 0;
  if (threadIdx.x < 3) t.tie[threadIdx.x] = 0;
  __syncthreads();
  {
    const int32_t o = a.off[e], c = a.cnt[e];
    if (!moves) {
      // no particle moved: every list entry is the element's, entry j goes to position j
#pragma unroll 1
      for (int j = threadIdx.x; j < c && j < CAP; j += THREADS) t.ord[j] = a.idx[o + j];
      if (threadIdx.x == 0) t.n_gathered = c;
    } else {
#pragma unroll 1
      for (int j0 = warp * 32; j0 < c; j0 += THREADS) {
        const int j = j0 + lane;
        int32_t q = -1;
        if (j < c) {
          q = a.idx[o + j];
          if (a.p.elem[q] != e) q = -1;
        }
        const unsigned keep = __ballot_sync(kFull, q >= 0);
        int base = 0;
        if (lane == 0 && keep) base = atomicAdd(&t.n_gathered, __popc(keep));
        base = __shfl_sync(kFull, base, 0);
        const int at = base + __popc(keep & below);
        if (q >= 0 && at < CAP) t.ord[at] = q;
      }
    }
    if (moves) {
      const int32_t gn = a.gain[e], g0 = a.goff[e];
#pragma unroll 1
      for (int j0 = warp * 32; j0 < gn; j0 += THREADS) {
        const int j = j0 + lane;
        int32_t q = j < gn ? a.movers[g0 + j] : -1;
        if (q >= a.np) q = -1;
        const unsigned keep = __ballot_sync(kFull, q >= 0);
        int base = 0;
        if (lane == 0 && keep) base = atomicAdd(&t.n_gathered, __popc(keep));
        base = __shfl_sync(kFull, base, 0);
        const int at = base + __popc(keep & below);
        if (q >= 0 && at < CAP) t.ord[at] = q;
      }
    }
  }
  __syncthreads();
  int n = t.n_gathered;
  if (n != N && threadIdx.x == 0) atomicCAS(a.err, 0, PDFX_ERR_CAPACITY);
  n = min(min(n, N), CAP);

  // effective bins (reading of Sect. 3.5): g_l = max(1, min(b_l, n / (g_1..g_{l-1} min_per_bin)));
  // Fox's projection: max(1, min(fox_bins, n / min_per_bin)) intervals
  int g[3];
  if constexpr (FOX) {
    int nc = n / a.min_per_bin;
    if (a.fox_bins < nc) nc = a.fox_bins;
    g[0] = nc < 1 ? 1 : nc;
    g[1] = g[2] = 1;
  } else {
    int Gp = 1;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int capl = n / (Gp * a.min_per_bin);
      int gl = a.bins[l] < capl ? a.bins[l] : capl;
      if (gl < 1) gl = 1;
      g[l] = gl;
      Gp *= gl;
    }
  }

  int32_t* cur = t.ord;
  int32_t* nxt = t.nord;
  if constexpr (!FOX) {
    // levels by (u, id), (v, id), (w, id) within the groups of the previous level
    int Gprev = 1;
    if (n > 0) {
#pragma unroll 1
      for (int l = 0; l < 3; ++l) {
        if (l > 0 && g[l] <= 1) continue;
        const ArrVal<T> val{l == 0 ? a.p.u : (l == 1 ? a.p.v : a.p.w)};
        const int M = (n + Gprev - 1) / Gprev;   // largest group
        const float invG = 1.0f / static_cast<float>(Gprev);
        if (M > 32 && warp == 0) chunk_tables(t, n, Gprev, invG, lane);
        __syncthreads();
        sort_level<T, CAP, THREADS, false, false>(a, t, t.sk.fast, cur, nxt, val, n, Gprev, M, invG,
                                                  &t.tie[l]);
        __syncthreads();
        if (t.tie[l]) {
          sort_level<T, CAP, THREADS, true, false>(a, t, t.sk.exact, cur, nxt, val, n, Gprev, M,
                                                   invG, nullptr);
          __syncthreads();
        }
        int32_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
        Gprev *= g[l];
      }
    }
    // moments (warp 0) in the final order
    if (warp == 0) element_moments_of(a, t, cur, n, e, g);
  } else {
    // Fox's projection (Eqs. 64-66): the particle-id order fixes the order of the moment
    // sums; the moments give the factors; then one level over the whole element by U_rho
    auto whole_level = [&](const auto& val, int ti) {
      const float invG = 1.0f;
      if (n > 32 && warp == 0) chunk_tables(t, n, 1, invG, lane);
      __syncthreads();
      sort_level<T, CAP, THREADS, false, true>(a, t, t.sk.fast, cur, nxt, val, n, 1, n, invG,
                                               &t.tie[ti]);
      __syncthreads();
      if (t.tie[ti]) {
        sort_level<T, CAP, THREADS, true, true>(a, t, t.sk.exact, cur, nxt, val, n, 1, n, invG,
                                                nullptr);
        __syncthreads();
      }
      int32_t* tmp = cur;
      cur = nxt;
      nxt = tmp;
    };
    if (n > 0) whole_level(PidVal<T>{a.p.pid}, 0);
    if (warp == 0) element_moments_of(a, t, cur, n, e, g);   // an empty element writes zeros
    if (n > 0) {
      if (threadIdx.x < 3) {
        const int k = threadIdx.x;
        t.proj.f[k] = t.fox[k];
        t.proj.m[k] = t.fox[3 + k];
        t.proj.c[k] = k == 0 ? a.p.u : (k == 1 ? a.p.v : a.p.w);
      }
      __syncthreads();
      // all factors zero (a constant scalar, or a degenerate correlation system): every
      // U_rho is 0 and the order of (U_rho, id) is the id order the element already has
      if (!(t.fox[0] == 0.0 && t.fox[1] == 0.0 && t.fox[2] == 0.0)) whole_level(ProjVal<T>{&t.proj}, 1);
    }
  }
  const int G = g[0] * g[1] * g[2];

  // Appendix A bins: conditional scalar means over the final order's bins
  double* vc = a.vcce + static_cast<size_t>(a.G) * e;
  const float invGb = 1.0f / static_cast<float>(G);
  for (int i = threadIdx.x; i < a.G; i += THREADS) {
    double mval = 0.0;
    if (i < G && n > 0) {
      const int b0 = group_start(i, n, G, invGb), b1 = group_start(i + 1, n, G, invGb);
      if (sizeof(T) == 4 && a.acc64) {
        double sum = 0.0;
#pragma unroll 1
        for (int p = b0; p < b1; ++p) sum += static_cast<double>(a.p.psi[cur[p]]);
        mval = sum / static_cast<double>(b1 - b0);
      } else {
        Acc<T> sum;
#pragma unroll 1
        for (int p = b0; p < b1; ++p) sum.add(a.p.psi[cur[p]]);
        mval = static_cast<double>(sum.value() / static_cast<T>(b1 - b0));
      }
    }
    vc[i] = mval;
  }
  // conditioning pointers (and the element-ordered copy of the state every few steps)
  const float inv_n = n > 0 ? 1.0f / static_cast<float>(n) : 0.0f;
  if (a.resort) {
    const int32_t fo = a.foff[e];
    for (int p = threadIdx.x; p < n; p += THREADS) {
      const int32_t d = fo + p;
      if (d >= a.np) break;
      const int32_t q = cur[p];
      store_pos(a.out, d, load_pos(a.p, q));
      a.out.u[d] = a.p.u[q];
      a.out.v[d] = a.p.v[q];
      a.out.w[d] = a.p.w[q];
      a.out.om[d] = a.p.om[q];
      a.out.psi[d] = a.p.psi[q];
      a.out.pid[d] = a.p.pid[q];
      a.out.elem[d] = e;
      a.out.cp[d] = static_cast<uint8_t>(fdiv(G * p, inv_n));
    }
  } else {
#pragma unroll 1
    for (int p = threadIdx.x; p < n; p += THREADS) a.p.cp[cur[p]] = static_cast<uint8_t>(fdiv(G * p, inv_n));
  }
}

// The element of block b in one size class of the plan's tile lists, or -1: block b is entry
// b of the list, which for instance k fills its element range [eb, ee) -- class 0 (up to
// kTileSplit particles) from the front of a.tiles, class 1 (kTileMid + 1 .. kSmallCap) from
// its back, class 2 (kTileSplit + 1 .. kTileMid) from the front of a.tiles_mid.  The class-0
// kernel advances the step counter once per step (no kernel of the statistics reads it).
template <int CLS, typename T>
__device__ __forceinline__ int tile_element(const StatsArgs<T>& a, int b, int& moves) {
  if (CLS == 0 && b == 0 && threadIdx.x == 0 && a.step_inc) atomicAdd(a.step_inc, 1u);
  const int inst = a.einst ? a.einst[b] : 0;
  const int eb = a.einst ? a.ielem[inst] : 0, ee = a.einst ? a.ielem[inst + 1] : a.ne;
  const int32_t* sc = a.scal + 16 * inst;
  if (CLS == 0 ? (b - eb >= sc[6]) : CLS == 1 ? (ee - 1 - b >= sc[7]) : (b - eb >= sc[8])) return -1;
  moves = sc[0] > 0;
  return CLS == 2 ? a.tiles_mid[b] : a.tiles[b];
}

// ---------------------------------------------------------------------------------------
// Hierarchical bins by per-level bucket ranks (the default conditioning, Sect. 3.5 and
// Appendix A).  A level needs each particle's rank by (key, id) inside its group of the
// previous level; it is found without sorting:
//   1. each group's smallest and largest key (as FP32, shared-memory atomics);
//   2. a bucket per particle, floor((key - min) NB_g / (max - min)) with NB_g buckets per
//      group, computed in FP32 from the key rounded to FP32: rounding, subtraction of the
//      group minimum and scaling are all monotone, so the bucket never decreases with the
//      key and equal keys share a bucket;
//   3. bucket counts (atomics), their exclusive scan (the first position of every bucket:
//      the groups lie in group order, so a bucket's first position is its group's first
//      position plus the particles of the group's lower buckets), the particles listed by
//      bucket;
//   4. a particle's position is its bucket's first position plus the number of particles of
//      its bucket that come before it by (key, id), counted directly (buckets hold a few
//      particles).
// The positions are a permutation, the order of an exact sort within the groups, so every
// level, the final order, the moment sums taken in it, the bins and the conditioning
// pointers are those of a full sort by (key, id).  The element's values, ids and slots are
// staged in shared memory once.
// ---------------------------------------------------------------------------------------
template <typename T, int CAP, int THREADS>
struct RankTile {
  static constexpr int kNB = CAP;   // buckets of one level over all of its groups
  using A = double;                 // moment combination and outputs
  T u[CAP], v[CAP], w[CAP], om[CAP], psi[CAP];
  uint32_t pid[CAP];
  int32_t slot[CAP];
  // the levels' bucket tables, and after the last level the moment sums in the same bytes
  // (the FP32 mid-size tile then fits 10 blocks per SM instead of 9)
  union {
    struct {
      int32_t start[kNB + 1];       // bucket counts, then each bucket's first position
      uint32_t glo[256], gsc[256];  // each group's key range, then its bucket origin and scale
    } x_b;
    struct {
      double mh[12], ml[12], msh[5];   // moment sums (value/error pairs) and shift values
    } x_m;
  };
  int16_t ord[CAP];                 // position -> particle (staging index), final level
  int16_t pos[CAP];                 // particle -> position, final level
  int16_t mem[CAP];                 // particles by bucket
  uint8_t grp[CAP];                 // particle -> group of the last level done
  int32_t wsum[THREADS / 32];
  float prior[6];                   // per level: the key's mean and standard deviation of the
                                    // last statistics pass (0, 0: none)
  int n_gathered;
};

// Order-preserving 32-bit image of an FP32 value and its inverse (-0 folded onto +0).
__device__ __forceinline__ uint32_t ord32(float x) { return ord_bits(x); }
__device__ __forceinline__ float unord32(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
__device__ __forceinline__ float bucket_key(float x) { return x; }
__device__ __forceinline__ float bucket_key(double x) { return __double2float_rn(x); }

// (a, ia) before (b, ib): value first, then particle id (the order of the FP32 and FP64
// keys of the sort-based levels; -0 equals +0).
__device__ __forceinline__ bool rank_before(float a, uint32_t ia, float b, uint32_t ib) {
  return (a < b) | ((a == b) & (ia < ib));
}
__device__ __forceinline__ bool rank_before(double a, uint32_t ia, double b, uint32_t ib) {
  const uint64_t oa = ord_bits(a), ob = ord_bits(b);
  return (oa < ob) | ((oa == ob) & (ia < ib));
}

// In-place exclusive scan of c[0, N) (N = E THREADS, E <= EMAX), c[N] = the total.
template <int EMAX, int THREADS>
__device__ __forceinline__ void block_scan_counts(int32_t* c, int E, int32_t* wsum) {
  const int N = E * THREADS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int v[EMAX];
  int sum = 0;
#pragma unroll
  for (int i = 0; i < EMAX; ++i) {
    v[i] = i < E ? c[tid * E + i] : 0;
    sum += v[i];
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int before = incl - sum;
  int total = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) {
    const int ws = wsum[w];
    if (w < warp) before += ws;
    total += ws;
  }
#pragma unroll
  for (int i = 0; i < EMAX; ++i) {
    if (i < E) c[tid * E + i] = before;
    before += v[i];
  }
  if (tid == 0) c[N] = total;
}

// Bucket tables of one level: each particle's bucket within its group (t.grp, or one group
// when Gprev is 1) and the bucket's arrival index; t.x_b.start ends as the first position of
// every bucket.  The buckets of all groups together number NB, a multiple of THREADS of at
// least nb_min (at most the tile's capacity), at least two per group.  The bucket of key x is floor((x - lo) scale) clamped to the group's NB_g
// buckets.  With a prior (mean m and standard deviation s of the key over the element, from
// the previous statistics pass) every group takes lo = m - 3 s and scale = NB_g / (6 s);
// otherwise each group's own smallest and largest key set them.  Either way the bucket never
// decreases with the key, which is all the ranks need.
template <typename T, int CAP, int THREADS>
__device__ __forceinline__ void bucket_level(RankTile<T, CAP, THREADS>& t, const T* key, int n, int Gprev,
                                             int nb_min, float prior_m, float prior_s,
                                             int (&bin)[CAP / THREADS], int (&arr)[CAP / THREADS]) {
  constexpr int KPT = CAP / THREADS, EMAX = RankTile<T, CAP, THREADS>::kNB / THREADS;
  const int tid = threadIdx.x;
  int E = 1;                                   // buckets per thread
  while (E < EMAX && (E * THREADS < nb_min || E * THREADS < 2 * Gprev)) E <<= 1;
  const int NB = E * THREADS;
  const int NBg = NB / Gprev;                  // Gprev <= 256, 2 Gprev <= NB
  const float fNBg = static_cast<float>(NBg);
  const bool prior = prior_s > 0.0f;           // false for NaN
  if (!prior) {
    for (int g = tid; g < Gprev; g += THREADS) {
      t.x_b.glo[g] = 0xffffffffu;
      t.x_b.gsc[g] = 0u;
    }
  }
#pragma unroll
  for (int k = 0; k <= KPT; ++k) {
    const int b = tid + k * THREADS;
    if (b <= NB) t.x_b.start[b] = 0;
  }
  int grp[KPT];
  float fk[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = tid + k * THREADS;
    grp[k] = 0;
    fk[k] = 0.0f;
    if (j < n) {
      if (Gprev > 1) grp[k] = t.grp[j];
      fk[k] = bucket_key(key[j]);
    }
  }
  float plo = 0.0f, pscale = 0.0f;
  if (prior) {
    plo = prior_m - 3.0f * prior_s;
    pscale = fNBg / (6.0f * prior_s);
    __syncthreads();
  } else {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int j = tid + k * THREADS;
      if (j < n) {
        const uint32_t o = ord32(fk[k]);
        atomicMin(&t.x_b.glo[grp[k]], o);
        atomicMax(&t.x_b.gsc[grp[k]], o);
      }
    }
    __syncthreads();
    // per group: the bucket origin (its smallest key) and scale NB_g / (largest - smallest)
    for (int g = tid; g < Gprev; g += THREADS) {
      const float lo = unord32(t.x_b.glo[g]), hi = unord32(t.x_b.gsc[g]);
      const float span = hi - lo;
      t.x_b.glo[g] = __float_as_uint(lo);
      t.x_b.gsc[g] = __float_as_uint(span > 0.0f ? fNBg / span : 0.0f);
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = tid + k * THREADS;
    bin[k] = 0;
    arr[k] = 0;
    if (j < n) {
      const float lo = prior ? plo : __uint_as_float(t.x_b.glo[grp[k]]);
      const float scale = prior ? pscale : __uint_as_float(t.x_b.gsc[grp[k]]);
      const float q = (fk[k] - lo) * scale;
      // q is non-decreasing in the key; NaN (a non-finite state) falls into bucket 0
      const int b = q >= fNBg ? NBg - 1 : (q > 0.0f ? static_cast<int>(q) : 0);
      bin[k] = grp[k] * NBg + b;
      arr[k] = atomicAdd(&t.x_b.start[bin[k]], 1);
    }
  }
  __syncthreads();
  block_scan_counts<EMAX, THREADS>(t.x_b.start, E, t.wsum);
  __syncthreads();
}

// Position of particle j in its bucket's order by (key, id), from the bucket's first
// position s0 and its members t.mem[s0, s1).
template <typename T, int CAP, int THREADS>
__device__ __forceinline__ int bucket_position(const RankTile<T, CAP, THREADS>& t, const T* key, int j,
                                               int s0, int s1) {
  const T kv = key[j];
  const uint32_t kid = t.pid[j];
  int r = 0;
#pragma unroll 1
  for (int m = s0; m < s1; ++m) {
    const int o = t.mem[m];
    r += rank_before(key[o], t.pid[o], kv, kid) ? 1 : 0;
  }
  return s0 + r;
}

// A level before the last: only each particle's new group floor(Gl p / n) is needed.  It
// follows from the bucket's position range unless the range straddles a group boundary;
// only the particles of such buckets are ranked inside their bucket.  t.ord receives an
// arrangement by group (each group's particles within its position range, in any order):
// a particle of a bucket inside one group takes the bucket's first position plus its
// arrival index, a particle of a straddling bucket its exact position.
template <typename T, int CAP, int THREADS>
__device__ void group_level(RankTile<T, CAP, THREADS>& t, const T* key, int n, int Gprev, int Gl,
                            float prior_m, float prior_s) {
  constexpr int KPT = CAP / THREADS;
  const int tid = threadIdx.x;
  const float inv_n = 1.0f / static_cast<float>(n);
  int bin[KPT], arr[KPT];
  bucket_level(t, key, n, Gprev, n, prior_m, prior_s, bin, arr);
  bool cut[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = tid + k * THREADS;
    cut[k] = false;
    if (j < n) {
      const int s0 = t.x_b.start[bin[k]], s1 = t.x_b.start[bin[k] + 1];
      const int g0 = fdiv(Gl * s0, inv_n), g1 = fdiv(Gl * (s1 - 1), inv_n);
      if (g0 == g1) {
        t.grp[j] = static_cast<uint8_t>(g0);
        t.ord[s0 + arr[k]] = static_cast<int16_t>(j);
      } else {
        cut[k] = true;
        t.mem[s0 + arr[k]] = static_cast<int16_t>(j);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = tid + k * THREADS;
    if (cut[k]) {
      const int p = bucket_position(t, key, j, t.x_b.start[bin[k]], t.x_b.start[bin[k] + 1]);
      t.grp[j] = static_cast<uint8_t>(fdiv(Gl * p, inv_n));
      t.ord[p] = static_cast<int16_t>(j);
    }
  }
  __syncthreads();
}

// A level whose groups hold at most 32 particles: a warp takes a whole group from the
// arrangement t.ord (its position range), sorts it in registers with a bitonic network and
// writes the order back into the same range: the exact positions (t.pos, t.ord) and, before
// the last level, the next level's groups.  The sort takes the value bits alone; only a
// group in which two sorted neighbours have equal values is sorted again by the exact key
// (value, particle id).  Either way the order is that of (value, id).
template <typename T, int CAP, int THREADS>
__device__ void warp_level(RankTile<T, CAP, THREADS>& t, const T* key, int n, int Gprev, int Gl,
                           bool last) {
  using PF = KeyPolicy<T, false>;
  using PE = KeyPolicy<T, true>;
  constexpr int W = THREADS / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float invG = 1.0f / static_cast<float>(Gprev), inv_n = 1.0f / static_cast<float>(n);
#pragma unroll 1
  for (int c = warp; c < Gprev; c += W) {
    const int gs = group_start(c, n, Gprev, invG), len = group_start(c + 1, n, Gprev, invG) - gs;
    const int32_t j0 = lane < len ? t.ord[gs + lane] : -1;
    int32_t j = j0;
    {
      typename PF::K k;
      if (lane < len) k = PF::make(key[j0], t.pid, j0);
      else pad_key(k);
      warp_sort32(k, j, lane);
      // a tie, or a real value equal to the padding key (a non-finite state), takes the
      // exact pass, whose keys always sort below the padding
      typename PF::K pad;
      pad_key(pad);
      const typename PF::K up = kdown(k);
      if (__any_sync(kFull, (lane + 1 < len && keq(k, up)) || (lane < len && keq(k, pad)))) {
        typename PE::K ke;
        j = j0;
        if (lane < len) ke = PE::make(key[j0], t.pid, j0);
        else pad_key(ke);
        warp_sort32(ke, j, lane);
      }
    }
    if (lane < len) {
      const int p = gs + lane;
      t.ord[p] = static_cast<int16_t>(j);
      t.pos[j] = static_cast<int16_t>(p);
      if (!last) t.grp[j] = static_cast<uint8_t>(fdiv(Gl * p, inv_n));
    }
  }
  __syncthreads();
}

// The last level: every particle's position in the final order (t.pos, t.ord).
template <typename T, int CAP, int THREADS>
__device__ void order_level(RankTile<T, CAP, THREADS>& t, const T* key, int n, int Gprev, float prior_m,
                            float prior_s) {
  constexpr int KPT = CAP / THREADS;
  const int tid = threadIdx.x;
  int bin[KPT], arr[KPT];
  bucket_level(t, key, n, Gprev, n, prior_m, prior_s, bin, arr);
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = tid + k * THREADS;
    if (j < n) {
      t.mem[t.x_b.start[bin[k]] + arr[k]] = static_cast<int16_t>(j);
      t.ord[j] = static_cast<int16_t>(j);   // every position holds a valid index
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int j = tid + k * THREADS;
    if (j < n) {
      const int p = bucket_position(t, key, j, t.x_b.start[bin[k]], t.x_b.start[bin[k] + 1]);
      t.pos[j] = static_cast<int16_t>(p);
      t.ord[p] = static_cast<int16_t>(j);
    }
  }
  __syncthreads();
}

// Sect. 3.3, Eqs. 35-36 in the final order.  Sums 0..4: d = x - x_0 of u, v, w, omega, psi;
// 5..11: uu, vv, ww, uv, uw, vw, psi psi (products of d; x_0 the first particle of the
// order).  Warp w < 4 takes three of the twelve sums over all particles, lane l the
// positions l, l + 32, ... (compensated FP32 per lane, or FP64; products rounded on their
// own as in element_moments, whose sums these equal bit for bit); the lanes then combine by
// a shuffle tree in a fixed order (value/error pairs in FP32).  Called by every thread.
template <typename A, typename T, int CAP, int THREADS>
__device__ __forceinline__ void rank_moments(RankTile<T, CAP, THREADS>& t, int n) {
  static_assert(THREADS >= 128, "four warps take the moment sums");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 4) {
    // warp 0: d_u, d_u d_u, d_u d_v; 1: d_v, d_v d_v, d_v d_w; 2: d_w, d_w d_w, d_u d_w;
    // 3: d_omega, d_psi, d_psi d_psi
    const T* xa = warp == 0 ? t.u : warp == 1 ? t.v : warp == 2 ? t.w : t.om;
    const T* xb = warp == 0 ? t.v : warp == 1 ? t.w : warp == 2 ? t.u : t.psi;
    A sa = A(0), sb = A(0);
    if (n > 0) {
      const int q0 = t.ord[0];
      sa = A(xa[q0]);
      sb = A(xb[q0]);
    }
    Acc<A> m0, m1, m2;
#pragma unroll 2
    for (int p = lane; p < n; p += 32) {
      const int q = t.ord[p];
      const A da = A(xa[q]) - sa, db = A(xb[q]) - sb;
      if (warp < 3) {
        m0.add(da);
        m1.add(xmul(da, da));
        m2.add(xmul(da, db));
      } else {
        m0.add(da);
        m1.add(db);
        m2.add(xmul(db, db));
      }
    }
    // sum index of each accumulator
    const int c0 = warp < 3 ? warp : 3;
    const int c1 = warp < 3 ? 5 + warp : 4;
    const int c2 = warp == 0 ? 8 : warp == 1 ? 10 : warp == 2 ? 9 : 11;
    A h0, l0, h1, l1, h2, l2;
    m0.warp_pair(h0, l0);
    m1.warp_pair(h1, l1);
    m2.warp_pair(h2, l2);
    if (lane == 0) {
      t.x_m.mh[c0] = h0; t.x_m.ml[c0] = l0;
      t.x_m.mh[c1] = h1; t.x_m.ml[c1] = l1;
      t.x_m.mh[c2] = h2; t.x_m.ml[c2] = l2;
      if (warp < 3) t.x_m.msh[warp] = static_cast<double>(sa);
      else { t.x_m.msh[3] = static_cast<double>(sa); t.x_m.msh[4] = static_cast<double>(sb); }
    }
  }
  __syncthreads();
}

// One element of N <= CAP particles by a block of THREADS (hierarchical bins).
template <typename T, int CAP, int THREADS>
__device__ void element_rank_tile(const StatsArgs<T>& a, RankTile<T, CAP, THREADS>& t, int e, int N,
                                  int moves) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  constexpr int KPT = CAP / THREADS;
  // gather: the element's list minus particles moved out, plus those moved in.  The list
  // entries (and the moved-out test) of a thread's first KPT rounds are loaded before any is
  // used, so that they are in flight together.
  if (threadIdx.x == 0) t.n_gathered = 0;
  // the bucket mapping's prior: the previous pass's count, means and variances of u, v, w,
  // loaded by one thread now and used after the gather (FP32 arithmetic from here on)
  double pri[7];
  if (threadIdx.x == 0 && a.prior) {
    const double* em = a.emom + static_cast<size_t>(kNS) * e;
#pragma unroll
    for (int k = 0; k < 7; ++k) pri[k] = __ldg(em + k);
  }
  __syncthreads();
  {
    const int32_t o = a.off[e], c = a.cnt[e];
    int32_t qk[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int j = warp * 32 + k * THREADS + lane;
      qk[k] = j < c ? __ldg(a.idx + o + j) : -1;
    }
    if (moves) {
      int32_t ek[KPT];
#pragma unroll
      for (int k = 0; k < KPT; ++k) ek[k] = qk[k] >= 0 ? __ldg(a.p.elem + qk[k]) : e;
#pragma unroll
      for (int k = 0; k < KPT; ++k)
        if (ek[k] != e) qk[k] = -1;
    }
    if (!moves && c <= KPT * THREADS) {
      // no particle moved: every list entry is the element's, entry j goes to position j
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        const int j = warp * 32 + k * THREADS + lane;
        if (j < c) t.slot[j] = qk[k];
      }
      if (threadIdx.x == 0) atomicAdd(&t.n_gathered, c);
    } else {
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        const int32_t q = qk[k];
        const unsigned keep = __ballot_sync(kFull, q >= 0);
        int base = 0;
        if (lane == 0 && keep) base = atomicAdd(&t.n_gathered, __popc(keep));
        base = __shfl_sync(kFull, base, 0);
        const int at = base + __popc(keep & below);
        if (q >= 0 && at < CAP) t.slot[at] = q;
      }
    }
    // a list longer than the capacity (particles leave it by moves) continues one round at
    // a time
#pragma unroll 1
    for (int j0 = warp * 32 + KPT * THREADS; j0 < c; j0 += THREADS) {
      const int j = j0 + lane;
      int32_t q = -1;
      if (j < c) {
        q = a.idx[o + j];
        if (moves && a.p.elem[q] != e) q = -1;
      }
      const unsigned keep = __ballot_sync(kFull, q >= 0);
      int base = 0;
      if (lane == 0 && keep) base = atomicAdd(&t.n_gathered, __popc(keep));
      base = __shfl_sync(kFull, base, 0);
      const int at = base + __popc(keep & below);
      if (q >= 0 && at < CAP) t.slot[at] = q;
    }
    if (moves) {
      const int32_t gn = a.gain[e], g0 = a.goff[e];
#pragma unroll 1
      for (int j0 = warp * 32; j0 < gn; j0 += THREADS) {
        const int j = j0 + lane;
        int32_t q = j < gn ? a.movers[g0 + j] : -1;
        if (q >= a.np) q = -1;
        const unsigned keep = __ballot_sync(kFull, q >= 0);
        int base = 0;
        if (lane == 0 && keep) base = atomicAdd(&t.n_gathered, __popc(keep));
        base = __shfl_sync(kFull, base, 0);
        const int at = base + __popc(keep & below);
        if (q >= 0 && at < CAP) t.slot[at] = q;
      }
    }
  }
  __syncthreads();
  int n = t.n_gathered;
  if (n != N && threadIdx.x == 0) atomicCAS(a.err, 0, PDFX_ERR_CAPACITY);
  n = min(min(n, N), CAP);
  // stage the element's values and ids: every load of a thread before any store (the
  // particle arrays are read only here), so that they are in flight together
  {
    T vu[KPT], vv[KPT], vw[KPT], vo[KPT], vp[KPT];
    uint32_t vi[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int j = threadIdx.x + k * THREADS;
      if (j < n) {
        const int32_t q = t.slot[j];
        vu[k] = __ldg(a.p.u + q);
        vv[k] = __ldg(a.p.v + q);
        vw[k] = __ldg(a.p.w + q);
        vo[k] = __ldg(a.p.om + q);
        vp[k] = __ldg(a.p.psi + q);
        vi[k] = __ldg(a.p.pid + q);
      }
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int j = threadIdx.x + k * THREADS;
      if (j < n) {
        t.u[j] = vu[k];
        t.v[j] = vv[k];
        t.w[j] = vw[k];
        t.om[j] = vo[k];
        t.psi[j] = vp[k];
        t.pid[j] = vi[k];
        t.ord[j] = static_cast<int16_t>(j);   // the first level's arrangement
      }
    }
  }
  // effective bins (reading of Sect. 3.5): g_l = max(1, min(b_l, n / (g_1..g_{l-1} min_per_bin)))
  int g[3];
  {
    int Gp = 1;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int capl = n / (Gp * a.min_per_bin);
      int gl = a.bins[l] < capl ? a.bins[l] : capl;
      if (gl < 1) gl = 1;
      g[l] = gl;
      Gp *= gl;
    }
  }
  // the prior per level, by one thread in FP32 (FP64 arithmetic runs at a small fraction of
  // the FP32 rate on this GPU); any monotone bucket mapping gives the same ranks
  if (threadIdx.x == 0) {
    const bool have = a.prior && static_cast<float>(pri[0]) >= 2.0f;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      float pm = 0.0f, ps = 0.0f;
      if (have) {
        const float m = static_cast<float>(pri[1 + l]), var = static_cast<float>(pri[4 + l]);
        if (var > 0.0f && fabsf(m) < 1e30f && var < 1e30f) {
          pm = m;
          ps = sqrtf(var);
        }
      }
      t.prior[2 * l] = pm;
      t.prior[2 * l + 1] = ps;
    }
  }
  __syncthreads();
  // levels by (u, id), (v, id), (w, id) within the groups of the previous level; the levels
  // before the last need only the groups, the last gives the final order
  if (n > 0) {
    int last = 0;
    for (int l = 1; l < 3; ++l)
      if (g[l] > 1) last = l;
    int Gprev = 1;
#pragma unroll 1
    for (int l = 0; l <= last; ++l) {
      if (l > 0 && g[l] <= 1) continue;
      const T* key = l == 0 ? t.u : (l == 1 ? t.v : t.w);
      const float pm = t.prior[2 * l], ps = t.prior[2 * l + 1];
      if ((n + Gprev - 1) / Gprev <= 32) warp_level<T, CAP, THREADS>(t, key, n, Gprev, Gprev * g[l], l == last);
      else if (l == last) order_level<T, CAP, THREADS>(t, key, n, Gprev, pm, ps);
      else group_level<T, CAP, THREADS>(t, key, n, Gprev, Gprev * g[l], pm, ps);
      Gprev *= g[l];
    }
  }
  const int G = g[0] * g[1] * g[2];
  // moments in the final order, then the 13 outputs in FP64 (one per lane of warp 0)
  if (sizeof(T) == 4 && a.acc64) rank_moments<double>(t, n);
  else rank_moments<T>(t, n);
  if (warp == 0) {
    if (lane < kNS) {
      const double inv = recip_n(n);
      const int ix = mom_nib(kMomX, lane), iy = mom_nib(kMomY, lane);
      const int iz = mom_nib(kMomZ, lane), iw = mom_nib(kMomW, lane);
      double v = ix < 15 ? t.x_m.msh[ix] : 0.0;
      if (iy < 15) v += (t.x_m.mh[iy] + t.x_m.ml[iy]) * inv;
      if (iz < 15) {
        const double z = (t.x_m.mh[iz] + t.x_m.ml[iz]) * inv;
        const double wv = (t.x_m.mh[iw] + t.x_m.ml[iw]) * inv;
        v -= z * wv;
      }
      if (lane == 0) v = static_cast<double>(n);
      else if (n == 0) v = 0.0;
      a.emom[static_cast<size_t>(kNS) * e + lane] = v;
    }
    if (lane < 3) a.gbin[3 * e + lane] = g[lane];
  }
  // Appendix A bins: conditional scalar means over the final order's bins
  double* vc = a.vcce + static_cast<size_t>(a.G) * e;
  const float invGb = 1.0f / static_cast<float>(G);
  for (int i = threadIdx.x; i < a.G; i += THREADS) {
    double mval = 0.0;
    if (i < G && n > 0) {
      const int b0 = group_start(i, n, G, invGb), b1 = group_start(i + 1, n, G, invGb);
      if (sizeof(T) == 4 && a.acc64) {
        double sum = 0.0;
#pragma unroll 1
        for (int p = b0; p < b1; ++p) sum += static_cast<double>(t.psi[t.ord[p]]);
        mval = sum / static_cast<double>(b1 - b0);
      } else {
        Acc<T> sum;
#pragma unroll 1
        for (int p = b0; p < b1; ++p) sum.add(t.psi[t.ord[p]]);
        mval = static_cast<double>(sum.value() / static_cast<T>(b1 - b0));
      }
    }
    vc[i] = mval;
  }
  // conditioning pointers (and the element-ordered copy of the state every few steps)
  const float inv_n = n > 0 ? 1.0f / static_cast<float>(n) : 0.0f;
  if (a.resort) {
    const int32_t fo = a.foff[e];
    Pos<T> vx[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int p = threadIdx.x + k * THREADS;
      if (p < n) vx[k] = load_pos(a.p, t.slot[t.ord[p]]);
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      const int p = threadIdx.x + k * THREADS;
      const int32_t d = fo + p;
      if (p >= n || d >= a.np) break;
      const int j = t.ord[p];
      store_pos(a.out, d, vx[k]);
      a.out.u[d] = t.u[j];
      a.out.v[d] = t.v[j];
      a.out.w[d] = t.w[j];
      a.out.om[d] = t.om[j];
      a.out.psi[d] = t.psi[j];
      a.out.pid[d] = t.pid[j];
      a.out.elem[d] = e;
      a.out.cp[d] = static_cast<uint8_t>(fdiv(G * p, inv_n));
    }
  } else {
    for (int j = threadIdx.x; j < n; j += THREADS)
      a.p.cp[t.slot[j]] = static_cast<uint8_t>(fdiv(G * t.pos[j], inv_n));
  }
}

// Residency: the FP32 tiles fit 12 blocks of 128 threads up to 256 particles (11 KB each),
// 10 up to 512 (22 KB) or 7 of 192 up to 768 (32 KB) per SM, the FP64 tiles fewer; the
// register cap matches.
template <typename T, int CAP, int THREADS, int CLS>
__global__ void __launch_bounds__(THREADS, (sizeof(T) == 4 ? (CAP == 256 ? 1536 : THREADS == 192 ? 1344 : 1280) : 1024) / THREADS)
    rank_tile_kernel(const StatsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char rank_smem[];
  RankTile<T, CAP, THREADS>& t = *reinterpret_cast<RankTile<T, CAP, THREADS>*>(rank_smem);
  int moves = 0;
  const int e = tile_element<CLS>(a, blockIdx.x, moves);
  if (e < 0) return;
  const int N = moves ? a.fin[e] : a.cnt[e];
  element_rank_tile<T, CAP, THREADS>(a, t, e, min(N, CAP), moves);
}

// The plan's large-element lists (every instance's), entries of up to kTileBig particles, on
// the bucket-rank tile of kTileBig: a few blocks per SM, each over entries gridDim.x apart;
// stats_big_kernel takes the larger ones.
template <typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 1280 : 1024) / 256) rank_big_kernel(const StatsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char rank_smem[];
  RankTile<T, kTileBig, 256>& t = *reinterpret_cast<RankTile<T, kTileBig, 256>*>(rank_smem);
  bool used = false;
  for (int inst = 0; inst < a.K; ++inst) {
    const int32_t* sc = a.scal + 16 * inst;
    const int eb = a.ielem ? a.ielem[inst] : 0;
    const int moves = sc[0] > 0;
    const int nbig = sc[3];
    for (int b = blockIdx.x; b < nbig; b += gridDim.x) {
      const int e = a.big_list[eb + b];
      const int N = moves ? a.fin[e] : a.cnt[e];
      if (N > kTileBig) continue;
      if (used) __syncthreads();   // the tile's previous element is done with the shared memory
      used = true;
      element_rank_tile<T, kTileBig, 256>(a, t, e, N, moves);
    }
  }
}

template <typename T> bool rank_configured[kMaxDevices];

// One block per entry of one size class of the plan's tile lists (tile_element); the grid
// covers every element and blocks past the class count return.  The register cap keeps 1536
// threads resident per SM in the FP32 form, 1024 in the FP64 form.
template <typename T, int CAP, int THREADS, int CLS, bool FOX>
__global__ void __launch_bounds__(THREADS, (sizeof(T) == 4 ? 1536 : 1024) / THREADS)
    stats_tile_kernel(const StatsArgs<T> a) {
  __shared__ Tile<T, CAP, FOX> t;
  int moves = 0;
  const int e = tile_element<CLS>(a, blockIdx.x, moves);
  if (e < 0) return;
  const int N = moves ? a.fin[e] : a.cnt[e];
  element_tile<T, CAP, THREADS, FOX>(a, t, e, min(N, CAP), moves);
}

}  // namespace

template <typename T>
void launch_stats_tiles_impl(const StatsArgs<T>& a, int num_sms, cudaStream_t s_small, cudaStream_t s_mid,
                             cudaStream_t s_large) {
  if (a.ne <= 0) return;
  static_assert(kSmallCap == 768 && kTileMid == 512 && kTileSplit == 256,
                "tile classes cover the small-element capacity");
  // hierarchical bins: bucket ranks in every class, up to the split (at most 256
  // particles) on a tile of 256 (4 warps), then up to 512 (4 warps) and 513..768 (6
  // warps).  Fox's projection: chunk sorts in every class (groups of at most 32 positions
  // are sorted by one warp in registers; the largest class in a tile of 1,024).
  const unsigned grid = static_cast<unsigned>(a.ne);
  if (a.cond_mode == 1) {
    stats_tile_kernel<T, 1024, 256, 1, true><<<grid, 256, 0, s_large>>>(a);
    stats_tile_kernel<T, 256, 128, 0, true><<<grid, 128, 0, s_small>>>(a);
    stats_tile_kernel<T, 512, 128, 2, true><<<grid, 128, 0, s_mid>>>(a);
  } else {
    constexpr size_t small = sizeof(RankTile<T, 256, 128>), mid = sizeof(RankTile<T, 512, 128>);
    constexpr size_t large = sizeof(RankTile<T, 768, 192>), big = sizeof(RankTile<T, kTileBig, 256>);
    static_assert(big <= 227 * 1024, "rank tile exceeds shared memory");
    if (first_use_on_device(rank_configured<T>)) {
      cudaFuncSetAttribute(rank_tile_kernel<T, 256, 128, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(small));
      cudaFuncSetAttribute(rank_tile_kernel<T, 512, 128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(mid));
      cudaFuncSetAttribute(rank_tile_kernel<T, 768, 192, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(large));
      cudaFuncSetAttribute(rank_big_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(big));
    }
    rank_tile_kernel<T, 768, 192, 1><<<grid, 192, large, s_large>>>(a);
    // 769..1024 from the large-element list: 4 blocks per SM
    rank_big_kernel<T><<<static_cast<unsigned>(4 * (num_sms > 0 ? num_sms : 1)), 256, big, s_large>>>(a);
    rank_tile_kernel<T, 256, 128, 0><<<grid, 128, small, s_small>>>(a);
    rank_tile_kernel<T, 512, 128, 2><<<grid, 128, mid, s_mid>>>(a);
  }
}

}  // namespace pdfx
