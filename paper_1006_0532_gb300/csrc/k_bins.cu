// Per-element statistics and conditional means, one warp per element (up to 1024
// particles; larger elements go through the block kernel in k_stats.cu).
//
// Sect. 3.5 / Appendix A: the element's particles are sorted by (u, id); the level-1 groups
// (positions with equal floor(g1 n / N)) are sorted by (v, id), the level-2 groups by
// (w, id), and particle n of the final order gets bin floor(G n / N).  Each level is one
// warp-wide bitonic sort of composite keys (group, order-preserving value, particle id)
// held in registers, 8, 16 or 32 per lane; no block barrier is involved.
// Sect. 3.3, Eqs. 35-36: element means, then central moments about them, summed in the
// level-1 order (deterministic); the FP32 form accumulates compensated FP32 per lane and
// combines lanes in FP64.
#include "pdfx_internal.h"

namespace pdfx {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpCap = 1024;

// ---------------------------------------------------------------------------------------
// Keys.  Particle ids must be below 2^28 (checked by the host).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ord_bits(float x) {
  const uint32_t b = __float_as_uint(x + 0.0f);   // -0 -> +0: equal values tie
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint64_t ord_bits(double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x + 0.0));
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

struct K64 {   // FP32 form: group (4 bits) | value (32 bits) | id (28 bits)
  uint64_t k;
};
struct K96 {   // FP64 form: value in hi; group (4 bits) | id (28 bits) in lo
  uint64_t hi;
  uint32_t lo;
};

__device__ __forceinline__ bool kless(const K64& a, const K64& b) { return a.k < b.k; }
__device__ __forceinline__ bool kless(const K96& a, const K96& b) {
  const uint32_t ga = a.lo >> 28, gb = b.lo >> 28;
  const bool hlt = a.hi < b.hi, heq = a.hi == b.hi;
  return (ga < gb) | ((ga == gb) & (hlt | (heq & (a.lo < b.lo))));
}
__device__ __forceinline__ K64 ksel(bool c, const K64& a, const K64& b) { return {c ? a.k : b.k}; }
__device__ __forceinline__ K96 ksel(bool c, const K96& a, const K96& b) {
  return {c ? a.hi : b.hi, c ? a.lo : b.lo};
}
__device__ __forceinline__ K64 kshfl(const K64& a, int m) { return {__shfl_xor_sync(kFull, a.k, m)}; }
__device__ __forceinline__ K96 kshfl(const K96& a, int m) {
  return {__shfl_xor_sync(kFull, a.hi, m), __shfl_xor_sync(kFull, a.lo, m)};
}
__device__ __forceinline__ K64 make_key(uint32_t grp, float v, uint32_t pid) {
  return {(static_cast<uint64_t>(grp) << 60) | (static_cast<uint64_t>(ord_bits(v)) << 28) |
          (pid & 0x0fffffffu)};
}
__device__ __forceinline__ K96 make_key(uint32_t grp, double v, uint32_t pid) {
  return {ord_bits(v), (grp << 28) | (pid & 0x0fffffffu)};
}
__device__ __forceinline__ void pad_key(K64& k) { k.k = ~0ull; }
__device__ __forceinline__ void pad_key(K96& k) { k.hi = ~0ull; k.lo = ~0u; }

template <typename T> struct KeyOf;
template <> struct KeyOf<float> { using type = K64; };
template <> struct KeyOf<double> { using type = K96; };

// Warp bitonic sort of 32 * KPL keys; lane l holds positions l * KPL + r.  Payload is the
// particle's slot.  Keys are distinct (the particle id is part of the key), so a
// compare-exchange is a branch-free select.  Merge levels below KPL stay inside a lane and
// are unrolled (directions known at compile time); from level KPL on, stages exchange
// across lanes by shuffles and finish with in-lane stages whose direction is fixed per lane.
template <int KPL, typename K>
__device__ __forceinline__ void cmp_swap(K& a, K& b, uint32_t& pa, uint32_t& pb, bool up) {
  const bool sw = kless(b, a) == up;
  const K ta = ksel(sw, b, a), tb = ksel(sw, a, b);
  const uint32_t qa = sw ? pb : pa, qb = sw ? pa : pb;
  a = ta; b = tb; pa = qa; pb = qb;
}

template <int KPL, int KK, int J, typename K>
struct StaticStages {   // merge level KK (<= KPL), stages J, J/2, ..., 1, all in-lane
  __device__ __forceinline__ static void run(K (&k)[KPL], uint32_t (&v)[KPL]) {
#pragma unroll
    for (int r = 0; r < KPL; ++r)
      if ((r & J) == 0) cmp_swap<KPL>(k[r], k[r | J], v[r], v[r | J], (r & KK) == 0);
    StaticStages<KPL, KK, J / 2, K>::run(k, v);
  }
};
template <int KPL, int KK, typename K>
struct StaticStages<KPL, KK, 0, K> {
  __device__ __forceinline__ static void run(K (&)[KPL], uint32_t (&)[KPL]) {}
};
template <int KPL, int KK, typename K>
struct StaticLevels {   // merge levels 2, 4, ..., KPL / 2: direction depends on r only
  __device__ __forceinline__ static void run(K (&k)[KPL], uint32_t (&v)[KPL]) {
    StaticStages<KPL, KK, KK / 2, K>::run(k, v);
    StaticLevels<KPL, KK * 2, K>::run(k, v);
  }
};
template <int KPL, typename K>
struct StaticLevels<KPL, KPL, K> {
  __device__ __forceinline__ static void run(K (&)[KPL], uint32_t (&)[KPL]) {}
};
template <int KPL, int J, typename K>
struct LaneStages {     // stages J, ..., 1 of a level longer than KPL: one direction per lane
  __device__ __forceinline__ static void run(K (&k)[KPL], uint32_t (&v)[KPL], bool up) {
#pragma unroll
    for (int r = 0; r < KPL; ++r)
      if ((r & J) == 0) cmp_swap<KPL>(k[r], k[r | J], v[r], v[r | J], up);
    LaneStages<KPL, J / 2, K>::run(k, v, up);
  }
};
template <int KPL, typename K>
struct LaneStages<KPL, 0, K> {
  __device__ __forceinline__ static void run(K (&)[KPL], uint32_t (&)[KPL], bool) {}
};

template <int KPL, typename K>
__device__ __forceinline__ void warp_sort(K (&k)[KPL], uint32_t (&v)[KPL]) {
  const int lane = threadIdx.x & 31;
  StaticLevels<KPL, 2, K>::run(k, v);
#pragma unroll 1
  for (int kk = KPL; kk <= 32 * KPL; kk <<= 1) {   // direction depends on the lane
    const bool up = ((lane * KPL) & kk) == 0;
#pragma unroll 1
    for (int j = kk >> 1; j >= KPL; j >>= 1) {
      const int lj = j / KPL;
      const bool keep_min = ((lane & lj) == 0) == up;
#pragma unroll
      for (int r = 0; r < KPL; ++r) {
        const K ok = kshfl(k[r], lj);
        const uint32_t ov = __shfl_xor_sync(kFull, v[r], lj);
        const bool take = kless(ok, k[r]) == keep_min;
        k[r] = ksel(take, ok, k[r]);
        v[r] = take ? ov : v[r];
      }
    }
    LaneStages<KPL, KPL / 2, K>::run(k, v, up);
  }
}

// Compensated (Kahan) accumulation for the FP32 form; plain for FP64.
template <typename T>
struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(s) - static_cast<double>(c); }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Per-warp shared memory: the element's particle slots (gathered list, later the final
// order).  Particle attributes are read through L1 by slot.

// Sorts, moments, bins of one element held by one warp (n particles, n <= 32 * KPL).
// Payload of the sort: the particle's slot in the state arrays.
template <typename T, int KPL>
__device__ void element_in_warp(const StatsArgs<T>& a, int32_t* sl, int e, int n) {
  using K = typename KeyOf<T>::type;
  const int lane = threadIdx.x & 31;
  K key[KPL];
  uint32_t pay[KPL];
  // level 1: (u, id); register r of lane l starts with list entry r * 32 + l
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int p = r * 32 + lane;
    if (p < n) {
      const int32_t q = sl[p];
      pay[r] = static_cast<uint32_t>(q);
      key[r] = make_key(0u, a.p.u[q], a.p.pid[q]);
    } else {
      pay[r] = 0u;
      pad_key(key[r]);
    }
  }
  warp_sort<KPL>(key, pay);

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
  // moments in level-1 order (deterministic): sums of d = x - x_0 and of products of d,
  // x_0 the first particle of the order; mean = x_0 + S1/N, central = S2/N - (S1/N)^2
  {
    T sh[5];
    {
      const uint32_t q0 = __shfl_sync(kFull, pay[0], 0);
      sh[0] = a.p.u[q0]; sh[1] = a.p.v[q0]; sh[2] = a.p.w[q0]; sh[3] = a.p.om[q0]; sh[4] = a.p.psi[q0];
    }
    Acc<T> s1[5], s2[7];
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      if (lane * KPL + r < n) {
        const uint32_t q = pay[r];
        const T du = a.p.u[q] - sh[0], dv = a.p.v[q] - sh[1], dw = a.p.w[q] - sh[2];
        const T dom = a.p.om[q] - sh[3], dp = a.p.psi[q] - sh[4];
        s1[0].add(du); s1[1].add(dv); s1[2].add(dw); s1[3].add(dom); s1[4].add(dp);
        s2[0].add(du * du); s2[1].add(dv * dv); s2[2].add(dw * dw);
        s2[3].add(du * dv); s2[4].add(du * dw); s2[5].add(dv * dw);
        s2[6].add(dp * dp);
      }
    }
    const double inv = n > 0 ? 1.0 / n : 0.0;
    double d1[5], d2[7];
#pragma unroll
    for (int c = 0; c < 5; ++c) d1[c] = warp_allsum(s1[c].value()) * inv;
#pragma unroll
    for (int c = 0; c < 7; ++c) d2[c] = warp_allsum(s2[c].value()) * inv;
    if (lane == 0) {
      double* em = a.emom + static_cast<size_t>(kNS) * e;
      em[0] = static_cast<double>(n);
      em[1] = static_cast<double>(sh[0]) + d1[0];
      em[2] = static_cast<double>(sh[1]) + d1[1];
      em[3] = static_cast<double>(sh[2]) + d1[2];
      em[4] = d2[0] - d1[0] * d1[0]; em[5] = d2[1] - d1[1] * d1[1]; em[6] = d2[2] - d1[2] * d1[2];
      em[7] = d2[3] - d1[0] * d1[1]; em[8] = d2[4] - d1[0] * d1[2]; em[9] = d2[5] - d1[1] * d1[2];
      em[10] = static_cast<double>(sh[3]) + d1[3];
      em[11] = static_cast<double>(sh[4]) + d1[4];
      em[12] = d2[6] - d1[4] * d1[4];
      if (n == 0) for (int c = 1; c < kNS; ++c) em[c] = 0.0;
      a.gbin[3 * e] = g[0];
      a.gbin[3 * e + 1] = g[1];
      a.gbin[3 * e + 2] = g[2];
    }
  }
  // levels 2 and 3: groups of the previous level sorted by (v, id), then (w, id)
  {
    int Gprev = g[0];
#pragma unroll
    for (int l = 1; l < 3; ++l) {
      if (g[l] > 1) {
        const T* val = l == 1 ? a.p.v : a.p.w;
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
          const int p = lane * KPL + r;
          if (p < n) {
            const uint32_t q = pay[r];
            const uint32_t grp = static_cast<uint32_t>((static_cast<int64_t>(Gprev) * p) / n);
            key[r] = make_key(grp, val[q], a.p.pid[q]);
          } else {
            pad_key(key[r]);
          }
        }
        warp_sort<KPL>(key, pay);
      }
      Gprev *= g[l];
    }
  }
  // final order -> shared slots; Appendix A bins, conditional means, pointers
  __syncwarp();
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int p = lane * KPL + r;
    if (p < n) sl[p] = static_cast<int32_t>(pay[r]);
  }
  __syncwarp();
  const int G = g[0] * g[1] * g[2];
  double* vc = a.vcce + static_cast<size_t>(a.G) * e;
  for (int i = lane; i < a.G; i += 32) {
    double mval = 0.0;
    if (i < G && n > 0) {
      const int lo = static_cast<int>((static_cast<int64_t>(i) * n + G - 1) / G);
      const int hi = static_cast<int>((static_cast<int64_t>(i + 1) * n + G - 1) / G);
      double sum = 0.0;
      for (int p = lo; p < hi; ++p) sum += static_cast<double>(a.p.psi[sl[p]]);
      mval = sum / (hi - lo);
    }
    vc[i] = mval;
  }
  if (a.resort) {
    const int32_t fo = a.foff[e];
    for (int p = lane; p < n; p += 32) {
      const int32_t d = fo + p;
      if (d >= a.np) break;
      const int32_t q = sl[p];
      a.out.x[d] = a.p.x[q];
      a.out.y[d] = a.p.y[q];
      a.out.u[d] = a.p.u[q];
      a.out.v[d] = a.p.v[q];
      a.out.w[d] = a.p.w[q];
      a.out.om[d] = a.p.om[q];
      a.out.psi[d] = a.p.psi[q];
      a.out.pid[d] = a.p.pid[q];
      a.out.elem[d] = e;
      a.out.cp[d] = static_cast<uint8_t>((static_cast<int64_t>(G) * p) / n);
    }
  } else {
    for (int p = lane; p < n; p += 32)
      a.p.cp[sl[p]] = static_cast<uint8_t>((static_cast<int64_t>(G) * p) / n);
  }
}

// Elements with lo < N <= hi (N <= 1024), one warp each.
template <typename T, int WARPS, int KMAX>
__global__ void __launch_bounds__(32 * WARPS) stats_warp_kernel(const StatsArgs<T> a, int lo, int hi) {
  __shared__ int32_t slots[WARPS][kWarpCap];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * WARPS + wid;
  if (e >= a.ne) return;
  int32_t* sl = slots[wid];
  const int moves = a.scal[0] > 0;
  const int N = moves ? a.fin[e] : a.cnt[e];
  if (N <= lo || N > hi) return;
  // gather: the element's list minus particles moved out, plus those moved in
  int n = 0;
  const int32_t o = a.off[e], c = a.cnt[e];
  for (int j0 = 0; j0 < c; j0 += 32) {
    const int j = j0 + lane;
    int32_t q = -1;
    if (j < c) {
      q = a.idx[o + j];
      if (moves && a.p.elem[q] != e) q = -1;
    }
    const unsigned keep = __ballot_sync(kFull, q >= 0);
    const int at = n + __popc(keep & ((1u << lane) - 1u));
    if (q >= 0 && at < kWarpCap) sl[at] = q;
    n += __popc(keep);
  }
  if (moves) {
    const int32_t gn = a.gain[e], g0 = a.goff[e];
    for (int j0 = 0; j0 < gn; j0 += 32) {
      const int j = j0 + lane;
      int32_t q = j < gn ? a.movers[g0 + j] : -1;
      if (q >= a.np) q = -1;
      const unsigned keep = __ballot_sync(kFull, q >= 0);
      const int at = n + __popc(keep & ((1u << lane) - 1u));
      if (q >= 0 && at < kWarpCap) sl[at] = q;
      n += __popc(keep);
    }
  }
  if (n != N && lane == 0) atomicCAS(a.err, 0, PDFX_ERR_CAPACITY);
  n = min(min(n, N), 32 * KMAX);
  __syncwarp();
  if (KMAX <= 16) {
    if (n <= 256) element_in_warp<T, 8>(a, sl, e, n);
    else element_in_warp<T, (KMAX < 16 ? 8 : 16)>(a, sl, e, n);
  } else {
    element_in_warp<T, KMAX>(a, sl, e, n);
  }
}

}  // namespace

template <typename T>
void launch_stats_warp(const StatsArgs<T>& a, cudaStream_t s) {
  constexpr int W = 4;
  if (a.ne <= 0) return;
  const unsigned grid = static_cast<unsigned>((a.ne + W - 1) / W);
  // elements of up to 512 particles (8 or 16 keys per lane), then 513..1024 (32 per lane)
  stats_warp_kernel<T, W, 16><<<grid, 32 * W, 0, s>>>(a, -1, 512);
  stats_warp_kernel<T, W, 32><<<grid, 32 * W, 0, s>>>(a, 512, kWarpCap);
}

template void launch_stats_warp<float>(const StatsArgs<float>&, cudaStream_t);
template void launch_stats_warp<double>(const StatsArgs<double>&, cudaStream_t);

}  // namespace pdfx
