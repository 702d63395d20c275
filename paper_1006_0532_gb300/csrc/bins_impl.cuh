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
#pragma once
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

// Warp bitonic sort over positions p = r * 32 + lane (register r of lane l), 32 * KPL real
// positions; registers past KPL up to the next power of two are virtual +infinity.  Every
// comparator sends the smaller key to the lower position (mirror stage, then half-cleaners),
// so a comparator with a virtual partner keeps its own key and virtual keys never enter
// real positions.  Sorting only the first log2(B) merge levels sorts aligned blocks of B
// positions independently.  Keys are distinct (the particle id is part of the key), so a
// compare-exchange is a branch-free select.  Payload: the particle's slot.
template <int N>
struct NextPow2 { static constexpr int value = N <= 1 ? 1 : 2 * NextPow2<(N + 1) / 2>::value; };
template <>
struct NextPow2<1> { static constexpr int value = 1; };

template <int KPL, typename K>
__device__ __forceinline__ void ce_lane(K (&k)[KPL], uint32_t (&v)[KPL], int pl, bool keep_min) {
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const K ok = kshfl(k[r], pl);
    const uint32_t ov = __shfl_xor_sync(kFull, v[r], pl);
    const bool take = kless(ok, k[r]) == keep_min;
    k[r] = ksel(take, ok, k[r]);
    v[r] = take ? ov : v[r];
  }
}

// Mirror stage of merge level 32 * M (M >= 2): position (r, l) against (r ^ (M-1), l ^ 31).
template <int KPL, int M, typename K>
__device__ __forceinline__ void mirror_regs(K (&k)[KPL], uint32_t (&v)[KPL]) {
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int r2 = r ^ (M - 1);
    if (r < r2 && r2 < KPL) {
      const K a = kshfl(k[r2], 31), b = kshfl(k[r], 31);
      const uint32_t va = __shfl_xor_sync(kFull, v[r2], 31), vb = __shfl_xor_sync(kFull, v[r], 31);
      const bool t1 = kless(a, k[r]);    // (r, l) is the lower position: keeps the minimum
      const bool t2 = kless(k[r2], b);   // (r2, l) is the higher position: keeps the maximum
      k[r] = ksel(t1, a, k[r]);
      v[r] = t1 ? va : v[r];
      k[r2] = ksel(t2, b, k[r2]);
      v[r2] = t2 ? vb : v[r2];
    }
  }
}

// Half-cleaner stages with distance 32 * JR, ..., 32 (inside a lane).
template <int KPL, int JR, typename K>
struct HalfRegs {
  __device__ __forceinline__ static void run(K (&k)[KPL], uint32_t (&v)[KPL]) {
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      if ((r & JR) == 0 && (r | JR) < KPL) {
        const int r2 = r | JR;
        const bool sw = kless(k[r2], k[r]);
        const K ta = ksel(sw, k[r2], k[r]), tb = ksel(sw, k[r], k[r2]);
        const uint32_t qa = sw ? v[r2] : v[r], qb = sw ? v[r] : v[r2];
        k[r] = ta; k[r2] = tb; v[r] = qa; v[r2] = qb;
      }
    }
    HalfRegs<KPL, JR / 2, K>::run(k, v);
  }
};
template <int KPL, typename K>
struct HalfRegs<KPL, 0, K> {
  __device__ __forceinline__ static void run(K (&)[KPL], uint32_t (&)[KPL]) {}
};

// Merge levels 32 * M, 64 * M, ... up to the block size B.
template <int KPL, int M, typename K>
struct Levels {
  __device__ __forceinline__ static void run(K (&k)[KPL], uint32_t (&v)[KPL], int B) {
    if (32 * M > B) return;
    const int lane = threadIdx.x & 31;
    mirror_regs<KPL, M>(k, v);
    HalfRegs<KPL, M / 4, K>::run(k, v);
#pragma unroll 1
    for (int j = 16; j >= 1; j >>= 1) ce_lane(k, v, j, (lane & j) == 0);
    Levels<KPL, 2 * M, K>::run(k, v, B);
  }
};
template <int KPL, typename K>
struct Levels<KPL, 2 * NextPow2<KPL>::value, K> {
  __device__ __forceinline__ static void run(K (&)[KPL], uint32_t (&)[KPL], int) {}
};

template <int KPL, typename K>
__device__ __forceinline__ void block_sort(K (&k)[KPL], uint32_t (&v)[KPL], int B) {
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int kk = 2; kk <= B && kk <= 32; kk <<= 1) {
    ce_lane(k, v, kk - 1, (lane & (kk >> 1)) == 0);
#pragma unroll 1
    for (int j = kk >> 2; j >= 1; j >>= 1) ce_lane(k, v, j, (lane & j) == 0);
  }
  Levels<KPL, 2, K>::run(k, v, B);
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
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
// sl: the warp's shared slot buffer (holds the gathered list on entry).
template <typename T, int KPL>
__device__ void element_in_warp(const StatsArgs<T>& a, int32_t* sl, int e, int n) {
  using K = typename KeyOf<T>::type;
  constexpr int P2 = 32 * NextPow2<KPL>::value;
  const int lane = threadIdx.x & 31;
  K key[KPL];
  uint32_t pay[KPL];
  // Layout after a sort: global (position p holds order position p) or aligned blocks of
  // lay_B positions for lay_G groups.  order_pos gives the position in the level order of the
  // particle at register position p, -1 for padding.
  int lay_B = 0, lay_G = 1;
  auto order_pos = [&](int p) -> int {
    if (lay_B == 0) return p < n ? p : -1;
    const int grp = p / lay_B, i = p - grp * lay_B;
    const int start = static_cast<int>((static_cast<int64_t>(grp) * n + lay_G - 1) / lay_G);
    const int end = static_cast<int>((static_cast<int64_t>(grp + 1) * n + lay_G - 1) / lay_G);
    return (grp < lay_G && i < end - start) ? start + i : -1;
  };

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
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int p = r * 32 + lane;
    pay[r] = p < n ? static_cast<uint32_t>(sl[p]) : 0u;
  }
  // Level 1 sorts the element by (u, id).  Level l > 1 sorts each group of the previous level
  // (positions with equal floor(Gprev gp / n)) by (v, id), then (w, id): the groups are laid
  // out in aligned blocks of B positions (B = next power of two of the largest group) and
  // sorted blockwise; if the blocks do not fit, one full sort of (group, value, id) keys.
  int Gprev = 1;
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    if (l > 0 && g[l] <= 1) { Gprev *= g[l]; continue; }
    const T* val = l == 0 ? a.p.u : (l == 1 ? a.p.v : a.p.w);
    int B = P2;
    bool aligned = false;
    if (l > 0) {
      B = pow2_at_least((n + Gprev - 1) / Gprev);
      aligned = Gprev * B <= 32 * KPL;
      if (!aligned) B = P2;
    }
    if (aligned) {
      __syncwarp();
      for (int p = lane; p < 32 * KPL; p += 32) sl[p] = -1;
      __syncwarp();
#pragma unroll
      for (int r = 0; r < KPL; ++r) {
        const int o = order_pos(r * 32 + lane);
        if (o >= 0) {
          const int grp = static_cast<int>((static_cast<int64_t>(Gprev) * o) / n);
          const int start = static_cast<int>((static_cast<int64_t>(grp) * n + Gprev - 1) / Gprev);
          sl[grp * B + (o - start)] = static_cast<int32_t>(pay[r]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < KPL; ++r) {
        const int32_t q = sl[r * 32 + lane];
        pay[r] = q >= 0 ? static_cast<uint32_t>(q) : 0u;
        if (q >= 0) key[r] = make_key(static_cast<uint32_t>((r * 32 + lane) / B), val[q], a.p.pid[q]);
        else pad_key(key[r]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < KPL; ++r) {
        const int o = order_pos(r * 32 + lane);
        if (o >= 0) {
          const uint32_t grp = static_cast<uint32_t>((static_cast<int64_t>(Gprev) * o) / n);
          key[r] = make_key(grp, val[pay[r]], a.p.pid[pay[r]]);
        } else {
          pad_key(key[r]);
        }
      }
    }
    block_sort<KPL>(key, pay, B);
    lay_B = aligned ? B : 0;
    lay_G = aligned ? Gprev : 1;
    if (l == 0) {
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
        if (r * 32 + lane < n) {
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
    }
    Gprev *= g[l];
  }
  // final order -> shared slots; Appendix A bins, conditional means, pointers
  __syncwarp();
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int o = order_pos(r * 32 + lane);
    if (o >= 0) sl[o] = static_cast<int32_t>(pay[r]);
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
    else if (n <= 384) element_in_warp<T, 12>(a, sl, e, n);
    else element_in_warp<T, 16>(a, sl, e, n);
  } else {
    if (n <= 640) element_in_warp<T, 20>(a, sl, e, n);
    else if (n <= 768) element_in_warp<T, 24>(a, sl, e, n);
    else element_in_warp<T, 32>(a, sl, e, n);
  }
}

}  // namespace

template <typename T>
void launch_stats_warp_impl(const StatsArgs<T>& a, cudaStream_t s) {
  constexpr int W = 4;
  if (a.ne <= 0) return;
  const unsigned grid = static_cast<unsigned>((a.ne + W - 1) / W);
  // elements of up to 512 particles (8, 12 or 16 keys per lane), then 513..1024 (20, 24, 32)
  stats_warp_kernel<T, W, 16><<<grid, 32 * W, 0, s>>>(a, -1, 512);
  stats_warp_kernel<T, W, 32><<<grid, 32 * W, 0, s>>>(a, 512, kWarpCap);
}

}  // namespace pdfx
