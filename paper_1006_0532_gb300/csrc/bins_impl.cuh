// Per-element statistics and conditional means, one thread block per element of up to 1024
// particles (larger elements go through the block kernel in k_stats.cu).
//
// Sect. 3.5 / Appendix A: the element's particles are sorted by (u, id); the level-1 groups
// (positions with equal floor(g1 p / N)) are sorted by (v, id), the level-2 groups by
// (w, id), and position p of the final order gets bin floor(G p / N).  One level: every
// group is cut into chunks of 32 consecutive positions, a warp sorts a chunk in registers
// (bitonic network, one key per lane), and a key's rank in its group is its rank in its
// chunk plus, for every other chunk of the group, the number of smaller keys found by a
// binary search of that sorted chunk.  Keys are distinct (the particle id is part of the
// key), so the ranks are a permutation and the new order is written by scatter.
// Sect. 3.3, Eqs. 35-36: element means, then central moments about them, summed by one
// warp in the final order (deterministic); the FP32 form accumulates compensated FP32 per
// lane and combines lanes as FP32 value/error pairs, the FP64 form sums in FP64.
#pragma once
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

struct K64 {   // FP32 form: value (32 bits) << 28 | id (28 bits)
  uint64_t k;
};
struct K96 {   // FP64 form: value, id
  uint64_t hi;
  uint32_t lo;
};

__device__ __forceinline__ bool kless(const K64& a, const K64& b) { return a.k < b.k; }
__device__ __forceinline__ bool kless(const K96& a, const K96& b) {
  return (a.hi < b.hi) | ((a.hi == b.hi) & (a.lo < b.lo));
}
__device__ __forceinline__ K64 ksel(bool c, const K64& a, const K64& b) { return {c ? a.k : b.k}; }
__device__ __forceinline__ K96 ksel(bool c, const K96& a, const K96& b) {
  return {c ? a.hi : b.hi, c ? a.lo : b.lo};
}
__device__ __forceinline__ K64 kshfl(const K64& a, int m) { return {__shfl_xor_sync(kFull, a.k, m)}; }
__device__ __forceinline__ K96 kshfl(const K96& a, int m) {
  return {__shfl_xor_sync(kFull, a.hi, m), __shfl_xor_sync(kFull, a.lo, m)};
}
__device__ __forceinline__ K64 make_key(float v, uint32_t pid) {
  return {(static_cast<uint64_t>(ord_bits(v)) << 28) | (pid & 0x0fffffffu)};
}
__device__ __forceinline__ K96 make_key(double v, uint32_t pid) { return {ord_bits(v), pid}; }
__device__ __forceinline__ void pad_key(K64& k) { k.k = ~0ull; }
__device__ __forceinline__ void pad_key(K96& k) { k.hi = ~0ull; k.lo = ~0u; }

template <typename T> struct KeyOf;
template <> struct KeyOf<float> { using type = K64; };
template <> struct KeyOf<double> { using type = K96; };

// Sorted chunk keys in shared memory.
template <typename K, int N> struct KeyArr;
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
// maximum and compare equal to each other only, so they end in the top lanes.
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

// Number of keys below k in a sorted, padded chunk of 32 keys starting at base.
template <typename Arr, typename K>
__device__ __forceinline__ int count_below(const Arr& s, int base, const K& k) {
  int pos = 0;
#pragma unroll
  for (int st = 16; st >= 1; st >>= 1) pos += kless(s.get(base + pos + st - 1), k) ? st : 0;
  return pos + (kless(s.get(base + pos), k) ? 1 : 0);
}

// Compensated (Kahan) accumulation for the FP32 form; plain for FP64.  warp_total() sums
// the 32 lanes' accumulators (every lane gets the same value).
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
  // value/error pairs: an exact two-sum of the leading parts, errors added, renormalised
  __device__ __forceinline__ double warp_total() const {
    float h = s, l = -c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(kFull, h, o), ol = __shfl_xor_sync(kFull, l, o);
      const float sh = h + oh;
      const float bb = sh - h;
      const float se = (h - (sh - bb)) + (oh - bb);
      const float lo = se + (l + ol);
      h = sh + lo;
      l = lo - (h - sh);
    }
    return static_cast<double>(h) + static_cast<double>(l);
  }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double warp_total() const {
    double v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
  }
};

__device__ __forceinline__ int group_start(int g, int n, int G) {
  return static_cast<int>((static_cast<int64_t>(g) * n + G - 1) / G);
}

// Shared tile of one element.  Chunk tables are needed only when groups exceed 32
// positions: then there are fewer than CAP/32 groups and fewer than 2 CAP/32 chunks.
template <typename T, int CAP>
struct Tile {
  static constexpr int kChunks = 2 * CAP / 32;
  int32_t ord[CAP];                 // particle slots in the current order
  int32_t nord[CAP];                // the next level's order
  KeyArr<typename KeyOf<T>::type, kChunks * 32> sk;   // sorted chunks (padded to 32)
  int32_t spay[kChunks * 32];       // their slots
  int32_t gfc[CAP / 32 + 1];        // first chunk of each group
  uint8_t cg[kChunks];              // group of each chunk
  int n_gathered;
};

// Elements with lo < N <= hi (hi <= CAP), one block of THREADS each.
template <typename T, int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) stats_tile_kernel(const StatsArgs<T> a, int lo, int hi) {
  using K = typename KeyOf<T>::type;
  constexpr int W = THREADS / 32;
  __shared__ Tile<T, CAP> t;
  const int e = blockIdx.x;
  if (e >= a.ne) return;
  const int moves = a.scal[0] > 0;
  const int N = moves ? a.fin[e] : a.cnt[e];
  if (N <= lo || N > hi) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;

  // gather: the element's list minus particles moved out, plus those moved in
  if (threadIdx.x == 0) t.n_gathered = 0;
  __syncthreads();
  {
    const int32_t o = a.off[e], c = a.cnt[e];
    for (int j0 = warp * 32; j0 < c; j0 += THREADS) {
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
      if (q >= 0 && at < CAP) t.ord[at] = q;
    }
    if (moves) {
      const int32_t gn = a.gain[e], g0 = a.goff[e];
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

  int32_t* cur = t.ord;
  int32_t* nxt = t.nord;
  int Gprev = 1;
  if (n > 0) {
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
      if (l > 0 && g[l] <= 1) continue;
      const T* val = l == 0 ? a.p.u : (l == 1 ? a.p.v : a.p.w);
      const int M = (n + Gprev - 1) / Gprev;   // largest group
      if (M <= 32) {
        // every group is one chunk: the warp sort is the whole level
        for (int c = warp; c < Gprev; c += W) {
          const int gs = group_start(c, n, Gprev), len = group_start(c + 1, n, Gprev) - gs;
          K k;
          int32_t q = -1;
          if (lane < len) {
            q = cur[gs + lane];
            k = make_key(val[q], a.p.pid[q]);
          } else {
            pad_key(k);
          }
          warp_sort32(k, q, lane);
          if (lane < len) nxt[gs + lane] = q;
        }
      } else {
        // chunk tables: Gprev < n / 32 <= CAP / 32 <= 32 groups, one lane each
        if (warp == 0) {
          int nch = 0;
          if (lane < Gprev) nch = (group_start(lane + 1, n, Gprev) - group_start(lane, n, Gprev) + 31) >> 5;
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
        __syncthreads();
        const int nchunks = t.gfc[Gprev];
        for (int c = warp; c < nchunks; c += W) {
          const int gi = t.cg[c];
          const int gs = group_start(gi, n, Gprev), ge = group_start(gi + 1, n, Gprev);
          const int cs = gs + 32 * (c - t.gfc[gi]), len = min(32, ge - cs);
          K k;
          int32_t q = -1;
          if (lane < len) {
            q = cur[cs + lane];
            k = make_key(val[q], a.p.pid[q]);
          } else {
            pad_key(k);
          }
          warp_sort32(k, q, lane);
          t.sk.set(c * 32 + lane, k);
          t.spay[c * 32 + lane] = q;
        }
        __syncthreads();
        for (int c = warp; c < nchunks; c += W) {
          const int gi = t.cg[c];
          const int gs = group_start(gi, n, Gprev), ge = group_start(gi + 1, n, Gprev);
          const int c0 = t.gfc[gi], c1 = t.gfc[gi + 1];
          const int cs = gs + 32 * (c - c0), len = min(32, ge - cs);
          const K k = t.sk.get(c * 32 + lane);
          int r = lane;
          for (int c2 = c0; c2 < c1; ++c2)
            if (c2 != c) r += count_below(t.sk, c2 * 32, k);
          if (lane < len) nxt[gs + r] = t.spay[c * 32 + lane];
        }
      }
      __syncthreads();
      int32_t* tmp = cur;
      cur = nxt;
      nxt = tmp;
      Gprev *= g[l];
    }
  }
  const int G = g[0] * g[1] * g[2];

  // moments (warp 0) in the final order: sums of d = x - x_0 and of products of d, x_0 the
  // first particle of the order; mean = x_0 + S1/N, central = S2/N - (S1/N)^2
  if (warp == 0) {
    T sh[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (n > 0) {
      const int32_t q0 = cur[0];
      sh[0] = a.p.u[q0]; sh[1] = a.p.v[q0]; sh[2] = a.p.w[q0]; sh[3] = a.p.om[q0]; sh[4] = a.p.psi[q0];
    }
    Acc<T> s1[5], s2[7];
    for (int p = lane; p < n; p += 32) {
      const int32_t q = cur[p];
      const T du = a.p.u[q] - sh[0], dv = a.p.v[q] - sh[1], dw = a.p.w[q] - sh[2];
      const T dom = a.p.om[q] - sh[3], dp = a.p.psi[q] - sh[4];
      s1[0].add(du); s1[1].add(dv); s1[2].add(dw); s1[3].add(dom); s1[4].add(dp);
      s2[0].add(du * du); s2[1].add(dv * dv); s2[2].add(dw * dw);
      s2[3].add(du * dv); s2[4].add(du * dw); s2[5].add(dv * dw);
      s2[6].add(dp * dp);
    }
    const double inv = n > 0 ? 1.0 / n : 0.0;
    double d1[5], d2[7];
#pragma unroll
    for (int c = 0; c < 5; ++c) d1[c] = s1[c].warp_total() * inv;
#pragma unroll
    for (int c = 0; c < 7; ++c) d2[c] = s2[c].warp_total() * inv;
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

  // Appendix A bins: conditional scalar means over the final order's bins
  double* vc = a.vcce + static_cast<size_t>(a.G) * e;
  for (int i = threadIdx.x; i < a.G; i += THREADS) {
    double mval = 0.0;
    if (i < G && n > 0) {
      const int b0 = group_start(i, n, G), b1 = group_start(i + 1, n, G);
      double sum = 0.0;
      for (int p = b0; p < b1; ++p) sum += static_cast<double>(a.p.psi[cur[p]]);
      mval = sum / (b1 - b0);
    }
    vc[i] = mval;
  }
  // conditioning pointers (and the element-ordered copy of the state every few steps)
  if (a.resort) {
    const int32_t fo = a.foff[e];
    for (int p = threadIdx.x; p < n; p += THREADS) {
      const int32_t d = fo + p;
      if (d >= a.np) break;
      const int32_t q = cur[p];
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
    for (int p = threadIdx.x; p < n; p += THREADS)
      a.p.cp[cur[p]] = static_cast<uint8_t>((static_cast<int64_t>(G) * p) / n);
  }
}

}  // namespace

template <typename T>
void launch_stats_warp_impl(const StatsArgs<T>& a, cudaStream_t s) {
  if (a.ne <= 0) return;
  static_assert(kSmallCap == 1024, "tile classes cover the small-element capacity");
  // elements of up to 512 particles (4 warps), then 513..1024 (8 warps)
  stats_tile_kernel<T, 512, 128><<<static_cast<unsigned>(a.ne), 128, 0, s>>>(a, -1, 512);
  stats_tile_kernel<T, 1024, 256><<<static_cast<unsigned>(a.ne), 256, 0, s>>>(a, 512, 1024);
}

}  // namespace pdfx
