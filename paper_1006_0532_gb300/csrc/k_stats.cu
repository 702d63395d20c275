// Statistics pipeline after the particle advance:
//   plan         counts -> list offsets; Appendix B particle-number control in closed form
//   scatter      element lists of particle slots
//   redistribute donor selection, new values of moved particles, commit
//   stats        per element: two-pass moments (Eqs. 35-36), adaptive sort-and-divide
//                binning and conditional means (Sect. 3.5, Appendix A), optional re-order
//   node average nodal statistics = mean over the surrounding non-empty elements (Sect. 3.3)
#include "pdfx_internal.h"

namespace pdfx {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPlanThreads = 1024;

// ---------------------------------------------------------------------------------------
// Block-wide exclusive scan (deterministic).
// ---------------------------------------------------------------------------------------
template <typename V>
__device__ V block_exclusive_scan(V v, V* tmp /* [32] */, V& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  V x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    V t = lane < nw ? tmp[lane] : V(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const V y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    tmp[lane] = t;
  }
  __syncthreads();
  const V before = (wid > 0 ? tmp[wid - 1] : V(0)) + x - v;
  total = tmp[nw - 1];
  __syncthreads();
  return before;
}

// ---------------------------------------------------------------------------------------
// Plan: one block.  Writes off / cursor (exclusive scan of counts), the big-element list,
// and, when particles must move, the Appendix B final counts in closed form.
//
// The Appendix B loop moves one particle at a time from the fullest element (lowest id on
// ties) to the emptiest (lowest id on ties) while min < MINNPEL and max - min >= 2.  A
// receiving element never becomes the fullest while the loop runs, nor a giving element
// the emptiest, so after t moves the receiving side is "water-filled" from below and the
// giving side drained from the top:
//   min_t = max{L : D(L) <= t},  D(L) = sum_e max(0, L - c_e)
//   max_t = min{H : S(H) <= t},  S(H) = sum_e max(0, c_e - H)
// and the loop stops at T = min{t : min_t >= MINNPEL or max_t - min_t <= 1}.  The extra
// units at the final levels go to (come from) the lowest element ids, exactly as the
// loop's tie-breaking picks them.
// ---------------------------------------------------------------------------------------
struct PlanShared {
  int32_t tmp32[32];
  int64_t tmp64[32];
  int32_t vmin[32], vmax[32];
  int32_t carry[8];
  int64_t Tm, L, H, r, rp, cmin, cmax;
  int need;
};

__device__ int64_t D_of(const int64_t* P0, const int64_t* P1, int64_t L, int64_t cmax) {
  // sum over c < L of h[c] (L - c), counts clipped at kHistCap
  if (L <= 0) return 0;
  int64_t x = L - 1;
  if (x > cmax) x = cmax;
  return L * P0[x] - P1[x];
}
__device__ int64_t S_of(const int64_t* P0, const int64_t* P1, int64_t H, int64_t cmax) {
  if (H >= cmax) return 0;
  const int64_t a0 = P0[cmax] - (H >= 0 ? P0[H] : 0);
  const int64_t a1 = P1[cmax] - (H >= 0 ? P1[H] : 0);
  return a1 - H * a0;
}

// Tile-class lists for the statistics kernels, in element order: elements of up to
// kTileSplit particles from the front of pl.tiles, of kTileMid + 1 .. kSmallCap from its
// back, and of kTileSplit + 1 .. kTileMid from the front of pl.tiles_mid.  The class flags
// ride in bits 28-39, 40-51 and 52-63 of a count's block scan (counts sum below 2^28 and a
// block holds kPlanThreads elements, so the fields never carry into each other).
constexpr int64_t kCountMask = (int64_t(1) << 28) - 1;
__device__ __forceinline__ int64_t tile_class_bits(bool valid, int32_t c, int split) {
  if (!valid || c > kSmallCap) return 0;
  return c <= split ? (int64_t(1) << 28) : (c <= kTileMid ? (int64_t(1) << 52) : (int64_t(1) << 40));
}
__device__ __forceinline__ void place_tile_class(Plan& pl, bool valid, int32_t c, int32_t e,
                                                 int32_t eb, int32_t ee, int64_t ex, int64_t tot,
                                                 int32_t& tA, int32_t& tB, int32_t& tM) {
  const int64_t bits = tile_class_bits(valid, c, pl.tile_split);
  if (bits == (int64_t(1) << 28)) pl.tiles[eb + tA + static_cast<int32_t>((ex >> 28) & 0xfff)] = e;
  else if (bits == (int64_t(1) << 40)) pl.tiles[ee - 1 - (tB + static_cast<int32_t>((ex >> 40) & 0xfff))] = e;
  else if (bits != 0) pl.tiles_mid[eb + tM + static_cast<int32_t>((ex >> 52) & 0xfff)] = e;
  tA += static_cast<int32_t>((tot >> 28) & 0xfff);
  tB += static_cast<int32_t>((tot >> 40) & 0xfff);
  tM += static_cast<int32_t>((tot >> 52) & 0xfff);
}

// Pass 1 for a single instance over many blocks: chunk k holds elements [k kPlanThreads,
// (k + 1) kPlanThreads).  plan_chunk_totals leaves each chunk's count sum with its tile-class
// counts packed above it (as pass 1's scan packs them; a chunk holds at most kPlanThreads
// elements) in tot[2 k], and its smallest and largest count in the two words of tot[2 k + 1].
__global__ void __launch_bounds__(kPlanThreads) plan_chunk_totals(Plan pl, int32_t ne, int64_t* tot) {
  __shared__ PlanShared sh;
  const int tid = threadIdx.x;
  const int32_t e = static_cast<int32_t>(blockIdx.x) * kPlanThreads + tid;
  const bool valid = e < ne;
  const int32_t c = valid ? pl.cnt[e] : 0;
  if (blockIdx.x == 0 && tid == 0) pl.scal[3] = 0;
  int64_t ptot;
  block_exclusive_scan<int64_t>(c | tile_class_bits(valid, c, pl.tile_split), sh.tmp64, ptot);
  int32_t lmin = valid ? c : 0x7fffffff, lmax = valid ? c : -1;
  for (int o = 16; o > 0; o >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(kFull, lmin, o));
    lmax = max(lmax, __shfl_xor_sync(kFull, lmax, o));
  }
  if ((tid & 31) == 0) { sh.vmin[tid >> 5] = lmin; sh.vmax[tid >> 5] = lmax; }
  __syncthreads();
  if (tid == 0) {
    int32_t a = 0x7fffffff, b = -1;
    for (int w = 0; w < kPlanThreads / 32; ++w) { a = min(a, sh.vmin[w]); b = max(b, sh.vmax[w]); }
    tot[2 * blockIdx.x] = ptot;
    int32_t* mm = reinterpret_cast<int32_t*>(tot + 2 * blockIdx.x + 1);
    mm[0] = a;
    mm[1] = b;
  }
}

// plan_chunk_offsets: chunk k's offsets and tile-class entries, from the totals of the
// chunks before it; the last chunk also writes the end offset, the class counts and the
// minimum and maximum count (scal 4, 5).  The same values as the one-block pass 1.
__global__ void __launch_bounds__(kPlanThreads) plan_chunk_offsets(Plan pl, int32_t ne, int nchunks,
                                                                    const int64_t* tot) {
  __shared__ PlanShared sh;
  const int tid = threadIdx.x;
  const int k = static_cast<int>(blockIdx.x);
  const bool last = k == nchunks - 1;
  if (tid < 32) {
    // counts and class counts of the chunks before k (all chunks for the last one's totals)
    int32_t cnt = 0, a = 0, b = 0, m = 0, mn = 0x7fffffff, mx = -1;
    for (int j = tid; j < nchunks; j += 32) {
      const int64_t t = tot[2 * j];
      if (j < k) {
        cnt += static_cast<int32_t>(t & kCountMask);
        a += static_cast<int32_t>((t >> 28) & 0xfff);
        b += static_cast<int32_t>((t >> 40) & 0xfff);
        m += static_cast<int32_t>((t >> 52) & 0xfff);
      }
      const int32_t* mm = reinterpret_cast<const int32_t*>(tot + 2 * j + 1);
      mn = min(mn, mm[0]);
      mx = max(mx, mm[1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(kFull, cnt, o);
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
      m += __shfl_xor_sync(kFull, m, o);
      mn = min(mn, __shfl_xor_sync(kFull, mn, o));
      mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if (tid == 0) {
      sh.carry[0] = cnt;
      sh.carry[1] = a;
      sh.carry[2] = b;
      sh.carry[3] = m;
      sh.carry[4] = mn;
      sh.carry[5] = mx;
    }
  }
  __syncthreads();
  const int32_t p0 = pl.ip0 ? static_cast<int32_t>(pl.ip0[0]) : 0;
  const int32_t carry = p0 + sh.carry[0];
  int32_t tA = sh.carry[1], tB = sh.carry[2], tM = sh.carry[3];
  const int32_t e = k * kPlanThreads + tid;
  const bool valid = e < ne;
  const int32_t c = valid ? pl.cnt[e] : 0;
  int64_t ptot;
  const int64_t pex = block_exclusive_scan<int64_t>(c | tile_class_bits(valid, c, pl.tile_split), sh.tmp64, ptot);
  place_tile_class(pl, valid, c, e, 0, ne, pex, ptot, tA, tB, tM);
  if (valid) {
    const int32_t o = carry + static_cast<int32_t>(pex & kCountMask);
    pl.off[e] = o;
    pl.foff[e] = o;
    pl.cursor[e] = o;
    if (c > kSmallCap) pl.big_list[atomicAdd(pl.scal + 3, 1)] = e;
  }
  if (last && tid == 0) {
    const int32_t end = carry + static_cast<int32_t>(ptot & kCountMask);
    pl.off[ne] = end;
    pl.foff[ne] = end;
    pl.scal[4] = sh.carry[4];
    pl.scal[5] = sh.carry[5];
    pl.scal[6] = tA;
    pl.scal[7] = tB;
    pl.scal[8] = tM;
  }
}

// One block per instance: elements [eb, ee) of the union grid, particle slots from p0.
// pass1_done: pass 1 (offsets, tile classes, min / max) was taken by plan_chunk_totals and
// plan_chunk_offsets; this block reads the minimum and maximum count they left in scal.
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(Plan pl, int32_t ne_all, int minnpel_one,
                                                             int allow_moves, int pass1_done) {
  __shared__ PlanShared sh;
  __shared__ int32_t hist[kHistCap + 1];
  const int tid = threadIdx.x;
  const int inst = blockIdx.x;
  const bool last = inst == static_cast<int>(gridDim.x) - 1;
  const int32_t eb = pl.ielem ? pl.ielem[inst] : 0, ee = pl.ielem ? pl.ielem[inst + 1] : ne_all;
  const int32_t ne = ee - eb;
  const int32_t p0 = pl.ip0 ? static_cast<int32_t>(pl.ip0[inst]) : 0;
  const int minnpel = pl.iminnpel ? pl.iminnpel[inst] : minnpel_one;
  int32_t* scal = pl.scal + 16 * inst;
  // pass 1: offsets of the element lists, min / max, big elements (no moves)
  int32_t carry = p0, lmin = 0x7fffffff, lmax = -1, tA = 0, tB = 0, tM = 0;
  if (tid == 0 && !pass1_done) scal[3] = 0;
  __syncthreads();
  // each pass's counts are loaded one pass ahead, so that the load overlaps the scan
  int32_t c_next = tid < ne && !pass1_done ? pl.cnt[eb + tid] : 0;
  for (int32_t base = 0; base < ne && !pass1_done; base += kPlanThreads) {
    const bool valid = base + tid < ne;
    const int32_t e = eb + base + tid;
    const int32_t c = c_next;
    c_next = base + kPlanThreads + tid < ne ? pl.cnt[e + kPlanThreads] : 0;
    int64_t ptot;
    const int64_t pex = block_exclusive_scan<int64_t>(c | tile_class_bits(valid, c, pl.tile_split), sh.tmp64, ptot);
    const int32_t ex = static_cast<int32_t>(pex & kCountMask), tot = static_cast<int32_t>(ptot & kCountMask);
    place_tile_class(pl, valid, c, e, eb, ee, pex, ptot, tA, tB, tM);
    if (valid) {
      pl.off[e] = carry + ex;
      pl.foff[e] = carry + ex;
      pl.cursor[e] = carry + ex;
      lmin = min(lmin, c);
      lmax = max(lmax, c);
      if (c > kSmallCap) pl.big_list[eb + atomicAdd(scal + 3, 1)] = e;
    }
    carry += tot;
  }
  if (tid == 0 && !pass1_done) {
    if (last) { pl.off[ee] = carry; pl.foff[ee] = carry; }
    scal[6] = tA;
    scal[7] = tB;
    scal[8] = tM;
  }
  for (int o = 16; o > 0; o >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(kFull, lmin, o));
    lmax = max(lmax, __shfl_xor_sync(kFull, lmax, o));
  }
  if ((tid & 31) == 0) { sh.vmin[tid >> 5] = lmin; sh.vmax[tid >> 5] = lmax; }
  __syncthreads();
  if (tid == 0) {
    int32_t a = 0x7fffffff, b = -1;
    for (int w = 0; w < kPlanThreads / 32; ++w) { a = min(a, sh.vmin[w]); b = max(b, sh.vmax[w]); }
    if (pass1_done) { a = scal[4]; b = scal[5]; }
    sh.cmin = a;
    sh.cmax = b;
    sh.need = allow_moves && minnpel > 0 && a < minnpel && (b - a) >= 2;
    scal[4] = a;
    scal[5] = b;
    if (!sh.need) { scal[0] = 0; scal[1] = 0; scal[2] = 0; }
  }
  __syncthreads();
  if (!sh.need) return;

  // pass 2: histogram of counts and its prefix sums P0[c] = #{c_e <= c}, P1[c] = sum c_e
  for (int i = tid; i <= kHistCap; i += kPlanThreads) hist[i] = 0;
  __syncthreads();
  for (int32_t e = eb + tid; e < ee; e += kPlanThreads) atomicAdd(&hist[min(pl.cnt[e], kHistCap)], 1);
  __syncthreads();
  int64_t* P0 = pl.hist + static_cast<size_t>(inst) * 2 * (kHistCap + 1);
  int64_t* P1 = P0 + (kHistCap + 1);
  {
    int64_t c0 = 0, c1 = 0;
    for (int base = 0; base <= kHistCap; base += kPlanThreads) {
      const int i = base + tid;
      const int64_t h = i <= kHistCap ? hist[i] : 0;
      int64_t t0, t1;
      const int64_t e0 = block_exclusive_scan<int64_t>(h, sh.tmp64, t0);
      const int64_t e1 = block_exclusive_scan<int64_t>(h * i, sh.tmp64, t1);
      if (i <= kHistCap) { P0[i] = c0 + e0 + h; P1[i] = c1 + e1 + h * i; }
      c0 += t0;
      c1 += t1;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const int64_t cmin = sh.cmin, cmax = sh.cmax < kHistCap ? sh.cmax : kHistCap;
    auto min_level = [&](int64_t t) {   // max{L in [cmin, minnpel] : D(L) <= t}
      int64_t lo = cmin, hi = minnpel;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (D_of(P0, P1, mid, cmax) <= t) lo = mid; else hi = mid - 1;
      }
      return lo;
    };
    auto max_level = [&](int64_t t) {   // min{H in [cmin, cmax] : S(H) <= t}
      int64_t lo = cmin, hi = cmax;
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (S_of(P0, P1, mid, cmax) <= t) hi = mid; else lo = mid + 1;
      }
      return lo;
    };
    int64_t lo = 0, hi = D_of(P0, P1, minnpel, cmax);
    while (lo < hi) {                   // first t at which the loop stops
      const int64_t mid = (lo + hi) / 2;
      const int64_t Lm = min_level(mid), Hm = max_level(mid);
      if (Lm >= minnpel || Hm - Lm <= 1) hi = mid; else lo = mid + 1;
    }
    const int64_t T = lo;
    sh.Tm = T;
    sh.L = min_level(T);
    sh.H = max_level(T);
    sh.r = T - D_of(P0, P1, sh.L, cmax);
    sh.rp = T - S_of(P0, P1, sh.H, cmax);
    scal[0] = static_cast<int32_t>(T);
    scal[3] = 0;
  }
  __syncthreads();
  // pass 3: gains, losses, final counts, offsets and the recipient / donor / big lists
  const int64_t L = sh.L, H = sh.H, r = sh.r, rp = sh.rp;
  int32_t cRankL = 0, cRankH = 0, cG = p0, cD = p0, cF = p0, cNR = 0, cND = 0;
  tA = 0;
  tB = 0;
  tM = 0;
  for (int32_t base = 0; base < ne; base += kPlanThreads) {
    const bool valid = base + tid < ne;
    const int32_t e = eb + base + tid;
    const int32_t c = valid ? pl.cnt[e] : 0;
    const int32_t atL = (valid && c <= L) ? 1 : 0;
    const int32_t atH = (valid && c >= H) ? 1 : 0;
    int32_t tot;
    const int32_t rankL = cRankL + block_exclusive_scan<int32_t>(atL, sh.tmp32, tot);
    cRankL += tot;
    const int32_t rankH = cRankH + block_exclusive_scan<int32_t>(atH, sh.tmp32, tot);
    cRankH += tot;
    int32_t g = 0, l = 0;
    if (valid) {
      if (c < L) g += static_cast<int32_t>(L - c);
      if (atL && rankL < r) g += 1;
      if (c > H) l += static_cast<int32_t>(c - H);
      if (atH && rankH < rp) l += 1;
    }
    const int32_t f = c + g - l;
    const int32_t go = cG + block_exclusive_scan<int32_t>(g, sh.tmp32, tot);
    cG += tot;
    const int32_t dof = cD + block_exclusive_scan<int32_t>(l, sh.tmp32, tot);
    cD += tot;
    int64_t ptot;
    const int64_t pex = block_exclusive_scan<int64_t>((valid ? f : 0) | tile_class_bits(valid, f, pl.tile_split),
                                                      sh.tmp64, ptot);
    const int32_t fo = cF + static_cast<int32_t>(pex & kCountMask);
    cF += static_cast<int32_t>(ptot & kCountMask);
    place_tile_class(pl, valid, f, e, eb, ee, pex, ptot, tA, tB, tM);
    const int32_t ri = cNR + block_exclusive_scan<int32_t>(g > 0 ? 1 : 0, sh.tmp32, tot);
    cNR += tot;
    const int32_t di = cND + block_exclusive_scan<int32_t>(l > 0 ? 1 : 0, sh.tmp32, tot);
    cND += tot;
    if (valid) {
      pl.gain[e] = g;
      pl.loss[e] = l;
      pl.goff[e] = go;
      pl.doff[e] = dof;
      pl.fin[e] = f;
      pl.foff[e] = fo;
      if (g > 0) pl.recips[eb + ri] = e;
      if (l > 0) pl.donors[eb + di] = e;
      if (f > kSmallCap) pl.big_list[eb + atomicAdd(scal + 3, 1)] = e;
    }
  }
  if (tid == 0) {
    scal[6] = tA;
    scal[7] = tB;
    scal[8] = tM;
    if (last) {
      pl.goff[ee] = cG;
      pl.doff[ee] = cD;
      pl.foff[ee] = cF;
    }
    scal[1] = cNR;
    scal[2] = cND;
  }
}

// Element lists: idx[off[e] .. off[e] + cnt[e]) holds the slots of the particles in e.
// An element id outside 0 .. ne - 1 (a caller's state) is skipped: the count kernel has
// left it out of the counts and reported it.  A thread takes kScatterPer particles, blockDim.x
// apart, and issues all their loads, then all their cursor atomics (one per run of lanes
// sharing an element), then all their stores, so that each kind is in flight together.
constexpr int kScatterPer = 8;
__global__ void scatter_kernel(const int32_t* __restrict__ elem, int64_t np, int32_t ne, int32_t* cursor,
                               int32_t* idx) {
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x * kScatterPer + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int e[kScatterPer];
  bool valid[kScatterPer];
#pragma unroll
  for (int k = 0; k < kScatterPer; ++k) {
    const int64_t i = i0 + static_cast<int64_t>(k) * blockDim.x;
    e[k] = i < np ? elem[i] : -1;
    valid[k] = i < np && e[k] >= 0 && e[k] < ne;
  }
  unsigned peers[kScatterPer];
  int base[kScatterPer];
#pragma unroll
  for (int k = 0; k < kScatterPer; ++k) {
    const unsigned active = __ballot_sync(kFull, valid[k]);
    peers[k] = 0u;
    base[k] = 0;
    if (valid[k]) {
      peers[k] = __match_any_sync(active, e[k]);
      if (lane == __ffs(peers[k]) - 1) base[k] = atomicAdd(cursor + e[k], __popc(peers[k]));
    }
  }
#pragma unroll
  for (int k = 0; k < kScatterPer; ++k) {
    if (valid[k]) {
      const int b = __shfl_sync(peers[k], base[k], __ffs(peers[k]) - 1);
      idx[b + __popc(peers[k] & ((1u << lane) - 1u))] =
          static_cast<int32_t>(i0 + static_cast<int64_t>(k) * blockDim.x);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Redistribution (Appendix B; reading: donors give their highest particle ids; a moved
// particle keeps its id, lands uniformly in the recipient and copies (U, omega, psi) of the
// recipient's resident of rank floor(u n) in ascending id, or of the lowest-id non-empty
// edge neighbour's when the recipient is empty; the source disc is re-applied).
// ---------------------------------------------------------------------------------------
constexpr int kRedistThreads = 256;
constexpr int kRedistCap = 4096;   // = PDFX_MAX_PER_ELEMENT

// Every instance in turn (its lists live in its element range, its moves in its slots).
template <typename T>
__global__ void __launch_bounds__(kRedistThreads) select_donors_kernel(Particles<T> p, Plan pl, int K) {
  __shared__ uint32_t spid[kRedistCap];
  __shared__ int32_t sslot[kRedistCap];
  for (int inst = 0; inst < K; ++inst) {
  const int32_t* sc = pl.scal + 16 * inst;
  const int32_t eb = pl.ielem ? pl.ielem[inst] : 0;
  const int32_t ndon = sc[0] > 0 ? sc[2] : 0;
  for (int32_t d = blockIdx.x; d < ndon; d += gridDim.x) {
    const int32_t e = pl.donors[eb + d];
    const int32_t n = min(pl.cnt[e], kRedistCap);
    const int32_t o = pl.off[e];
    const int32_t l = pl.loss[e];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int32_t s = pl.idx[o + j];
      sslot[j] = s;
      spid[j] = p.pid[s];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const uint32_t me = spid[j];
      int rank = 0;   // particles with a higher id
      for (int m = 0; m < n; ++m) rank += spid[m] > me;
      if (rank < l) pl.movers[pl.doff[e] + rank] = sslot[j];
    }
    __syncthreads();
  }
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedistThreads) apply_moves_kernel(
    Particles<T> p, Plan pl, int K, const InstDev<T>* inst_tab, int64_t np, const ElemGeo<T>* geo,
    const ElemTopo* topo, const uint32_t* stepc) {
  const uint32_t step = *stepc;
  extern __shared__ __align__(16) unsigned char dyn[];
  uint32_t* spid = reinterpret_cast<uint32_t*>(dyn);
  int32_t* sslot = reinterpret_cast<int32_t*>(dyn + 4 * kRedistCap);
  int32_t* sorted = reinterpret_cast<int32_t*>(dyn + 8 * kRedistCap);
  for (int inst = 0; inst < K; ++inst) {
  const int32_t* sc = pl.scal + 16 * inst;
  const int32_t eb = pl.ielem ? pl.ielem[inst] : 0;
  const int32_t nrec = sc[0] > 0 ? sc[1] : 0;
  const Model<T>& mi = inst_tab[inst].m;
  const T period_x = mi.period_x, sr = mi.src_r;
  const int source_on = mi.source_on;
  const uint32_t k0 = inst_tab[inst].k0, k1 = inst_tab[inst].k1;
  for (int32_t ri = blockIdx.x; ri < nrec; ri += gridDim.x) {
    const int32_t r = pl.recips[eb + ri];
    int32_t src = r;
    if (pl.cnt[r] == 0) {
      const ElemTopo t = topo[r];
      const int nbs[3] = {t.nb0, t.nb1, t.nb2};
      src = -1;
      for (int k = 0; k < 3; ++k)
        if (nbs[k] >= 0 && pl.cnt[nbs[k]] > 0 && (src < 0 || nbs[k] < src)) src = nbs[k];
    }
    const int32_t n = src >= 0 ? min(pl.cnt[src], kRedistCap) : 0;
    if (n > 0) {
      const int32_t o = pl.off[src];
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int32_t s = pl.idx[o + j];
        sslot[j] = s;
        spid[j] = p.pid[s];
      }
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const uint32_t me = spid[j];
        int rank = 0;
        for (int m = 0; m < n; ++m) rank += spid[m] < me;
        sorted[rank] = sslot[j];
      }
      __syncthreads();
    }
    const ElemGeo<T> g = geo[r];
    const int32_t g0 = pl.goff[r], gn = pl.gain[r];
    for (int j = threadIdx.x; j < gn; j += blockDim.x) {
      const int32_t k = g0 + j;
      const int32_t q = pl.movers[k];
      if (q < 0 || q >= np) { pl.mrecip[k] = -1; continue; }
      const uint32_t pid = p.pid[q];
      const uint4 rw = philox(make_uint4(pid, step, kPurRedist, 0u), k0, k1);
      const T s = sqrt(uniform01(rw.x, T(0)));
      const T t = uniform01(rw.y, T(0));
      Pos<T> P = triangle_point(g, s, t, period_x);
      pos_wrap(P, period_x);
      int32_t from = q;
      if (n > 0) {
        const double uu = uniform01(rw.z, 0.0);   // rank choice in double in both forms
        int jj = static_cast<int>(uu * static_cast<double>(n));
        if (jj >= n) jj = n - 1;
        from = sorted[jj];
      }
      double* mv = pl.mvals + static_cast<size_t>(k) * 7;
      mv[0] = pos_x(P);
      mv[1] = pos_y(P);
      mv[2] = static_cast<double>(p.u[from]);
      mv[3] = static_cast<double>(p.v[from]);
      mv[4] = static_cast<double>(p.w[from]);
      mv[5] = static_cast<double>(p.om[from]);
      bool insrc = false;
      if (source_on) {
        const T ddx = rel_x(P, mi.src_x, mi.src_xl, period_x), ddy = rel_y(P, mi.src_y, mi.src_yl);
        insrc = ddx * ddx + ddy * ddy <= sr * sr;
      }
      mv[6] = insrc ? 1.0 : static_cast<double>(p.psi[from]);
      pl.mrecip[k] = r;
    }
    __syncthreads();
  }
  }
}

template <typename T>
__global__ void commit_moves_kernel(Particles<T> p, Plan pl, int K, int64_t np, int32_t ne,
                                    unsigned long long* diag, int* err) {
  for (int inst = 0; inst < K; ++inst) {
  const int32_t T_moves = pl.scal[16 * inst];
  const int32_t p0 = pl.ip0 ? static_cast<int32_t>(pl.ip0[inst]) : 0;
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < T_moves; j += gridDim.x * blockDim.x) {
    const int32_t k = p0 + j;
    const int32_t q = pl.movers[k];
    const int32_t r = pl.mrecip[k];
    if (q < 0 || q >= np || r < 0 || r >= ne) {   // an inconsistent move table is an error
      atomicCAS(err, 0, PDFX_ERR_CAPACITY);
      continue;
    }
    const double* mv = pl.mvals + static_cast<size_t>(k) * 7;
    store_pos(p, q, pos_of(mv[0], mv[1], T(0)));
    p.u[q] = static_cast<T>(mv[2]);
    p.v[q] = static_cast<T>(mv[3]);
    p.w[q] = static_cast<T>(mv[4]);
    p.om[q] = static_cast<T>(mv[5]);
    p.psi[q] = static_cast<T>(mv[6]);
    p.elem[q] = r;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && T_moves > 0)
    atomicAdd(diag + kDiagMoves, static_cast<unsigned long long>(T_moves));
  }
}

// ---------------------------------------------------------------------------------------
// Per-element statistics and conditional means.
// ---------------------------------------------------------------------------------------
constexpr int kStatsThreads = 256;

template <typename T>
struct StatsSmem {
  T* u; T* v; T* w; T* om; T* psi;
  uint32_t* pid;
  int32_t* slot;
  uint16_t* perm;
  uint8_t* grp;
};

template <typename T>
__device__ __forceinline__ bool key_less(const StatsSmem<T>& s, const T* key, int a, int b, int N) {
  if (a >= N) return false;        // padding sorts last
  if (b >= N) return true;
  if (s.grp[a] != s.grp[b]) return s.grp[a] < s.grp[b];
  const T ka = key[a], kb = key[b];
  if (ka < kb) return true;
  if (kb < ka) return false;
  return s.pid[a] < s.pid[b];
}

// Bitonic sort of perm[0, P) (P a power of two) by (group, key, particle id).
template <typename T>
__device__ void bitonic_sort(const StatsSmem<T>& s, const T* key, int N, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int q = threadIdx.x; q < P / 2; q += blockDim.x) {
        const int lo = 2 * j * (q / j) + (q % j);
        const int hi = lo + j;
        const bool up = (lo & k) == 0;
        const int a = s.perm[lo], b = s.perm[hi];
        const bool swap = up ? key_less(s, key, b, a, N) : key_less(s, key, a, b, N);
        if (swap) { s.perm[lo] = b; s.perm[hi] = a; }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}

// Deterministic block sums of NV values (fixed reduction order).
template <int NV>
__device__ void block_sums(double (&v)[NV], double* red /* [32 * NV] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) red[wid * NV + k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * NV + threadIdx.x];
    red[32 * NV + threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = red[32 * NV + k];
  __syncthreads();
}

template <typename T>
__device__ void process_element(const StatsArgs<T>& a, int e, int N, int cap, unsigned char* raw,
                                int moves) {
  __shared__ double red[32 * 10 + 10];
  __shared__ int sh_n;
  // smem carve-up for cap entries
  StatsSmem<T> s;
  unsigned char* ptr = raw;
  auto take = [&](size_t bytes) { unsigned char* r = ptr; ptr += (bytes + 15) & ~size_t(15); return r; };
  s.u = reinterpret_cast<T*>(take(sizeof(T) * cap));
  s.v = reinterpret_cast<T*>(take(sizeof(T) * cap));
  s.w = reinterpret_cast<T*>(take(sizeof(T) * cap));
  s.om = reinterpret_cast<T*>(take(sizeof(T) * cap));
  s.psi = reinterpret_cast<T*>(take(sizeof(T) * cap));
  s.pid = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * cap));
  s.slot = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * cap));
  s.perm = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * cap));
  s.grp = reinterpret_cast<uint8_t*>(take(cap));

  const int tid = threadIdx.x;
  if (tid == 0) sh_n = 0;
  __syncthreads();
  // gather the element's particles: its list minus those moved out, plus those moved in
  const int32_t o = a.off[e], c = a.cnt[e];
  for (int j = tid; j < c; j += blockDim.x) {
    const int32_t q = a.idx[o + j];
    if (moves && a.p.elem[q] != e) continue;
    const int at = atomicAdd(&sh_n, 1);
    if (at < cap) s.slot[at] = q;
  }
  if (moves) {
    const int32_t gn = a.gain[e], g0 = a.goff[e];
    for (int j = tid; j < gn; j += blockDim.x) {
      const int32_t q = a.movers[g0 + j];
      if (q < 0 || q >= a.np) continue;
      const int at = atomicAdd(&sh_n, 1);
      if (at < cap) s.slot[at] = q;
    }
  }
  __syncthreads();
  const int n = min(min(sh_n, cap), N);
  if (tid == 0 && sh_n != N) atomicCAS(a.err, 0, PDFX_ERR_CAPACITY);
  for (int j = tid; j < n; j += blockDim.x) {
    const int32_t q = s.slot[j];
    s.u[j] = a.p.u[q];
    s.v[j] = a.p.v[q];
    s.w[j] = a.p.w[q];
    s.om[j] = a.p.om[q];
    s.psi[j] = a.p.psi[q];
    s.pid[j] = a.p.pid[q];
    s.grp[j] = 0;
  }
  int P = 1;
  while (P < n) P <<= 1;
  for (int j = tid; j < P; j += blockDim.x) s.perm[j] = static_cast<uint16_t>(j);
  __syncthreads();

  // effective bins (Sect. 3.5 reading): g_l = max(1, min(b_l, n / (g_1..g_{l-1} min_per_bin)));
  // Fox's projection (Eqs. 64-66): max(1, min(fox_bins, n / min_per_bin)) intervals
  const bool fox = a.cond_mode == 1;
  int g[3];
  if (fox) {
    int nc = n / a.min_per_bin;
    if (a.fox_bins < nc) nc = a.fox_bins;
    g[0] = nc < 1 ? 1 : nc;
    g[1] = g[2] = 1;
  } else {
    int Gp = 1;
    for (int l = 0; l < 3; ++l) {
      int cap_l = n / (Gp * a.min_per_bin);
      int gl = a.bins[l] < cap_l ? a.bins[l] : cap_l;
      if (gl < 1) gl = 1;
      g[l] = gl;
      Gp *= gl;
    }
  }
  // level 1: sort by (u, id)
  if (n > 1) bitonic_sort(s, s.u, n, P);

  // moments in sorted order (deterministic): means, then central moments
  {
    double m[5] = {0, 0, 0, 0, 0};
    for (int j = tid; j < n; j += blockDim.x) {
      const int q = s.perm[j];
      m[0] += static_cast<double>(s.u[q]);
      m[1] += static_cast<double>(s.v[q]);
      m[2] += static_cast<double>(s.w[q]);
      m[3] += static_cast<double>(s.om[q]);
      m[4] += static_cast<double>(s.psi[q]);
    }
    block_sums<5>(m, red);
    const double inv = n > 0 ? 1.0 / n : 0.0;
    const double mu = m[0] * inv, mv = m[1] * inv, mw = m[2] * inv, mo = m[3] * inv, mp = m[4] * inv;
    double c2[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = tid; j < n; j += blockDim.x) {
      const int q = s.perm[j];
      const double du = static_cast<double>(s.u[q]) - mu, dv = static_cast<double>(s.v[q]) - mv,
                   dw = static_cast<double>(s.w[q]) - mw, dp = static_cast<double>(s.psi[q]) - mp;
      c2[0] += du * du; c2[1] += dv * dv; c2[2] += dw * dw;
      c2[3] += du * dv; c2[4] += du * dw; c2[5] += dv * dw;
      c2[6] += dp * dp;
      c2[7] += du * dp; c2[8] += dv * dp; c2[9] += dw * dp;
    }
    block_sums<10>(c2, red);
    __shared__ double fox_f[3], fox_m[3];
    if (tid == 0) {
      double* em = a.emom + static_cast<size_t>(kNS) * e;
      em[0] = static_cast<double>(n);
      em[1] = mu; em[2] = mv; em[3] = mw;
      for (int k = 0; k < 6; ++k) em[4 + k] = c2[k] * inv;
      em[10] = mo; em[11] = mp; em[12] = c2[6] * inv;
      a.gbin[3 * e] = g[0];
      a.gbin[3 * e + 1] = g[1];
      a.gbin[3 * e + 2] = g[2];
      if (fox) {
        double loc[kNS], uphi[3];
        for (int k = 0; k < kNS; ++k) loc[k] = em[k];
        for (int k = 0; k < 3; ++k) uphi[k] = c2[7 + k] * inv;
        fox_factors(loc, uphi, fox_f);
        fox_m[0] = mu; fox_m[1] = mv; fox_m[2] = mw;
      }
    }
    __syncthreads();
    if (fox && n > 1) {
      // Eq. 64: sort once more, one group, by the projected velocity.  Its key takes the
      // place of omega, whose moments are done; omega is copied out from the particle
      // arrays, which this kernel does not write.
      for (int j = tid; j < n; j += blockDim.x) {
        s.om[j] = static_cast<T>(fox_f[0] * (static_cast<double>(s.u[j]) - fox_m[0]) +
                                 fox_f[1] * (static_cast<double>(s.v[j]) - fox_m[1]) +
                                 fox_f[2] * (static_cast<double>(s.w[j]) - fox_m[2]));
        s.grp[j] = 0;
      }
      __syncthreads();
      bitonic_sort(s, s.om, n, P);
    }
  }
  // levels 2 and 3: sort each group of the previous level by (v, id), then (w, id)
  if (!fox) {
    int Gprev = g[0];
    const T* keys[2] = {s.v, s.w};
    for (int l = 1; l < 3; ++l) {
      if (g[l] > 1) {
        for (int j = tid; j < n; j += blockDim.x)
          s.grp[s.perm[j]] = static_cast<uint8_t>((static_cast<int64_t>(Gprev) * j) / n);
        __syncthreads();
        bitonic_sort(s, keys[l - 1], n, P);
      }
      Gprev *= g[l];
    }
  }
  // Appendix A: bin i = G n / N, conditional means, conditioning pointers
  const int G = g[0] * g[1] * g[2];
  double* vc = a.vcce + static_cast<size_t>(a.G) * e;
  for (int i = tid; i < a.G; i += blockDim.x) {
    if (i < G && n > 0) {
      const int lo = static_cast<int>((static_cast<int64_t>(i) * n + G - 1) / G);
      const int hi = static_cast<int>((static_cast<int64_t>(i + 1) * n + G - 1) / G);
      double sum = 0.0;
      for (int j = lo; j < hi; ++j) sum += static_cast<double>(s.psi[s.perm[j]]);
      vc[i] = sum / (hi - lo);
    } else {
      vc[i] = 0.0;
    }
  }
  if (a.resort) {
    const int32_t fo = a.foff[e];
    for (int j = tid; j < n; j += blockDim.x) {
      const int q = s.perm[j];
      const int32_t d = fo + j;
      if (d >= a.np) break;
      const int32_t src = s.slot[q];
      store_pos(a.out, d, load_pos(a.p, src));
      a.out.u[d] = s.u[q];
      a.out.v[d] = s.v[q];
      a.out.w[d] = s.w[q];
      a.out.om[d] = a.p.om[src];
      a.out.psi[d] = s.psi[q];
      a.out.pid[d] = s.pid[q];
      a.out.elem[d] = e;
      a.out.cp[d] = static_cast<uint8_t>((static_cast<int64_t>(G) * j) / n);
    }
  } else {
    for (int j = tid; j < n; j += blockDim.x)
      a.p.cp[s.slot[s.perm[j]]] = static_cast<uint8_t>((static_cast<int64_t>(G) * j) / n);
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kStatsThreads) stats_big_kernel(const StatsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char raw[];
  for (int inst = 0; inst < a.K; ++inst) {
  const int32_t* sc = a.scal + 16 * inst;
  const int eb = a.ielem ? a.ielem[inst] : 0;
  const int moves = sc[0] > 0;
  const int nbig = sc[3];
  for (int b = blockIdx.x; b < nbig; b += gridDim.x) {
    const int e = a.big_list[eb + b];
    const int N = moves ? a.fin[e] : a.cnt[e];
    if (N <= kTileBig && a.cond_mode != 1) continue;   // rank_big_kernel's (hierarchical bins)
    if (N > kBigCap) {
      if (threadIdx.x == 0) {
        atomicAdd(a.diag + kDiagCapacity, 1ull);
        atomicCAS(a.err, 0, PDFX_ERR_CAPACITY);
      }
      continue;
    }
    process_element(a, e, N, kBigCap, raw, moves);
  }
  }
}

template <typename T>
size_t stats_smem_bytes(int cap) {
  auto r = [](size_t b) { return (b + 15) & ~size_t(15); };
  return 5 * r(sizeof(T) * cap) + r(4 * cap) + r(4 * cap) + r(2 * cap) + r(cap);
}

// The nodal moments: the mean of each element statistic over the node's elements that hold
// particles (the count, statistic 0, at least one), summed in the order of the node's element
// list.  One thread per node and statistic (k = kNS n + s), so that the FP64 additions spread
// over every SM and the stores are contiguous.  The count is tested on its bits (for a
// non-negative or NaN double, x >= 1 exactly when its bits as a signed integer are at least
// those of 1.0), which keeps the test off the FP64 pipe; the mean is the sum times 1/c from a
// table of correctly rounded reciprocals (within one rounding of the quotient), since an FP64
// division per output would make this kernel FP64-bound on this GPU.
struct NodeRecip {
  double v[65];
  constexpr NodeRecip() : v() {
    for (int i = 1; i < 65; ++i) v[i] = 1.0 / i;
  }
};
__device__ const NodeRecip g_node_recip{};

__global__ void node_average_kernel(const double* __restrict__ emom, const int32_t* __restrict__ ne_off,
                                    const int32_t* __restrict__ ne_list, int32_t nn, double* nmom) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= static_cast<int64_t>(nn) * kNS) return;
  const int32_t n = static_cast<int32_t>(k / kNS);
  const int s = static_cast<int>(k - static_cast<int64_t>(n) * kNS);
  double acc = 0.0;
  int c = 0;
  for (int i = ne_off[n]; i < ne_off[n + 1]; ++i) {
    const double* em = emom + static_cast<size_t>(kNS) * ne_list[i];
    if (__double_as_longlong(em[0]) < 0x3FF0000000000000LL) continue;
    acc += em[s];
    ++c;
  }
  const double r = c <= 0 ? 0.0 : (c < 65 ? g_node_recip.v[c] : 1.0 / c);
  nmom[k] = acc * r;
}

template <typename T> bool redist_configured[kMaxDevices];
template <typename T> bool stats_configured[kMaxDevices];

}  // namespace

int launch_plan(Plan& pl, int32_t ne, int K, int minnpel, int allow_moves, cudaStream_t s) {
  // one instance with its histogram scratch: pass 1 over many blocks (the chunk totals live
  // in the histogram, which only the later passes of the particle-number control use), then
  // the one-block kernel for those passes, which returns at once when no particle moves
  const int nchunks = ne > 0 ? (ne + kPlanThreads - 1) / kPlanThreads : 1;
  if (K <= 1 && pl.hist && nchunks <= kHistCap) {
    plan_chunk_totals<<<static_cast<unsigned>(nchunks), kPlanThreads, 0, s>>>(pl, ne, pl.hist);
    plan_chunk_offsets<<<static_cast<unsigned>(nchunks), kPlanThreads, 0, s>>>(pl, ne, nchunks, pl.hist);
    plan_kernel<<<1, kPlanThreads, 0, s>>>(pl, ne, minnpel, allow_moves, 1);
    return 3;
  }
  plan_kernel<<<static_cast<unsigned>(K > 0 ? K : 1), kPlanThreads, 0, s>>>(pl, ne, minnpel, allow_moves, 0);
  return 1;
}

void launch_scatter(const int32_t* elem, int64_t np, int32_t ne, Plan& pl, cudaStream_t s) {
  if (np <= 0) return;
  const int64_t per_block = 256 * kScatterPer;
  scatter_kernel<<<static_cast<unsigned>((np + per_block - 1) / per_block), 256, 0, s>>>(elem, np, ne, pl.cursor,
                                                                                          pl.idx);
}

template <typename T>
void launch_redistribute(Particles<T> p, Plan& pl, int K, const InstDev<T>* inst, int32_t ne,
                         int64_t np, const ElemGeo<T>* geo, const ElemTopo* topo, const uint32_t* stepc,
                         int num_sms, unsigned long long* diag, int* err, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(num_sms > 0 ? num_sms : 1);
  const size_t apply_smem = 12 * static_cast<size_t>(kRedistCap);
  if (first_use_on_device(redist_configured<T>)) {
    cudaFuncSetAttribute(apply_moves_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(apply_smem));
  }
  select_donors_kernel<T><<<grid, kRedistThreads, 0, s>>>(p, pl, K);
  apply_moves_kernel<T><<<grid, kRedistThreads, apply_smem, s>>>(p, pl, K, inst, np, geo, topo, stepc);
  commit_moves_kernel<T><<<grid, 256, 0, s>>>(p, pl, K, np, ne, diag, err);
}

template <typename T>
void launch_stats(const StatsArgs<T>& a, int num_sms, cudaStream_t s, const SideStreams* side) {
  const size_t big = stats_smem_bytes<T>(kBigCap);
  static_assert(5 * 8 * kBigCap + 11 * kBigCap <= 227 * 1024, "large-element tile exceeds shared memory");
  if (first_use_on_device(stats_configured<T>)) {
    cudaFuncSetAttribute(stats_big_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(big));
  }
  // The tile classes and the large-element kernel take disjoint elements and write disjoint
  // outputs: with the context's side streams they run as parallel branches (the 513..768
  // class and the large-element list's 769..1024 on side[0]; the class of up to 256 and the
  // large-element kernel on side[1]; the
  // 257..512 class on s), so that each one's last wave, and its blocks of other classes,
  // which return at once, overlap the others' work; s then waits for both branches.
  const bool fork = side && side->ok;
  cudaStream_t s_large = s, s_small = s;
  if (fork) {
    cudaEventRecord(side->ev[0], s);
    cudaStreamWaitEvent(side->side[0], side->ev[0], 0);
    cudaStreamWaitEvent(side->side[1], side->ev[0], 0);
    s_large = side->side[0];
    s_small = side->side[1];
  }
  launch_stats_tiles<T>(a, num_sms, s_small, s, s_large);
  stats_big_kernel<T><<<static_cast<unsigned>(num_sms > 0 ? num_sms : 1), kStatsThreads, big, s_small>>>(a);
  if (fork) {
    cudaEventRecord(side->ev[1], side->side[0]);
    cudaEventRecord(side->ev[2], side->side[1]);
    cudaStreamWaitEvent(s, side->ev[1], 0);
    cudaStreamWaitEvent(s, side->ev[2], 0);
  }
}

void launch_node_average(const double* emom, const int32_t* ne_off, const int32_t* ne_list,
                         int32_t nn, double* nmom, cudaStream_t s) {
  if (nn <= 0) return;
  const int64_t work = static_cast<int64_t>(nn) * kNS;
  node_average_kernel<<<static_cast<unsigned>((work + 255) / 256), 256, 0, s>>>(emom, ne_off, ne_list, nn, nmom);
}

namespace {

// Eq. 26's denominator: the largest ||(<U>, <V>, <W>, <omega>, <psi>)||_2 over the nodes.
__global__ void __launch_bounds__(256) cfl_norm_kernel(const double* __restrict__ nmom, int32_t nn,
                                                      double* out) {
  __shared__ double red[8];
  double m = 0.0;
  for (int32_t n = threadIdx.x; n < nn; n += blockDim.x) {
    const double* z = nmom + static_cast<size_t>(kNS) * n;
    const double v = sqrt(z[1] * z[1] + z[2] * z[2] + z[3] * z[3] + z[10] * z[10] + z[11] * z[11]);
    m = fmax(m, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    out[0] = m;
  }
}

}  // namespace

void launch_cfl_norm(const double* nmom, int32_t nn, double* out, cudaStream_t s) {
  cfl_norm_kernel<<<1, 256, 0, s>>>(nmom, nn, out);
}

namespace {

// Eq. 39 with Eq. 40's shapefunction derivatives, per element, for nq nodal quantities
// q[n * stride + off + i]: out[e][2 i + 0/1] = (dQ_i/dx, dQ_i/dy).  The stored node x are the
// canonical images: x differences are taken as minimum images of the element's period (its
// instance's in a batch, einst and inst non-null).
template <typename T>
__global__ void elem_gradient_kernel(const ElemGeo<T>* __restrict__ geo, const ElemTopo* __restrict__ topo,
                                     int32_t ne, double L0, const int32_t* __restrict__ einst,
                                     const InstDev<T>* __restrict__ inst, const double* __restrict__ q,
                                     int stride, int off, int nq, double* __restrict__ out) {
  const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const ElemGeo<T> g = geo[e];
  const ElemTopo t = topo[e];
  const double L = einst ? static_cast<double>(inst[einst[e]].m.period_x) : L0;
  const double xBA = min_image(node_x(g, 1) - node_x(g, 0), L);
  const double yBA = node_y(g, 1) - node_y(g, 0);
  const double xCA = min_image(node_x(g, 2) - node_x(g, 0), L);
  const double yCA = node_y(g, 2) - node_y(g, 0);
  const double inv = static_cast<double>(g.inv2a);
  const double dNx0 = (-yCA + yBA) * inv, dNx1 = yCA * inv, dNx2 = -yBA * inv;
  const double dNy0 = (xCA - xBA) * inv, dNy1 = -xCA * inv, dNy2 = xBA * inv;
  for (int i = 0; i < nq; ++i) {
    const double q0 = q[static_cast<size_t>(stride) * t.n0 + off + i];
    const double q1 = q[static_cast<size_t>(stride) * t.n1 + off + i];
    const double q2 = q[static_cast<size_t>(stride) * t.n2 + off + i];
    out[static_cast<size_t>(2 * nq) * e + 2 * i] = dNx0 * q0 + dNx1 * q1 + dNx2 * q2;
    out[static_cast<size_t>(2 * nq) * e + 2 * i + 1] = dNy0 * q0 + dNy1 * q1 + dNy2 * q2;
  }
}

// Transfer to nodes: the mean of w element values over the elements around each node
// (ascending element id).
__global__ void node_mean_kernel(const int32_t* __restrict__ ne_off, const int32_t* __restrict__ ne_list,
                                 int32_t nn, const double* __restrict__ ev, int w, double* __restrict__ out) {
  const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int32_t a = ne_off[n], b = ne_off[n + 1];
  for (int k = 0; k < w; ++k) {
    double s = 0.0;
    for (int32_t i = a; i < b; ++i) s += ev[static_cast<size_t>(w) * ne_list[i] + k];
    out[static_cast<size_t>(w) * n + k] = b > a ? s / (b - a) : 0.0;
  }
}

// The nodal fields the statistics provide: <U_i>, d<U_i>/dx_j, laplacians, <u_i u_j>, <omega>.
template <typename T>
__global__ void write_fields_kernel(int32_t nn, const double* __restrict__ nmom,
                                    const double* __restrict__ g1, const double* __restrict__ g2,
                                    T* __restrict__ F) {
  const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const double* m = nmom + static_cast<size_t>(kNS) * n;
  T* f = F + static_cast<size_t>(kNF) * n;
  for (int i = 0; i < 3; ++i) f[i] = static_cast<T>(m[1 + i]);
  for (int k = 0; k < 6; ++k) f[5 + k] = static_cast<T>(g1[6 * static_cast<size_t>(n) + k]);
  // g2[n][12]: (d/dx, d/dy) of each of the 6 first derivatives, (dU_i/dx at 2i, dU_i/dy at 2i+1)
  for (int i = 0; i < 3; ++i)
    f[11 + i] = static_cast<T>(g2[12 * static_cast<size_t>(n) + 4 * i] + g2[12 * static_cast<size_t>(n) + 4 * i + 3]);
  for (int k = 0; k < 6; ++k) f[23 + k] = static_cast<T>(m[4 + k]);
  f[29] = static_cast<T>(m[10]);
}

}  // namespace

template <typename T>
void launch_derive_fields(const ElemGeo<T>* geo, const ElemTopo* topo, int32_t ne, double period_x,
                          const int32_t* einst, const InstDev<T>* inst, const int32_t* ne_off,
                          const int32_t* ne_list, int32_t nn, const double* nmom, double* scratch,
                          T* fields, cudaStream_t s) {
  if (ne <= 0 || nn <= 0) return;
  double* eg1 = scratch;                                   // [ne][6]
  double* ng1 = eg1 + 6 * static_cast<size_t>(ne);         // [nn][6]
  double* eg2 = ng1 + 6 * static_cast<size_t>(nn);         // [ne][12]
  double* ng2 = eg2 + 12 * static_cast<size_t>(ne);        // [nn][12]
  const unsigned be = static_cast<unsigned>((ne + 127) / 128), bn = static_cast<unsigned>((nn + 127) / 128);
  elem_gradient_kernel<T><<<be, 128, 0, s>>>(geo, topo, ne, period_x, einst, inst, nmom, kNS, 1, 3, eg1);
  node_mean_kernel<<<bn, 128, 0, s>>>(ne_off, ne_list, nn, eg1, 6, ng1);
  elem_gradient_kernel<T><<<be, 128, 0, s>>>(geo, topo, ne, period_x, einst, inst, ng1, 6, 0, 6, eg2);
  node_mean_kernel<<<bn, 128, 0, s>>>(ne_off, ne_list, nn, eg2, 12, ng2);
  write_fields_kernel<T><<<bn, 128, 0, s>>>(nn, nmom, ng1, ng2, fields);
}

namespace {

// Eq. 31 (rho = 1) on each particle: U -= corr of its element, corr[e][2] = dt grad(dP).
template <typename T>
__global__ void correct_velocity_kernel(Particles<T> p, int64_t np, const double* __restrict__ corr) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int e = p.elem[i];
  p.u[i] = static_cast<T>(static_cast<double>(p.u[i]) - corr[2 * static_cast<size_t>(e)]);
  p.v[i] = static_cast<T>(static_cast<double>(p.v[i]) - corr[2 * static_cast<size_t>(e) + 1]);
}

__global__ void scale_kernel(int64_t n, double f, double* __restrict__ v) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) v[i] *= f;
}

// Eq. 31 shifts every particle of an element by the same vector, so the element's mean
// velocity moves by it and its central moments and conditioning order stay: emom means of
// U and V of the elements that hold particles -= corr.
__global__ void shift_means_kernel(int32_t ne, const double* __restrict__ corr, double* __restrict__ emom) {
  const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double* em = emom + static_cast<size_t>(kNS) * e;
  if (em[0] < 1.0) return;
  em[1] -= corr[2 * static_cast<size_t>(e)];
  em[2] -= corr[2 * static_cast<size_t>(e) + 1];
}

}  // namespace

template <typename T>
void launch_correction_field(const ElemGeo<T>* geo, const ElemTopo* topo, int32_t ne, double period_x,
                             const int32_t* einst, const InstDev<T>* inst, const double* dp, double dt,
                             double* corr, cudaStream_t s) {
  if (ne <= 0) return;
  elem_gradient_kernel<T><<<static_cast<unsigned>((ne + 127) / 128), 128, 0, s>>>(
      geo, topo, ne, period_x, einst, inst, dp, 1, 0, 1, corr);
  const int64_t n = 2 * static_cast<int64_t>(ne);
  scale_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(n, dt, corr);
}

template <typename T>
void launch_apply_correction(Particles<T> p, int64_t np, const double* corr, cudaStream_t s) {
  if (np > 0)
    correct_velocity_kernel<T><<<static_cast<unsigned>((np + 255) / 256), 256, 0, s>>>(p, np, corr);
}

void launch_shift_means(int32_t ne, const double* corr, double* emom, cudaStream_t s) {
  if (ne > 0) shift_means_kernel<<<static_cast<unsigned>((ne + 127) / 128), 128, 0, s>>>(ne, corr, emom);
}

template <typename T>
void launch_correct_velocity(const ElemGeo<T>* geo, const ElemTopo* topo, int32_t ne, double period_x,
                             const int32_t* einst, const InstDev<T>* inst, const double* dp,
                             double* egrad, Particles<T> p, int64_t np, double dt, cudaStream_t s) {
  launch_correction_field<T>(geo, topo, ne, period_x, einst, inst, dp, dt, egrad, s);
  launch_apply_correction<T>(p, np, egrad, s);
}

template void launch_correction_field<float>(const ElemGeo<float>*, const ElemTopo*, int32_t, double,
                                             const int32_t*, const InstDev<float>*, const double*, double,
                                             double*, cudaStream_t);
template void launch_correction_field<double>(const ElemGeo<double>*, const ElemTopo*, int32_t, double,
                                              const int32_t*, const InstDev<double>*, const double*, double,
                                              double*, cudaStream_t);
template void launch_apply_correction<float>(Particles<float>, int64_t, const double*, cudaStream_t);
template void launch_apply_correction<double>(Particles<double>, int64_t, const double*, cudaStream_t);

template void launch_correct_velocity<float>(const ElemGeo<float>*, const ElemTopo*, int32_t, double,
                                             const int32_t*, const InstDev<float>*, const double*,
                                             double*, Particles<float>, int64_t, double, cudaStream_t);
template void launch_correct_velocity<double>(const ElemGeo<double>*, const ElemTopo*, int32_t, double,
                                              const int32_t*, const InstDev<double>*, const double*,
                                              double*, Particles<double>, int64_t, double, cudaStream_t);

template void launch_derive_fields<float>(const ElemGeo<float>*, const ElemTopo*, int32_t, double,
                                          const int32_t*, const InstDev<float>*, const int32_t*,
                                          const int32_t*, int32_t, const double*, double*, float*,
                                          cudaStream_t);
template void launch_derive_fields<double>(const ElemGeo<double>*, const ElemTopo*, int32_t, double,
                                           const int32_t*, const InstDev<double>*, const int32_t*,
                                           const int32_t*, int32_t, const double*, double*, double*,
                                           cudaStream_t);

#define PDFX_INSTANTIATE(T)                                                                    \
  template void launch_redistribute<T>(Particles<T>, Plan&, int, const InstDev<T>*, int32_t,   \
                                       int64_t, const ElemGeo<T>*, const ElemTopo*,            \
                                       const uint32_t*,                                        \
                                       int, unsigned long long*, int*, cudaStream_t);          \
  template void launch_stats<T>(const StatsArgs<T>&, int, cudaStream_t, const SideStreams*);
PDFX_INSTANTIATE(double)
PDFX_INSTANTIATE(float)
#undef PDFX_INSTANTIATE

}  // namespace pdfx
