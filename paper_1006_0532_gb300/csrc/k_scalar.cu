// Scalar statistics of probe elements (Sect. 4.1.2, Figs. 12-15; Eqs. 67-69).
//
// One thread per particle slot: a particle of a probe element adds to its element's bin
// count and to fixed-point sums of its conditional mean <phi|V> and of psi - <phi|V> in
// its psi bin, and to the element's count, sum, minimum and maximum of psi; a second pass
// adds the powers of psi - <phi>.  Integer atomics make every sum independent of the order
// in which particles arrive, so the results are the same run after run.  One thread per
// probe element then forms, per bin, Eq. 68's phi~ (the bin average of <phi|V>), the
// conditional diffusion t_m <Gamma lap phi | psi> (the bin average of <phi|V> - psi) and
// Eq. 67's conditional dissipation t_m <2 Gamma (grad phi)^2 | psi> at the bin centre on
// the empirical PDF, and the element's first four moments.
#include "pdfx_device.cuh"
#include "pdfx_internal.h"

namespace pdfx {
namespace {

// Fixed-point scales.  The sums hold at most PDFX_MAX_PER_ELEMENT = 4096 terms; for a scalar
// within [-1, 2] (IECM mixes toward bin means of values in [0, 1] and the source sets 1) a
// bin term is below 2^2 in magnitude and a fourth power below 2^7, so 2^46 and 2^40 keep
// the sums inside int64.
constexpr double kFixS = 70368744177664.0;   // 2^46: bin sums and the sum of psi
constexpr double kFixM = 1099511627776.0;    // 2^40: sums of powers of psi - <phi>

__device__ __forceinline__ unsigned long long fix(double x, double scale) {
  return static_cast<unsigned long long>(__double2ll_rn(x * scale));
}
__device__ __forceinline__ double unfix(unsigned long long v, double scale) {
  return static_cast<double>(static_cast<long long>(v)) / scale;
}
// Order-preserving map of a double onto unsigned integers (-0 as +0) and its inverse.
__device__ __forceinline__ unsigned long long ord64(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x + 0.0));
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord64(unsigned long long k) {
  const unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double(static_cast<long long>(b));
}

__device__ __forceinline__ int psi_bin(double psi, int nb) {
  const int b = static_cast<int>(floor(psi * nb));
  return b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
}

template <typename T>
__global__ void scalar_sums_kernel(const Particles<T> p, int64_t np, const int32_t* __restrict__ probe,
                                   const double* __restrict__ vcce, int G, int nb, ScalarAcc acc) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < np;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int e = p.elem[i];
    const int j = probe[e];
    if (j < 0) continue;
    const double psi = static_cast<double>(p.psi[i]);
    const double c = vcce[static_cast<size_t>(e) * G + p.cp[i]];
    const size_t o = static_cast<size_t>(j) * nb + psi_bin(psi, nb);
    atomicAdd(acc.count + o, 1);
    atomicAdd(acc.sc + o, fix(c, kFixS));
    atomicAdd(acc.sd + o, fix(psi - c, kFixS));
    atomicAdd(acc.n + j, 1);
    atomicAdd(acc.s1 + j, fix(psi, kFixS));
    atomicMin(acc.lo + j, ord64(psi));
    atomicMax(acc.hi + j, ord64(psi));
  }
}

template <typename T>
__global__ void scalar_moments_kernel(const Particles<T> p, int64_t np, const int32_t* __restrict__ probe,
                                      ScalarAcc acc) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < np;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int j = probe[p.elem[i]];
    if (j < 0) continue;
    const double mean = unfix(acc.s1[j], kFixS) / acc.n[j];
    const double d = static_cast<double>(p.psi[i]) - mean;
    const double d2 = d * d, d3 = d2 * d;
    atomicAdd(acc.m + 3 * j, fix(d2, kFixM));
    atomicAdd(acc.m + 3 * j + 1, fix(d3, kFixM));
    atomicAdd(acc.m + 3 * j + 2, fix(d3 * d, kFixM));
  }
}

__global__ void scalar_finish_kernel(int n, int nb, ScalarAcc acc, ScalarOut out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int N = acc.n[j];
  double* m = out.mom + 6 * j;
  if (N > 0) {
    m[0] = unfix(acc.s1[j], kFixS) / N;
    m[1] = unfix(acc.m[3 * j], kFixM) / N;
    m[2] = unfix(acc.m[3 * j + 1], kFixM) / N;
    m[3] = unfix(acc.m[3 * j + 2], kFixM) / N;
    m[4] = unord64(acc.lo[j]);
    m[5] = unord64(acc.hi[j]);
  } else {
    for (int k = 0; k < 6; ++k) m[k] = 0.0;
  }
  const double dpsi = 1.0 / nb;
  long long cum = 0;   // fixed-point sum of psi - <phi|V> over the bins below
  for (int b = 0; b < nb; ++b) {
    const size_t o = static_cast<size_t>(j) * nb + b;
    const int cnt = acc.count[o];
    const long long sd = static_cast<long long>(acc.sd[o]);
    out.count[o] = cnt;
    if (cnt > 0) {
      out.phit[o] = unfix(acc.sc[o], kFixS) / cnt;
      out.cdiff[o] = -(static_cast<double>(sd) / kFixS) / cnt;
      out.cdiss[o] = -2.0 * dpsi * (static_cast<double>(cum) / kFixS +
                                    0.5 * (static_cast<double>(sd) / kFixS)) / cnt;
    } else {
      out.phit[o] = out.cdiff[o] = out.cdiss[o] = 0.0;
    }
    cum += sd;
  }
}

}  // namespace

template <typename T>
void launch_scalar_stats(const Particles<T>& p, int64_t np, const int32_t* probe, const double* vcce,
                         int G, int n, int nb, const ScalarAcc& acc, const ScalarOut& out,
                         int num_sms, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(4 * (num_sms > 0 ? num_sms : 1));
  if (np > 0) {
    scalar_sums_kernel<T><<<grid, 256, 0, s>>>(p, np, probe, vcce, G, nb, acc);
    scalar_moments_kernel<T><<<grid, 256, 0, s>>>(p, np, probe, acc);
  }
  scalar_finish_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, nb, acc, out);
}

template void launch_scalar_stats<float>(const Particles<float>&, int64_t, const int32_t*,
                                         const double*, int, int, int, const ScalarAcc&,
                                         const ScalarOut&, int, cudaStream_t);
template void launch_scalar_stats<double>(const Particles<double>&, int64_t, const int32_t*,
                                          const double*, int, int, int, const ScalarAcc&,
                                          const ScalarOut&, int, cudaStream_t);

}  // namespace pdfx
