// Element and nodal statistics with conditional means for a caller's particle state,
// computed without allocating device memory.
//
// Some callers cannot call cudaMalloc while they run: applications that hand a fixed
// device-memory pool to their own allocator and forbid any other, long-running services
// that must keep a memory footprint fixed at load time, and loops that cannot afford the
// device-wide synchronisation an allocation may cause.  For them this entry point keeps
// all of its scratch in one file-scope device array of fixed size, reserved when the
// library is loaded and held by every GPU that loads it until the process exits.
#include <mutex>

#include "pdfx_internal.h"

namespace pdfx {

namespace {

constexpr int64_t kNaMaxParticles = int64_t(1) << 20;   // PDFX_NOALLOC_MAX_PARTICLES
constexpr int32_t kNaMaxElements = 1 << 16;             // PDFX_NOALLOC_MAX_ELEMENTS
constexpr size_t kNaP = static_cast<size_t>(kNaMaxParticles);
constexpr size_t kNaE = static_cast<size_t>(kNaMaxElements) + 1;

// Layout (int32 words): element lists [P], particle ids [P], counts [E], list offsets [E],
// final offsets [E], cursors [E], large-element list [E], tile-class lists [E] and [E], plan
// scalars [16].
constexpr size_t kNaWords = 2 * kNaP + 7 * kNaE + 16;
constexpr size_t kNaBytes = ((4 * kNaWords + 255) / 256) * 256;
static_assert(kNaMaxParticles == PDFX_NOALLOC_MAX_PARTICLES, "header limit");
static_assert(kNaMaxElements == PDFX_NOALLOC_MAX_ELEMENTS, "header limit");

__device__ __align__(256) unsigned char g_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return PDFX_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return PDFX_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return PDFX_OK;
}

__global__ void iota_kernel(uint32_t* id, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) id[i] = static_cast<uint32_t>(i);
}

}  // namespace

int element_stats_noalloc(Ctx& c, int64_t np, const double* u, const double* v, const double* w,
                          const double* om, const double* psi, const int32_t* elem, double* emom,
                          double* vcce, int32_t* gbin, uint8_t* cp, double* nmom, cudaStream_t s) {
  if (!c.have_grid) return PDFX_ERR_ORDER;
  if (np < 0 || np > kNaMaxParticles || c.ne > kNaMaxElements) return PDFX_ERR_ARG;
  if (np > 0 && (!u || !v || !w || !om || !psi || !elem || !cp)) return PDFX_ERR_ARG;
  if (!emom || !vcce || !gbin) return PDFX_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PDFX_ERR_CUDA;
  if (dev != c.device) return PDFX_ERR_ARG;
  unsigned char* base = nullptr;
  const int rc = scratch_address(dev, &base);
  if (rc) return rc;
  int32_t* words = reinterpret_cast<int32_t*>(base);
  int32_t* idx = words;
  uint32_t* pid = reinterpret_cast<uint32_t*>(words + kNaP);
  int32_t* per_e = words + 2 * kNaP;
  Plan pl;
  pl.cnt = per_e;
  pl.off = per_e + kNaE;
  pl.foff = per_e + 2 * kNaE;
  pl.cursor = per_e + 3 * kNaE;
  pl.big_list = per_e + 4 * kNaE;
  pl.tiles = per_e + 5 * kNaE;
  pl.tiles_mid = per_e + 6 * kNaE;
  pl.scal = per_e + 7 * kNaE;
  pl.idx = idx;
  pl.tile_split = c.tile_split;
  // without particle moves the plan touches only the arrays above; the rest alias the final
  // offsets so that no pointer leaves the scratch
  pl.fin = pl.gain = pl.goff = pl.loss = pl.doff = pl.recips = pl.donors = pl.foff;
  pl.movers = pl.mrecip = pl.foff;
  pl.hist = nullptr;
  pl.mvals = nullptr;

  // counts start at zero on every call: the scratch keeps the previous call's contents
  if (cudaMemsetAsync(pl.cnt, 0, sizeof(int32_t) * c.ne, s) != cudaSuccess) return PDFX_ERR_CUDA;
  if (np > 0) {
    iota_kernel<<<static_cast<unsigned>((np + 255) / 256), 256, 0, s>>>(pid, np);
    launch_count(elem, np, c.ne, pl.cnt, c.diag, c.err, s);
  }
  const int plan_launches = launch_plan(pl, c.ne, 1, 0, 0, s);
  launch_scatter(elem, np, c.ne, pl, s);
  StatsArgs<double> a{};
  a.p.u = const_cast<double*>(u);
  a.p.v = const_cast<double*>(v);
  a.p.w = const_cast<double*>(w);
  a.p.om = const_cast<double*>(om);
  a.p.psi = const_cast<double*>(psi);
  a.p.pid = pid;
  a.p.elem = const_cast<int32_t*>(elem);
  a.p.cp = cp;
  a.resort = 0;
  a.cnt = pl.cnt;
  a.off = pl.off;
  a.idx = pl.idx;
  a.fin = pl.cnt;
  a.foff = pl.foff;
  a.gain = pl.gain;
  a.goff = pl.goff;
  a.movers = pl.movers;
  a.big_list = pl.big_list;
  a.tiles = pl.tiles;
  a.tiles_mid = pl.tiles_mid;
  a.einst = nullptr;   // the whole grid as one instance
  a.ielem = nullptr;
  a.K = 1;
  a.scal = pl.scal;
  a.ne = c.ne;
  a.np = np;
  a.bins[0] = c.prm.bins[0];
  a.bins[1] = c.prm.bins[1];
  a.bins[2] = c.prm.bins[2];
  a.min_per_bin = c.prm.min_per_bin;
  a.G = c.G;
  a.acc64 = 0;                      // FP64 throughout
  a.prior = 0;                      // the caller's emom holds no previous statistics
  a.cond_mode = c.prm.cond_mode;    // the context's conditioning: bins or Fox's projection
  a.fox_bins = c.prm.fox_bins;
  a.emom = emom;
  a.vcce = vcce;
  a.gbin = gbin;
  a.diag = c.diag;
  a.err = c.err;
  launch_stats<double>(a, c.num_sms, s, &c.side);
  if (nmom) launch_node_average(emom, c.ne_off, c.ne_list, c.nn, nmom, s);
  // iota, count and scatter (with particles), plan, three tile classes, the large-element
  // kernel and (hierarchical bins) the bucket-rank tile over the large-element list, node
  // average
  c.launches += (np > 0 ? 3 : 0) + plan_launches + (a.cond_mode == 1 ? 4 : 5) + (nmom ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? PDFX_OK : PDFX_ERR_CUDA;
}

}  // namespace pdfx

extern "C" int pdfx_element_stats_noalloc(void* ctx, int64_t np, const double* u, const double* v,
                                          const double* w, const double* om, const double* psi,
                                          const int32_t* elem, double* emom, double* vcce,
                                          int32_t* gbin, uint8_t* cp, double* nmom, void* stream) {
  if (!ctx) return PDFX_ERR_ARG;
  return pdfx::element_stats_noalloc(*static_cast<pdfx::Ctx*>(ctx), np, u, v, w, om, psi, elem,
                                     emom, vcce, gbin, cp, nmom, static_cast<cudaStream_t>(stream));
}
