// C ABI of pdfx: context, grid preprocessing, buffers and the timestep orchestration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fem_host.h"
#include "pdfx_internal.h"

namespace pdfx {

namespace {

int cerr(cudaError_t e) { return e == cudaSuccess ? PDFX_OK : PDFX_ERR_CUDA; }
#define PDFX_CUDA(call)                          \
  do {                                           \
    const cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) return PDFX_ERR_CUDA; \
  } while (0)
#define PDFX_TRY(call)             \
  do {                             \
    const int r_ = (call);         \
    if (r_ != PDFX_OK) return r_;  \
  } while (0)

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void* dev_alloc(Ctx& c, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c.has_alloc) {
    p = c.alloc.alloc(bytes, c.alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) c.owned.push_back({p, bytes});
  return p;
}

void dev_free(Ctx& c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c.owned.size(); ++i) {
    if (c.owned[i].first == p) {
      if (c.has_alloc) c.alloc.release(p, c.owned[i].second, c.alloc.user);
      else cudaFree(p);
      c.owned.erase(c.owned.begin() + static_cast<long>(i));
      return;
    }
  }
}

template <typename P>
int alloc_into(Ctx& c, P*& out, size_t count) {
  dev_free(c, out);
  out = static_cast<P*>(dev_alloc(c, sizeof(P) * (count ? count : 1)));
  return out ? PDFX_OK : PDFX_ERR_ALLOC;
}

bool params_valid(const pdfx_params& p) {
  if (!(p.C4 > 0.0 && p.C4 <= 1.0)) return false;        // Marsaglia-Tsang needs shape >= 1
  for (int l = 0; l < 3; ++l)
    if (p.bins[l] < 1 || p.bins[l] > 16) return false;
  if (p.bins[0] * p.bins[1] * p.bins[2] > 256) return false;  // conditioning pointer is 8-bit
  if (p.min_per_bin < 1 || p.minnpel < 0 || p.minnpel > PDFX_MAX_PER_ELEMENT) return false;
  if (p.precision != 0 && p.precision != 1) return false;
  if (p.sort_every < 0 || !(p.nu >= 0.0) || !(p.period_x >= 0.0)) return false;
  if (p.acc64 != 0 && p.acc64 != 1) return false;
  if (p.cond_mode != 0 && p.cond_mode != 1) return false;
  if (p.cond_mode == 1 && (p.fox_bins < 1 || p.fox_bins > 256)) return false;
  if (p.model != 0 && p.model != 1) return false;
  if (!std::isfinite(p.alpha)) return false;
  if (!(p.cfl > 0.0) || !std::isfinite(p.cfl)) return false;
  return true;
}

template <typename T>
Model<T> model_of(const pdfx_params& p) {
  Model<T> m;
  m.C1 = T(p.C1); m.C2 = T(p.C2); m.C3 = T(p.C3); m.C4 = T(p.C4); m.CT = T(p.CT);
  m.Cw1 = T(p.Cw1); m.Cw2 = T(p.Cw2); m.nu = T(p.nu); m.C0 = T(p.C0); m.Cs = T(p.Cs);
  m.Ct = T(p.Ct); m.Cphi = T(p.Cphi); m.src_x = T(p.src_x); m.src_y = T(p.src_y);
  m.src_r = T(p.src_r); m.period_x = T(p.period_x);
  // FP32 form: the source centre as hi + lo pairs (the particle positions are pairs)
  m.src_xl = T(p.src_x - static_cast<double>(m.src_x));
  m.src_yl = T(p.src_y - static_cast<double>(m.src_y));
  m.nuCT2 = T(p.nu * p.CT * p.CT);
  m.s2nu = T(std::sqrt(2.0 * p.nu));
  m.cs_r2 = T(p.Cs * std::cbrt(p.src_r * p.src_r));
  m.c0_mode = p.c0_mode; m.tm_mode = p.tm_mode; m.interp_mode = p.interp_mode;
  m.source_on = p.source_on;
  m.model = p.model;
  m.alpha = T(p.alpha);
  return m;
}

inline uint32_t key0(const pdfx_params& p) { return static_cast<uint32_t>(p.seed & 0xffffffffu); }
inline uint32_t key1(const pdfx_params& p) {
  return static_cast<uint32_t>(p.seed >> 32) ^ p.instance;
}

// Parameters of instance k (the context's own for a single grid).
const pdfx_params& inst_params(const Ctx& c, int k) { return c.K > 1 ? c.iprm[k] : c.prm; }

// Instance k of element e (host).
int inst_of_element(const Ctx& c, int32_t e) {
  if (c.K <= 1) return 0;
  return static_cast<int>(std::upper_bound(c.h_ielem.begin(), c.h_ielem.end(), e) - c.h_ielem.begin()) - 1;
}

// Device table of the instances (model, Philox key, element and particle ranges).
template <typename T>
int upload_inst(Ctx& c) {
  const int K = c.K;
  std::vector<InstDev<T>> h(static_cast<size_t>(K));
  for (int k = 0; k < K; ++k) {
    const pdfx_params& p = inst_params(c, k);
    h[k].m = model_of<T>(p);
    h[k].k0 = key0(p);
    h[k].k1 = key1(p);
    h[k].e0 = c.h_ielem[k];
    h[k].e1 = c.h_ielem[k + 1];
    h[k].p0 = c.h_ip0[k];
    h[k].np = c.h_ip0[k + 1] - c.h_ip0[k];
    h[k].ppe = c.h_ippe.empty() ? 0 : c.h_ippe[k];
    h[k].minnpel = p.minnpel;
  }
  if (c.inst_cap < K || !c.inst) {
    dev_free(c, c.inst);
    c.inst = dev_alloc(c, sizeof(InstDev<double>) * static_cast<size_t>(K));
    if (!c.inst) return PDFX_ERR_ALLOC;
    c.inst_cap = K;
  }
  PDFX_CUDA(cudaMemcpy(c.inst, h.data(), sizeof(InstDev<T>) * K, cudaMemcpyHostToDevice));
  if (K > 1) PDFX_CUDA(cudaMemcpy(c.ip0, c.h_ip0.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice));
  return PDFX_OK;
}

int upload_inst_any(Ctx& c) {
  return c.prm.precision == 1 ? upload_inst<float>(c) : upload_inst<double>(c);
}

double min_image_h(double d, double L) {
  if (L > 0.0) {
    if (d > 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
  }
  return d;
}

struct HostGeo {
  std::vector<double> vx, vy;   // [ne][3] vertices, unwrapped toward vertex A
  std::vector<double> nx;       // [ne][3] node x as given (canonical image)
  std::vector<double> ax, area2;
};

// Boundary line of edge k (opposite vertex k) of element f, normal toward vertex k.
void edge_line_h(const HostGeo& g, int f, int k, double out[4]) {
  const double* vx = g.vx.data() + 3 * f;
  const double* vy = g.vy.data() + 3 * f;
  const int a = (k + 1) % 3, b = (k + 2) % 3;
  const double tx = vx[b] - vx[a], ty = vy[b] - vy[a];
  const double len = std::sqrt(tx * tx + ty * ty);
  double mx = -ty / len, my = tx / len;
  if ((vx[k] - vx[a]) * mx + (vy[k] - vy[a]) * my < 0.0) { mx = -mx; my = -my; }
  out[0] = vx[a]; out[1] = vy[a]; out[2] = mx; out[3] = my;
}

template <typename T>
Particles<T> carve(void* base, int64_t np) {
  Particles<T> p;
  auto* b = static_cast<unsigned char*>(base);
  const size_t n = static_cast<size_t>(np > 0 ? np : 1);
  auto step = [&](size_t bytes) { unsigned char* r = b; b += (bytes + 255) & ~size_t(255); return r; };
  p.x = reinterpret_cast<T*>(step(sizeof(T) * n));
  p.y = reinterpret_cast<T*>(step(sizeof(T) * n));
  p.u = reinterpret_cast<T*>(step(sizeof(T) * n));
  p.v = reinterpret_cast<T*>(step(sizeof(T) * n));
  p.w = reinterpret_cast<T*>(step(sizeof(T) * n));
  p.om = reinterpret_cast<T*>(step(sizeof(T) * n));
  p.psi = reinterpret_cast<T*>(step(sizeof(T) * n));
  p.pid = reinterpret_cast<uint32_t*>(step(4 * n));
  p.elem = reinterpret_cast<int32_t*>(step(4 * n));
  p.cp = reinterpret_cast<uint8_t*>(step(n));
  if (sizeof(T) == 4) {   // the positions' trailing parts
    p.xl = reinterpret_cast<T*>(step(sizeof(T) * n));
    p.yl = reinterpret_cast<T*>(step(sizeof(T) * n));
  }
  return p;
}

template <typename T>
size_t particle_bytes(int64_t np) {
  const size_t n = static_cast<size_t>(np > 0 ? np : 1);
  auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
  return (sizeof(T) == 4 ? 9 : 7) * r(sizeof(T) * n) + r(4 * n) + r(4 * n) + r(n);
}

// ---- profiling ----------------------------------------------------------------------------
cudaEvent_t take_event(Ctx& c) {
  if (!c.ev_pool.empty()) {
    cudaEvent_t e = c.ev_pool.back();
    c.ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct StageTimer {
  Ctx& c;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(Ctx& cc, int st, cudaStream_t ss) : c(cc), stage(st), s(ss) {
    if (c.profiling) {
      a = take_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~StageTimer() {
    if (c.profiling && a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, s);
      c.ev_pending.push_back({stage, {a, b}});
    }
  }
};

void collect_times(Ctx& c) {
  for (auto& pe : c.ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      c.stage_ms[pe.first] += ms;
      c.stage_n[pe.first] += 1;
    }
    c.ev_pool.push_back(pe.second.first);
    c.ev_pool.push_back(pe.second.second);
  }
  c.ev_pending.clear();
}

// ---- pipeline -------------------------------------------------------------------------------
template <typename T>
int ensure_particles(Ctx& c, int64_t np) {
  const size_t bytes = particle_bytes<T>(np);
  if (c.pbuf[0] && c.pbuf_bytes >= bytes && c.np == np) return PDFX_OK;
  for (int b = 0; b < 2; ++b) {
    dev_free(c, c.pbuf[b]);
    c.pbuf[b] = dev_alloc(c, bytes);
    if (!c.pbuf[b]) return PDFX_ERR_ALLOC;
  }
  c.pbuf_bytes = bytes;
  c.np = np;
  c.cur = 0;
  const size_t n = static_cast<size_t>(np > 0 ? np : 1);
  PDFX_TRY(alloc_into(c, c.plan.idx, n));
  PDFX_TRY(alloc_into(c, c.plan.movers, n));
  PDFX_TRY(alloc_into(c, c.plan.mrecip, n));
  PDFX_TRY(alloc_into(c, c.plan.mvals, 7 * n));
  return PDFX_OK;
}

// Statistics and conditional means of the current state (after advance or a new state).
template <typename T>
int run_statistics(Ctx& c, bool counts_ready, bool allow_moves, bool force_resort, cudaStream_t s) {
  Particles<T> p = carve<T>(c.pbuf[c.cur], c.np);
  if (!counts_ready) {
    PDFX_CUDA(cudaMemsetAsync(c.plan.cnt, 0, sizeof(int32_t) * c.ne, s));
    launch_count(p.elem, c.np, c.ne, c.plan.cnt, c.diag, c.err, s);
    c.launches++;
  }
  {
    StageTimer t(c, 1, s);
    c.plan.tile_split = c.tile_split;
    c.launches += launch_plan(c.plan, c.ne, c.K, c.prm.minnpel, allow_moves ? 1 : 0, s);
  }
  {
    StageTimer t(c, 2, s);
    launch_scatter(p.elem, c.np, c.ne, c.plan, s);
    c.launches++;
  }
  bool any_minnpel = false;
  for (int k = 0; k < c.K; ++k) any_minnpel |= inst_params(c, k).minnpel > 0;
  if (allow_moves && any_minnpel) {
    StageTimer t(c, 3, s);
    launch_redistribute<T>(p, c.plan, c.K, static_cast<const InstDev<T>*>(c.inst), c.ne, c.np,
                           static_cast<const ElemGeo<T>*>(c.geo), c.topo, c.dstep, c.num_sms,
                           c.diag, c.err, s);
    c.launches += 3;
  }
  const bool resort = force_resort || (c.prm.sort_every > 0 && c.steps_since_sort + 1 >= c.prm.sort_every);
  {
    StageTimer t(c, 4, s);
    StatsArgs<T> a{};
    a.p = p;
    a.out = carve<T>(c.pbuf[1 - c.cur], c.np);
    a.resort = resort ? 1 : 0;
    a.cnt = c.plan.cnt;
    a.off = c.plan.off;
    a.idx = c.plan.idx;
    a.fin = c.plan.fin;
    a.foff = c.plan.foff;
    a.gain = c.plan.gain;
    a.goff = c.plan.goff;
    a.movers = c.plan.movers;
    a.big_list = c.plan.big_list;
    a.tiles = c.plan.tiles;
    a.tiles_mid = c.plan.tiles_mid;
    a.einst = c.K > 1 ? c.einst : nullptr;
    a.ielem = c.K > 1 ? c.ielem : nullptr;
    a.K = c.K;
    a.scal = c.plan.scal;
    a.ne = c.ne;
    a.np = c.np;
    a.bins[0] = c.prm.bins[0]; a.bins[1] = c.prm.bins[1]; a.bins[2] = c.prm.bins[2];
    a.min_per_bin = c.prm.min_per_bin;
    a.G = c.G;
    a.emom = c.emom;
    a.vcce = c.vcce;
    a.gbin = c.gbin;
    a.step_inc = allow_moves ? c.dstep : nullptr;   // only a step advances the counter
    a.acc64 = c.prm.acc64;
    a.prior = 1;
    a.cond_mode = c.prm.cond_mode;
    a.fox_bins = c.prm.fox_bins;
    a.diag = c.diag;
    a.err = c.err;
    launch_stats<T>(a, c.num_sms, s, &c.side);
    // three tile classes, the large-element kernel and (hierarchical bins) the bucket-rank
    // tile over the large-element list
    c.launches += a.cond_mode == 1 ? 4 : 5;
  }
  if (resort) {
    c.cur = 1 - c.cur;
    c.steps_since_sort = 0;
  } else {
    c.steps_since_sort++;
  }
  {
    StageTimer t(c, 5, s);
    launch_node_average(c.emom, c.ne_off, c.ne_list, c.nn, c.nmom, s);
    c.launches++;
  }
  return cerr(cudaGetLastError());
}

template <typename T>
int do_step(Ctx& c, double dt, cudaStream_t s) {
  c.last_dt = dt;
  Particles<T> p = carve<T>(c.pbuf[c.cur], c.np);
  PDFX_CUDA(cudaMemsetAsync(c.plan.cnt, 0, sizeof(int32_t) * c.ne, s));
  {
    StageTimer t(c, 0, s);
    AdvanceArgs<T> a{};
    a.p = p;
    a.np = c.np;
    a.geo = static_cast<const ElemGeo<T>*>(c.geo);
    a.topo = c.topo;
    a.walls = static_cast<const Line<T>*>(c.walls);
    a.wall2 = c.wall2;
    a.fslines = static_cast<const Line<T>*>(c.fslines);
    a.fsedges = static_cast<const Line<T>*>(c.fsedges);
    a.ne_off = c.ne_off;
    a.ne_list = c.ne_list;
    a.ne = c.ne;
    a.fields = static_cast<const T*>(c.fields);
    a.vcce = c.vcce;
    a.G = c.G;
    a.nmom = c.nmom;
    a.cnt = c.plan.cnt;
    a.diag = c.diag;
    a.err = c.err;
    a.brute_list = c.brute_list;
    a.brute_count = c.err + 1;
    a.brute_cap = kBruteCap;
    a.lost_rec = c.lost_rec;
    a.m = model_of<T>(c.prm);
    a.dt = T(dt);
    a.sdt = T(std::sqrt(dt));
    a.stepc = c.dstep;
    a.corr = c.corr_pending ? c.corr : nullptr;   // consumed by this advance
    a.k0 = key0(c.prm);
    a.k1 = key1(c.prm);
    a.inst = c.K > 1 ? static_cast<const InstDev<T>*>(c.inst) : nullptr;
    a.einst = c.K > 1 ? c.einst : nullptr;
    launch_advance<T>(a, c.num_sms, c.adv_block, s);
    c.launches += 2;   // the advance and the brute-force search
    c.corr_pending = false;
  }
  PDFX_TRY(run_statistics<T>(c, true, true, false, s));
  c.step++;
  c.steps_done++;
  return cerr(cudaGetLastError());
}

// Applies a pending Eq. 31 correction to the particles now (before a caller reads them, or
// before steps are captured into a graph).
template <typename T>
void apply_pending_correction(Ctx& c, cudaStream_t s) {
  if (!c.corr_pending) return;
  launch_apply_correction<T>(carve<T>(c.pbuf[c.cur], c.np), c.np, c.corr, s);
  c.launches++;
  c.corr_pending = false;
}
void apply_pending_correction_any(Ctx& c, cudaStream_t s) {
  if (c.prm.precision == 1) apply_pending_correction<float>(c, s);
  else apply_pending_correction<double>(c, s);
}

template <typename T>
int do_init(Ctx& c, const int32_t* ppe, cudaStream_t s) {
  c.h_ippe.assign(ppe, ppe + c.K);
  c.h_ip0.assign(static_cast<size_t>(c.K) + 1, 0);
  for (int k = 0; k < c.K; ++k)
    c.h_ip0[k + 1] = c.h_ip0[k] + static_cast<int64_t>(ppe[k]) * (c.h_ielem[k + 1] - c.h_ielem[k]);
  const int64_t np = c.h_ip0[c.K];
  PDFX_TRY(ensure_particles<T>(c, np));
  PDFX_TRY(upload_inst<T>(c));
  Particles<T> p = carve<T>(c.pbuf[c.cur], np);
  if (c.K > 1)
    launch_init_batch<T>(p, np, c.K, static_cast<const InstDev<T>*>(c.inst), c.ip0,
                         static_cast<const ElemGeo<T>*>(c.geo), c.topo,
                         static_cast<const T*>(c.fields), c.diag, s);
  else
    launch_init<T>(p, c.ne, ppe[0], static_cast<const ElemGeo<T>*>(c.geo), c.topo,
                   static_cast<const T*>(c.fields), model_of<T>(c.prm), key0(c.prm), key1(c.prm),
                   c.diag, s);
  c.launches++;
  c.step = 0;
  PDFX_CUDA(cudaMemsetAsync(c.dstep, 0, sizeof(uint32_t), s));
  c.steps_since_sort = 0;
  c.corr_pending = false;
  return run_statistics<T>(c, false, false, false, s);
}

template <typename T>
int do_set_particles(Ctx& c, int64_t np, const pdfx_soa* soa, uint32_t step, int on_device,
                     cudaStream_t s) {
  PDFX_TRY(ensure_particles<T>(c, np));
  PDFX_TRY(upload_inst<T>(c));
  Particles<T> p = carve<T>(c.pbuf[c.cur], np);
  const size_t n = static_cast<size_t>(np);
  double* tmp = nullptr;
  int32_t* tel = nullptr;
  const double* src[7] = {soa->x, soa->y, soa->u, soa->v, soa->w, soa->om, soa->psi};
  const int32_t* el = soa->elem;
  if (!on_device && np > 0) {
    tmp = static_cast<double*>(dev_alloc(c, sizeof(double) * 7 * n));
    tel = static_cast<int32_t*>(dev_alloc(c, sizeof(int32_t) * n));
    if (!tmp || !tel) { dev_free(c, tmp); dev_free(c, tel); return PDFX_ERR_ALLOC; }
    for (int k = 0; k < 7; ++k) {
      PDFX_CUDA(cudaMemcpyAsync(tmp + k * n, src[k], sizeof(double) * n, cudaMemcpyHostToDevice, s));
      src[k] = tmp + k * n;
    }
    PDFX_CUDA(cudaMemcpyAsync(tel, el, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    el = tel;
  }
  launch_load_state<T>(p, np, c.K > 1 ? c.einst : nullptr, c.K > 1 ? c.ip0 : nullptr, src[0],
                       src[1], src[2], src[3], src[4], src[5], src[6], el, c.ne, c.diag, c.err, s);
  c.launches++;
  c.step = step;
  PDFX_CUDA(cudaMemcpyAsync(c.dstep, &step, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  c.steps_since_sort = 0;
  c.corr_pending = false;
  int rc = run_statistics<T>(c, false, false, true, s);
  if (tmp) {
    cudaStreamSynchronize(s);
    dev_free(c, tmp);
    dev_free(c, tel);
  }
  if (rc == PDFX_OK && on_device) {
    // device element ids are range-checked by the load kernel: report a bad one now
    int err = 0;
    PDFX_CUDA(cudaMemcpyAsync(&err, c.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PDFX_CUDA(cudaStreamSynchronize(s));
    if (err == PDFX_ERR_ELEMENT) rc = err;
  }
  return rc;
}

template <typename T>
int do_get_particles(Ctx& c, pdfx_soa* soa, int on_device, cudaStream_t s) {
  apply_pending_correction<T>(c, s);
  Particles<T> p = carve<T>(c.pbuf[c.cur], c.np);
  const size_t n = static_cast<size_t>(c.np);
  if (on_device) {
    launch_gather_by_pid<T>(p, c.np, c.K > 1 ? c.einst : nullptr, c.K > 1 ? c.ip0 : nullptr,
                            soa->x, soa->y, soa->u, soa->v, soa->w, soa->om, soa->psi, soa->elem,
                            soa->cp, s);
    c.launches++;
    return cerr(cudaGetLastError());
  }
  if (n == 0) return PDFX_OK;
  double* tmp = static_cast<double*>(dev_alloc(c, sizeof(double) * 7 * n + 5 * n));
  if (!tmp) return PDFX_ERR_ALLOC;
  int32_t* tel = reinterpret_cast<int32_t*>(tmp + 7 * n);
  uint8_t* tcp = reinterpret_cast<uint8_t*>(tel + n);
  launch_gather_by_pid<T>(p, c.np, c.K > 1 ? c.einst : nullptr, c.K > 1 ? c.ip0 : nullptr, tmp,
                          tmp + n, tmp + 2 * n, tmp + 3 * n, tmp + 4 * n, tmp + 5 * n, tmp + 6 * n,
                          tel, tcp, s);
  c.launches++;
  double* dst[7] = {soa->x, soa->y, soa->u, soa->v, soa->w, soa->om, soa->psi};
  int rc = PDFX_OK;
  for (int k = 0; k < 7 && rc == PDFX_OK; ++k)
    if (dst[k]) rc = cerr(cudaMemcpyAsync(dst[k], tmp + k * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (rc == PDFX_OK && soa->elem)
    rc = cerr(cudaMemcpyAsync(soa->elem, tel, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  if (rc == PDFX_OK && soa->cp) rc = cerr(cudaMemcpyAsync(soa->cp, tcp, n, cudaMemcpyDeviceToHost, s));
  if (rc == PDFX_OK) rc = cerr(cudaStreamSynchronize(s));
  dev_free(c, tmp);
  return rc;
}

// Element geometry in the working precision: node coordinates (canonical x) and 1 / (2 A_e);
// the FP32 form stores each coordinate as an FP32 pair.
void geo_of(const HostGeo& g, int32_t e, ElemGeo<double>& o) {
  for (int k = 0; k < 3; ++k) {
    o.x[k] = g.nx[3 * e + k];
    o.y[k] = g.vy[3 * e + k];
  }
  o.inv2a = 1.0 / g.area2[e];
  o.pad = 0.0;
}
void geo_of(const HostGeo& g, int32_t e, const int32_t* tri, double L, ElemGeo<float>& o) {
  for (int k = 0; k < 3; ++k) {
    pair_of(g.nx[3 * e + k], o.xh[k], o.xl[k]);
    pair_of(g.vy[3 * e + k], o.yh[k], o.yl[k]);
  }
  // edge opposite vertex k: counter-clockwise from a = k + 1 to b = k + 2; pivot at the
  // lower node id, vector from the pivot to the other node (minimum image in x)
  o.code = 0u;
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    const bool flip = tri[3 * e + b] < tri[3 * e + a];
    const int p = flip ? b : a, q = flip ? a : b;
    o.ex[k] = static_cast<float>(min_image(g.nx[3 * e + q] - g.nx[3 * e + p], L));
    o.ey[k] = static_cast<float>(g.vy[3 * e + q] - g.vy[3 * e + p]);
    o.code |= (static_cast<uint32_t>(p) | (flip ? 4u : 0u)) << (3 * k);
  }
  o.inv2a = static_cast<float>(1.0 / g.area2[e]);
  o.pad[0] = o.pad[1] = 0.0f;
}
void geo_of(const HostGeo& g, int32_t e, const int32_t*, double, ElemGeo<double>& o) { geo_of(g, e, o); }
void line_of(const double* src, Line<double>& o) {
  o.px = src[0]; o.py = src[1]; o.nx = src[2]; o.ny = src[3];
}
void line_of(const double* src, Line<float>& o) {
  pair_of(src[0], o.px, o.pxl);
  pair_of(src[1], o.py, o.pyl);
  o.nx = static_cast<float>(src[2]);
  o.ny = static_cast<float>(src[3]);
  o.pad0 = o.pad1 = 0.0f;
}

template <typename T>
int upload_grid(Ctx& c, const HostGeo& g, const std::vector<ElemTopo>& topo,
                const std::vector<double>& walls, const std::vector<double>& fsl,
                const std::vector<double>& fse, const int32_t* tri, const std::vector<double>& period) {
  const int32_t ne = c.ne;
  std::vector<ElemGeo<T>> hg(static_cast<size_t>(ne));
  for (int32_t e = 0; e < ne; ++e) geo_of(g, e, tri, period[e], hg[e]);
  dev_free(c, c.geo);
  c.geo = dev_alloc(c, sizeof(ElemGeo<T>) * ne);
  if (!c.geo) return PDFX_ERR_ALLOC;
  PDFX_CUDA(cudaMemcpy(c.geo, hg.data(), sizeof(ElemGeo<T>) * ne, cudaMemcpyHostToDevice));
  PDFX_TRY(alloc_into(c, c.topo, static_cast<size_t>(ne)));
  PDFX_CUDA(cudaMemcpy(c.topo, topo.data(), sizeof(ElemTopo) * ne, cudaMemcpyHostToDevice));
  for (int which = 0; which < 3; ++which) {
    const std::vector<double>& src = which == 0 ? walls : (which == 1 ? fsl : fse);
    void*& dst = which == 0 ? c.walls : (which == 1 ? c.fslines : c.fsedges);
    const size_t nl = src.size() / 4;
    if (which == 0) c.n_wall_lines = static_cast<int>(nl);
    std::vector<Line<T>> hl(nl ? nl : 1);
    for (size_t i = 0; i < nl; ++i) line_of(&src[4 * i], hl[i]);
    dev_free(c, dst);
    dst = dev_alloc(c, sizeof(Line<T>) * hl.size());
    if (!dst) return PDFX_ERR_ALLOC;
    PDFX_CUDA(cudaMemcpy(dst, hl.data(), sizeof(Line<T>) * hl.size(), cudaMemcpyHostToDevice));
  }
  return PDFX_OK;
}

void drop_pcg_graphs(Ctx& c);

int set_grid(Ctx& c, int32_t nn, const double* xy, int32_t ne, const int32_t* tri, const int8_t* tag) {
  if (nn <= 0 || ne <= 0 || !xy || !tri || !tag) return PDFX_ERR_ARG;
  if (c.K > 1 && c.h_ielem.back() != ne) return PDFX_ERR_ARG;
  if (c.K <= 1) c.h_ielem = {0, ne};
  std::vector<int32_t> hinst(static_cast<size_t>(ne), 0);   // instance of each element
  for (int k = 0; k < c.K; ++k)
    for (int32_t e = c.h_ielem[k]; e < c.h_ielem[k + 1]; ++e) hinst[e] = k;
  auto period_of = [&](int32_t e) { return inst_params(c, hinst[e]).period_x; };
  HostGeo g;
  g.vx.resize(3 * static_cast<size_t>(ne));
  g.vy.resize(3 * static_cast<size_t>(ne));
  g.nx.resize(3 * static_cast<size_t>(ne));
  g.ax.resize(ne);
  g.area2.resize(ne);
  for (int32_t e = 0; e < ne; ++e) {
    const double L = period_of(e);
    const int A = tri[3 * e], B = tri[3 * e + 1], C = tri[3 * e + 2];
    if (A < 0 || B < 0 || C < 0 || A >= nn || B >= nn || C >= nn || A == B || B == C || A == C)
      return PDFX_ERR_MESH;
    const int n3[3] = {A, B, C};
    for (int k = 0; k < 3; ++k) {
      double x = xy[2 * n3[k]];
      if (L > 0.0 && k > 0) {   // the image nearest vertex A
        const double d = x - xy[2 * A];
        if (d > 0.5 * L) x -= L;
        else if (d < -0.5 * L) x += L;
      }
      g.vx[3 * e + k] = x;
      g.vy[3 * e + k] = xy[2 * n3[k] + 1];
      g.nx[3 * e + k] = xy[2 * n3[k]];
    }
    g.ax[e] = g.vx[3 * e];
    const double bx = min_image_h(xy[2 * B] - xy[2 * A], L), by = xy[2 * B + 1] - xy[2 * A + 1];
    const double cx = min_image_h(xy[2 * C] - xy[2 * A], L), cy = xy[2 * C + 1] - xy[2 * A + 1];
    g.area2[e] = bx * cy - by * cx;   // 2 A_e (Eq. 40 denominator)
    if (!(g.area2[e] > 0.0)) return PDFX_ERR_MESH;
  }
  // node -> elements, ascending element id
  std::vector<int32_t> off(static_cast<size_t>(nn) + 1, 0), lst(3 * static_cast<size_t>(ne));
  for (int32_t e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k) off[tri[3 * e + k] + 1]++;
  for (int32_t n = 0; n < nn; ++n) off[n + 1] += off[n];
  {
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int32_t e = 0; e < ne; ++e)
      for (int k = 0; k < 3; ++k) lst[fill[tri[3 * e + k]]++] = e;
  }
  // neighbours across edges: sort the (min node, max node) edge keys
  struct EdgeRec { int64_t key; int32_t e; int8_t k; };
  std::vector<EdgeRec> edges(3 * static_cast<size_t>(ne));
  for (int32_t e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k) {
      const int64_t a = tri[3 * e + (k + 1) % 3], b = tri[3 * e + (k + 2) % 3];
      edges[3 * e + k] = {std::min(a, b) * static_cast<int64_t>(nn) + std::max(a, b), e,
                          static_cast<int8_t>(k)};
    }
  std::sort(edges.begin(), edges.end(), [](const EdgeRec& x, const EdgeRec& y) {
    return x.key != y.key ? x.key < y.key : (x.e != y.e ? x.e < y.e : x.k < y.k);
  });
  std::vector<int32_t> nbr(3 * static_cast<size_t>(ne), -1);
  for (size_t i = 0; i < edges.size();) {
    size_t j = i + 1;
    while (j < edges.size() && edges[j].key == edges[i].key) ++j;
    if (j - i > 2) return PDFX_ERR_MESH;
    if (j - i == 2) {
      nbr[3 * edges[i].e + edges[i].k] = edges[i + 1].e;
      nbr[3 * edges[i + 1].e + edges[i + 1].k] = edges[i].e;
    }
    i = j;
  }
  for (int32_t e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k)
      if ((nbr[3 * e + k] < 0) != (tag[3 * e + k] != 0)) return PDFX_ERR_MESH;
  if (c.K > 1) {
    // the instances of a batch share no edge and no node
    for (int32_t e = 0; e < ne; ++e)
      for (int k = 0; k < 3; ++k)
        if (nbr[3 * e + k] >= 0 && hinst[nbr[3 * e + k]] != hinst[e]) return PDFX_ERR_MESH;
    std::vector<int32_t> owner(static_cast<size_t>(nn), -1);
    for (int32_t e = 0; e < ne; ++e)
      for (int k = 0; k < 3; ++k) {
        int32_t& o = owner[tri[3 * e + k]];
        if (o >= 0 && o != hinst[e]) return PDFX_ERR_MESH;
        o = hinst[e];
      }
  }
  // boundary lines (Sect. 3.8 reading, extended to corners): the element's own edges of the
  // type (local order), then edges of the type incident to one of its nodes (nodes in local
  // order, elements ascending, edges in local order) whose line, oriented into the fluid by
  // the edge's own element, has the element's centroid strictly in front; lines equal to
  // one already taken are skipped; at most two no-slip lines and one free-slip line
  std::vector<ElemTopo> topo(static_cast<size_t>(ne));
  std::vector<double> walls, fsl, fse;
  std::vector<int32_t> wall2(static_cast<size_t>(ne), -1);
  auto same_line = [](const double* p, const double* q) {
    if (p[2] * q[2] + p[3] * q[3] < 1.0 - 1e-9) return false;
    const double d = (q[0] - p[0]) * p[2] + (q[1] - p[1]) * p[3];
    return std::fabs(d) <= 1e-9 * (1.0 + std::fabs(p[0]) + std::fabs(p[1]));
  };
  for (int32_t e = 0; e < ne; ++e) {
    ElemTopo& t = topo[e];
    t.n0 = tri[3 * e]; t.n1 = tri[3 * e + 1]; t.n2 = tri[3 * e + 2];
    t.nb0 = nbr[3 * e]; t.nb1 = nbr[3 * e + 1]; t.nb2 = nbr[3 * e + 2];
    // a free-slip boundary edge reflects the walk (Sect. 4.2): -2 - (its line's index)
    for (int k = 0; k < 3; ++k) {
      if (nbr[3 * e + k] >= 0 || tag[3 * e + k] != 2) continue;
      double line[4];
      edge_line_h(g, e, k, line);
      const int j = static_cast<int>(fse.size() / 4);
      fse.insert(fse.end(), line, line + 4);
      (k == 0 ? t.nb0 : (k == 1 ? t.nb1 : t.nb2)) = -2 - j;
    }
    t.wall = -1;
    t.fslip = -1;
    const double gx = (g.vx[3 * e] + g.vx[3 * e + 1] + g.vx[3 * e + 2]) / 3.0;
    const double gy = (g.vy[3 * e] + g.vy[3 * e + 1] + g.vy[3 * e + 2]) / 3.0;
    for (int type = 1; type <= 2; ++type) {
      const int max_lines = type == 1 ? 2 : 1;
      double found[2][4];
      int nf = 0;
      auto take = [&](const double* line) {
        for (int j = 0; j < nf; ++j)
          if (same_line(found[j], line)) return;
        for (int q = 0; q < 4; ++q) found[nf][q] = line[q];
        ++nf;
      };
      for (int k = 0; k < 3 && nf < max_lines; ++k)
        if (tag[3 * e + k] == type) {
          double line[4];
          edge_line_h(g, e, k, line);
          take(line);
        }
      for (int kv = 0; kv < 3 && nf < max_lines; ++kv) {
        const int n = tri[3 * e + kv];
        for (int32_t i = off[n]; i < off[n + 1] && nf < max_lines; ++i) {
          const int f = lst[i];
          for (int k = 0; k < 3 && nf < max_lines; ++k) {
            if (tag[3 * f + k] != type) continue;
            if (tri[3 * f + (k + 1) % 3] != n && tri[3 * f + (k + 2) % 3] != n) continue;
            double line[4];
            edge_line_h(g, f, k, line);
            line[0] = g.ax[e] + min_image_h(line[0] - g.ax[e], period_of(e));
            if ((gx - line[0]) * line[2] + (gy - line[1]) * line[3] <= 0.0) continue;
            take(line);
          }
        }
      }
      std::vector<double>& dst = type == 1 ? walls : fsl;
      for (int j = 0; j < nf; ++j) {
        const int idx = static_cast<int>(dst.size() / 4);
        if (type == 2) t.fslip = idx;
        else if (j == 0) t.wall = idx;
        else wall2[e] = idx;
        dst.insert(dst.end(), found[j], found[j] + 4);
      }
    }
  }
  c.nn = nn;
  c.ne = ne;
  std::vector<double> eperiod(static_cast<size_t>(ne));
  for (int32_t e = 0; e < ne; ++e) eperiod[e] = period_of(e);
  int rc = c.prm.precision == 1 ? upload_grid<float>(c, g, topo, walls, fsl, fse, tri, eperiod)
                                : upload_grid<double>(c, g, topo, walls, fsl, fse, tri, eperiod);
  if (rc) return rc;
  PDFX_TRY(alloc_into(c, c.wall2, wall2.size()));
  PDFX_TRY(alloc_into(c, c.dnorm, static_cast<size_t>(1)));
  {
    // Eq. 26's numerator: min over nodes of sqrt(A_n), A_n the mean area of its elements
    double m = 0.0;
    bool any = false;
    for (int32_t n = 0; n < nn; ++n) {
      const int32_t k = off[n + 1] - off[n];
      if (k <= 0) continue;
      double a = 0.0;
      for (int32_t i = off[n]; i < off[n + 1]; ++i) a += 0.5 * std::fabs(g.area2[lst[i]]);
      const double r = std::sqrt(a / k);
      if (!any || r < m) m = r;
      any = true;
    }
    c.min_sqrt_an = m;
  }
  PDFX_CUDA(cudaMemcpy(c.wall2, wall2.data(), sizeof(int32_t) * wall2.size(), cudaMemcpyHostToDevice));
  PDFX_TRY(alloc_into(c, c.ne_off, off.size()));
  PDFX_TRY(alloc_into(c, c.ne_list, lst.size()));
  PDFX_CUDA(cudaMemcpy(c.ne_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice));
  PDFX_CUDA(cudaMemcpy(c.ne_list, lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice));
  c.h_ne_off = off;
  c.h_ne_list = lst;
  // per-element and per-node buffers
  const size_t E = static_cast<size_t>(ne), N = static_cast<size_t>(nn);
  Plan& pl = c.plan;
  for (int32_t** b : {&pl.cnt, &pl.cursor, &pl.fin, &pl.gain, &pl.loss, &pl.recips, &pl.donors,
                      &pl.big_list, &pl.tiles, &pl.tiles_mid})
    PDFX_TRY(alloc_into(c, *b, E));
  for (int32_t** b : {&pl.off, &pl.foff, &pl.goff, &pl.doff}) PDFX_TRY(alloc_into(c, *b, E + 1));
  const int K = c.K;
  PDFX_TRY(alloc_into(c, pl.scal, 16 * static_cast<size_t>(K)));
  PDFX_TRY(alloc_into(c, pl.hist, static_cast<size_t>(K) * 2 * (kHistCap + 1)));
  if (K > 1) {
    PDFX_TRY(alloc_into(c, c.einst, E));
    PDFX_TRY(alloc_into(c, c.ielem, static_cast<size_t>(K) + 1));
    PDFX_TRY(alloc_into(c, c.ip0, static_cast<size_t>(K) + 1));
    PDFX_TRY(alloc_into(c, c.iminnpel, static_cast<size_t>(K)));
    std::vector<int32_t> mn(static_cast<size_t>(K));
    for (int k = 0; k < K; ++k) mn[k] = c.iprm[k].minnpel;
    PDFX_CUDA(cudaMemcpy(c.einst, hinst.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice));
    PDFX_CUDA(cudaMemcpy(c.ielem, c.h_ielem.data(), sizeof(int32_t) * (K + 1), cudaMemcpyHostToDevice));
    PDFX_CUDA(cudaMemcpy(c.iminnpel, mn.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice));
    pl.ielem = c.ielem;
    pl.ip0 = c.ip0;
    pl.iminnpel = c.iminnpel;
  } else {
    pl.ielem = nullptr;
    pl.ip0 = nullptr;
    pl.iminnpel = nullptr;
  }
  PDFX_TRY(alloc_into(c, c.emom, E * kNS));
  PDFX_TRY(alloc_into(c, c.nmom, N * kNS));
  PDFX_TRY(alloc_into(c, c.vcce, E * c.G));
  PDFX_TRY(alloc_into(c, c.gbin, E * 3));
  PDFX_CUDA(cudaMemset(pl.scal, 0, sizeof(int32_t) * 16 * K));
  PDFX_CUDA(cudaMemset(c.vcce, 0, sizeof(double) * E * c.G));
  PDFX_CUDA(cudaMemset(c.emom, 0, sizeof(double) * E * kNS));
  PDFX_CUDA(cudaMemset(c.nmom, 0, sizeof(double) * N * kNS));
  dev_free(c, c.fields);
  dev_free(c, c.fields64);
  c.fields = dev_alloc(c, (c.prm.precision == 1 ? sizeof(float) : sizeof(double)) * N * kNF);
  c.fields64 = c.prm.precision == 1 ? static_cast<double*>(dev_alloc(c, sizeof(double) * N * kNF)) : nullptr;
  if (!c.fields || (c.prm.precision == 1 && !c.fields64)) return PDFX_ERR_ALLOC;
  for (int b = 0; b < 2; ++b) { dev_free(c, c.pbuf[b]); c.pbuf[b] = nullptr; }
  c.np = 0;
  c.h_tri.assign(tri, tri + 3 * E);
  c.h_tag.assign(tag, tag + 3 * E);
  c.h_vx = g.vx;
  c.h_vy = g.vy;
  c.h_area2 = g.area2;
  c.fem_ready = false;   // the Eulerian calls rebuild their FEM data for this grid
  drop_pcg_graphs(c);
  c.corr_pending = false;
  c.have_grid = true;
  c.have_fields = false;
  return PDFX_OK;
}

// A captured cycle of steps bakes in dt, the grid, the particle storage and the model
// parameters: any change of those drops it.
void drop_graph(Ctx& c) {
  if (c.gexec) cudaGraphExecDestroy(c.gexec);
  c.gexec = nullptr;
  c.g_steps = 0;
}

template <typename T>
int capture_cycle(Ctx& c, double dt, int nsteps) {
  drop_graph(c);
  if (!c.gstream && cudaStreamCreateWithFlags(&c.gstream, cudaStreamNonBlocking) != cudaSuccess)
    return PDFX_ERR_CUDA;
  // host bookkeeping is replayed after capture: keep the state of the cycle's start
  const uint32_t step0 = c.step;
  const int64_t done0 = c.steps_done, launches0 = c.launches;
  const int cur0 = c.cur, since0 = c.steps_since_sort;
  const bool prof = c.profiling;
  c.profiling = false;
  PDFX_CUDA(cudaStreamBeginCapture(c.gstream, cudaStreamCaptureModeThreadLocal));
  int rc = PDFX_OK;
  for (int k = 0; k < nsteps && rc == PDFX_OK; ++k) rc = do_step<T>(c, dt, c.gstream);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c.gstream, &g);
  c.profiling = prof;
  const int64_t launches1 = c.launches;
  c.step = step0;
  c.steps_done = done0;
  c.launches = launches0;
  if (rc != PDFX_OK || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    c.cur = cur0;
    c.steps_since_sort = since0;
    return rc != PDFX_OK ? rc : PDFX_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&c.gexec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) { c.gexec = nullptr; return PDFX_ERR_CUDA; }
  if (c.cur != cur0 || c.steps_since_sort != since0) { drop_graph(c); return PDFX_ERR_ORDER; }
  c.g_dt = dt;
  c.g_steps = nsteps;
  c.g_buf = c.pbuf[0];
  c.g_np = c.np;
  c.g_launches = launches1 - launches0;
  return PDFX_OK;
}

template <typename T>
int do_step_many(Ctx& c, double dt, int32_t nsteps, int use_graph, cudaStream_t s) {
  apply_pending_correction<T>(c, s);   // a captured step must not carry it
  const int cycle = c.prm.sort_every > 0 ? 2 * c.prm.sort_every : 1;
  int32_t left = nsteps;
  if (use_graph) {
    // eager steps up to the start of a re-order cycle, then whole cycles from the graph
    while (left > 0 && c.steps_since_sort != 0) { PDFX_TRY(do_step<T>(c, dt, s)); --left; }
    if (left >= cycle) {
      if (!c.gexec || c.g_dt != dt || c.g_steps != cycle || c.g_buf != c.pbuf[0] || c.g_np != c.np)
        PDFX_TRY(capture_cycle<T>(c, dt, cycle));
      while (left >= cycle) {
        PDFX_CUDA(cudaGraphLaunch(c.gexec, s));
        c.step += static_cast<uint32_t>(cycle);
        c.steps_done += cycle;
        c.launches += c.g_launches;
        left -= cycle;
      }
    }
  }
  for (; left > 0; --left) PDFX_TRY(do_step<T>(c, dt, s));
  return cerr(cudaGetLastError());
}

// Launch shapes that leave every result unchanged: the advance kernel's block size (each
// particle is independent) and the re-order period (no result depends on the slots'
// order: every ordering decision of the method goes through particle ids).  Each candidate
// runs one re-order cycle from the same snapshot of the state; the state, counters and
// diagnostics are restored afterwards.
template <typename T>
int do_autotune(Ctx& c, double dt, cudaStream_t s, int32_t* best_block, int32_t* best_se) {
  apply_pending_correction<T>(c, s);
  const size_t pb = c.pbuf_bytes;
  const size_t vb = sizeof(double) * static_cast<size_t>(c.ne) * c.G;
  const size_t eb = sizeof(double) * static_cast<size_t>(c.ne) * kNS;
  const size_t nb = sizeof(double) * static_cast<size_t>(c.nn) * kNS;
  const size_t gb = sizeof(int32_t) * static_cast<size_t>(c.ne) * 3;
  const size_t db = sizeof(unsigned long long) * kDiagCount;
  const size_t rb = sizeof(double) * 4 * kLostRecords;
  unsigned char* snap = static_cast<unsigned char*>(dev_alloc(c, pb + vb + eb + nb + gb + db + rb + 16));
  if (!snap) return PDFX_ERR_ALLOC;
  struct Piece { void* dev; size_t bytes; };
  const Piece pieces[] = {{c.pbuf[c.cur], pb}, {c.vcce, vb}, {c.emom, eb}, {c.nmom, nb},
                          {c.gbin, gb}, {c.diag, db}, {c.lost_rec, rb}, {c.err, 16}};
  size_t off = 0;
  for (const Piece& q : pieces) {
    PDFX_CUDA(cudaMemcpyAsync(snap + off, q.dev, q.bytes, cudaMemcpyDeviceToDevice, s));
    off += q.bytes;
  }
  const int cur0 = c.cur, since0 = c.steps_since_sort, block0 = c.adv_block;
  const int se0 = c.prm.sort_every;
  const uint32_t step0 = c.step;
  const int64_t done0 = c.steps_done, launches0 = c.launches;
  const bool prof0 = c.profiling;
  c.profiling = false;
  auto restore = [&]() -> int {
    c.cur = cur0;
    size_t o = 0;
    const Piece back[] = {{c.pbuf[cur0], pb}, {c.vcce, vb}, {c.emom, eb}, {c.nmom, nb},
                          {c.gbin, gb}, {c.diag, db}, {c.lost_rec, rb}, {c.err, 16}};
    for (const Piece& q : back) {
      PDFX_CUDA(cudaMemcpyAsync(q.dev, snap + o, q.bytes, cudaMemcpyDeviceToDevice, s));
      o += q.bytes;
    }
    c.steps_since_sort = since0;
    c.step = step0;
    c.steps_done = done0;
    c.launches = launches0;
    PDFX_CUDA(cudaMemcpyAsync(c.dstep, &step0, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    return cerr(cudaStreamSynchronize(s));
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    dev_free(c, snap);
    return PDFX_ERR_CUDA;
  }
  const int blocks[] = {128, 256};
  const int periods[] = {4, 8, 16};
  const int splits[] = {0, 128, 192, 256};
  const int split0 = c.tile_split;
  // one re-order cycle from the snapshot with the given shapes: milliseconds per step
  auto time_cycle = [&](int blk, int se, int split, double* ms_step) -> int {
    PDFX_TRY(restore());
    c.adv_block = blk;
    c.prm.sort_every = se;
    c.tile_split = split;
    PDFX_TRY(do_step<T>(c, dt, s));                    // warm-up
    const int n = 2 * se;
    PDFX_CUDA(cudaEventRecord(e0, s));
    for (int k = 0; k < n; ++k) PDFX_TRY(do_step<T>(c, dt, s));
    PDFX_CUDA(cudaEventRecord(e1, s));
    PDFX_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    PDFX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *ms_step = ms / n;
    return PDFX_OK;
  };
  double best = 1e300;
  int bb = block0, bs = se0, bsp = split0;
  int rc = PDFX_OK;
  for (int blk : blocks)
    for (int se : periods) {
      double ms = 0.0;
      if (rc == PDFX_OK) rc = time_cycle(blk, se, split0, &ms);
      if (rc == PDFX_OK && ms < best) { best = ms; bb = blk; bs = se; }
    }
  // then the binning's size-class split with the chosen block size and period
  for (int sp : splits) {
    double ms = 0.0;
    if (rc == PDFX_OK && sp != split0) rc = time_cycle(bb, bs, sp, &ms);
    else continue;
    if (rc == PDFX_OK && ms < best) { best = ms; bsp = sp; }
  }
  const int rr = restore();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(c, snap);
  c.profiling = prof0;
  if (rc != PDFX_OK || rr != PDFX_OK) {
    c.adv_block = block0;
    c.prm.sort_every = se0;
    c.tile_split = split0;
    return rc != PDFX_OK ? rc : rr;
  }
  c.adv_block = bb;
  c.prm.sort_every = bs;
  c.tile_split = bsp;
  drop_graph(c);
  if (best_block) *best_block = bb;
  if (best_se) *best_se = bs;
  return PDFX_OK;
}

Ctx* as_ctx(void* p) { return static_cast<Ctx*>(p); }

// The simplified model of Eqs. 46-47 has no wall treatment: its grid may not have no-slip
// walls (free-slip boundaries and a periodic direction only).
bool model_fits_grid(const Ctx& c) { return c.prm.model != 1 || c.n_wall_lines == 0; }

// Eq. 26 from the nodal means of the last statistics pass (synchronises the stream).
int cfl_dt(Ctx& c, cudaStream_t s, double* dt) {
  if (c.K > 1 || !c.dnorm || c.nn <= 0) return PDFX_ERR_ARG;
  launch_cfl_norm(c.nmom, c.nn, c.dnorm, s);
  c.launches++;
  double norm = 0.0;
  PDFX_CUDA(cudaMemcpyAsync(&norm, c.dnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
  PDFX_CUDA(cudaStreamSynchronize(s));
  if (!(norm > 0.0) || !std::isfinite(norm)) return PDFX_ERR_ARG;
  *dt = c.prm.cfl * c.min_sqrt_an / norm;
  return (*dt > 0.0 && std::isfinite(*dt)) ? PDFX_OK : PDFX_ERR_ARG;
}


// ---------------------------------------------------------------------------------------
// Eulerian solves of the coupled loop (Sect. 3.2): FEM data, Jacobi-PCG, the elliptic
// relaxation (Eqs. 12-18, 59), the pressure projection (Eqs. 33, 61) and the coupled step
// in the order of Table 1.  Single grids only (a batch's instances would each need their
// own pressure null space).
// ---------------------------------------------------------------------------------------

template <typename P>
int upload_vec(Ctx& c, P*& dst, const std::vector<P>& src) {
  PDFX_TRY(alloc_into(c, dst, src.size()));
  if (!src.empty()) PDFX_CUDA(cudaMemcpy(dst, src.data(), sizeof(P) * src.size(), cudaMemcpyHostToDevice));
  return PDFX_OK;
}

// Work arrays of the Eulerian calls, carved from c.ew.
struct EWork {
  double *x, *b, *r, *z, *d, *q, *d2;   // [9][nn] solver vectors (d2: second direction)
  double *rhs;                     // [9][nn] right-hand side of Eq. 12
  double *L;                       // [nn] length scale of Eq. 16
  double *aval, *adiag;            // [nnz], [nn] elliptic-relaxation matrix
  double *src, *flux;              // [nn] Eq. 33 source, increment normal derivative
  double *pcg;                     // PCG partial sums and scalars
  double *prs;                     // derivative passes of the pressure source
  double *big;                     // 18 (ne + nn): derived fields, element gradients
  double *red;                     // kRedBlocks + 8: reductions
  unsigned *ticket;                // [9] last-block counters (zeroed once)
};

size_t ework_doubles(const Ctx& c) {
  const size_t N = static_cast<size_t>(c.nn), E = static_cast<size_t>(c.ne);
  return 8 * 9 * N + N + static_cast<size_t>(c.fem.nnz) + N + 2 * N + pcg_scratch_doubles(c.nn, 9) +
         pressure_rhs_scratch_doubles(c.nn, c.ne) + 18 * (E + N) + (kRedBlocks + 8) + 8;
}

EWork ework(Ctx& c) {
  const size_t N = static_cast<size_t>(c.nn), N9 = 9 * N, E = static_cast<size_t>(c.ne);
  double* p = c.ew;
  EWork w{};
  w.x = p; p += N9;
  w.b = p; p += N9;
  w.r = p; p += N9;
  w.z = p; p += N9;
  w.d = p; p += N9;
  w.q = p; p += N9;
  w.d2 = p; p += N9;
  w.rhs = p; p += N9;
  w.L = p; p += N;
  w.aval = p; p += static_cast<size_t>(c.fem.nnz);
  w.adiag = p; p += N;
  w.src = p; p += N;
  w.flux = p; p += N;
  w.pcg = p; p += pcg_scratch_doubles(c.nn, 9);
  w.prs = p; p += pressure_rhs_scratch_doubles(c.nn, c.ne);
  w.big = p; p += 18 * (E + N);
  w.red = p; p += kRedBlocks + 8;
  w.ticket = reinterpret_cast<unsigned*>(p);
  return w;
}

// The FEM data of the current grid (host, FP64) and the device work arrays.
int ensure_fem(Ctx& c) {
  if (c.fem_ready) return PDFX_OK;
  if (!c.have_grid || c.K > 1) return PDFX_ERR_ARG;
  FemHost h;
  if (!build_fem_host(c.nn, c.ne, c.h_tri, c.h_tag, c.h_vx, c.h_vy, c.h_area2, h)) return PDFX_ERR_MESH;
  FemDev& m = c.fem;
  m.nn = c.nn;
  m.ne = c.ne;
  m.nnz = h.row[c.nn];
  m.area = h.area;
  m.cxi = h.cxi;
  const size_t nn = static_cast<size_t>(c.nn);
  PDFX_TRY(upload_vec(c, m.row, h.row));
  PDFX_TRY(upload_vec(c, m.col, h.col));
  PDFX_TRY(upload_vec(c, m.dpos, h.dpos));
  PDFX_TRY(upload_vec(c, m.cptr, h.cptr));
  PDFX_TRY(upload_vec(c, m.clist, h.clist));
  PDFX_TRY(upload_vec(c, m.tri, c.h_tri));
  PDFX_TRY(upload_vec(c, m.fe, h.fe));
  PDFX_TRY(upload_vec(c, m.mval, h.mval));
  PDFX_TRY(upload_vec(c, m.kval, h.kval));
  PDFX_TRY(upload_vec(c, m.kdiag, h.kdiag));
  PDFX_TRY(upload_vec(c, m.mlump, h.mlump));
  PDFX_TRY(upload_vec(c, m.ncls, h.cls));
  PDFX_TRY(upload_vec(c, m.nrm, h.nrm));
  PDFX_TRY(upload_vec(c, m.boff, h.boff));
  PDFX_TRY(upload_vec(c, m.bnb, h.bnb));
  PDFX_TRY(upload_vec(c, m.blen, h.blen));
  PDFX_TRY(alloc_into(c, c.ew, ework_doubles(c)));
  PDFX_CUDA(cudaMemset(ework(c).ticket, 0, 8 * sizeof(double)));
  PDFX_TRY(alloc_into(c, c.efixed, 9 * nn));
  PDFX_TRY(alloc_into(c, c.eflag, 1));
  PDFX_TRY(alloc_into(c, c.P, nn));
  PDFX_TRY(alloc_into(c, c.dP, nn));
  PDFX_TRY(alloc_into(c, c.corr, 2 * static_cast<size_t>(c.ne)));
  PDFX_CUDA(cudaMemset(c.P, 0, sizeof(double) * nn));
  PDFX_CUDA(cudaMemset(c.dP, 0, sizeof(double) * nn));
  c.fem_ready = true;
  return PDFX_OK;
}

WpConst wp_const(const Ctx& c) {
  const pdfx_params& p = c.prm;
  WpConst k{};
  k.C1 = p.C1; k.C2 = p.C2; k.Cv = p.Cv; k.gamma5 = p.gamma5; k.CL = p.CL; k.Ceta = p.Ceta;
  k.CT = p.CT; k.nu = p.nu; k.cxi = c.fem.cxi;
  return k;
}

// 16 conjugate-gradient iterations (two kernels each) as a CUDA graph for this solve
// configuration, captured on the library's stream the first time and kept until the grid
// changes (the arrays are the grid's work arrays).
constexpr int kPcgChunk = 16;
int pcg_graph(Ctx& c, const PcgArgs& a, cudaGraphExec_t* out) {
  const void* key[4] = {a.val, a.x, a.b, a.fixed};
  Ctx::PcgGraph* free_slot = nullptr;
  for (Ctx::PcgGraph& g : c.pcg_graphs) {
    if (g.exec && g.C == a.C && g.tol == a.tol && std::equal(key, key + 4, g.key)) {
      *out = g.exec;
      return PDFX_OK;
    }
    if (!g.exec && !free_slot) free_slot = &g;
  }
  if (!free_slot) {                      // all in use: replace the first
    free_slot = &c.pcg_graphs[0];
    cudaGraphExecDestroy(free_slot->exec);
    free_slot->exec = nullptr;
  }
  if (!c.gstream && cudaStreamCreateWithFlags(&c.gstream, cudaStreamNonBlocking) != cudaSuccess)
    return PDFX_ERR_CUDA;
  PDFX_CUDA(cudaStreamBeginCapture(c.gstream, cudaStreamCaptureModeThreadLocal));
  for (int j = 0; j < kPcgChunk / 2; ++j) launch_pcg_two_iterations(c.fem, a, c.gstream);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c.gstream, &g);
  if (ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return PDFX_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&free_slot->exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) { free_slot->exec = nullptr; return PDFX_ERR_CUDA; }
  free_slot->C = a.C;
  free_slot->tol = a.tol;
  std::copy(key, key + 4, free_slot->key);
  *out = free_slot->exec;
  return PDFX_OK;
}
void drop_pcg_graphs(Ctx& c) {
  for (Ctx::PcgGraph& g : c.pcg_graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = Ctx::PcgGraph{};
  }
}

// Iterates until every component meets its stopping rule, in chunks of 16 iterations
// replayed from a graph and checked on the host after each chunk (a component that has
// converged stops changing); more than max_iter iterations of a component is an error.
int run_pcg(Ctx& c, const PcgArgs& a, int32_t max_iter, int32_t* iters, cudaStream_t s) {
  launch_pcg_setup(c.fem, a, s);
  c.launches += 8;
  const double* sc = pcg_scalars(a, c.nn);
  std::vector<double> h(static_cast<size_t>(a.C) * kPcgScalars);
  cudaGraphExec_t chunk = nullptr;
  int32_t done = 0;
  for (;;) {
    PDFX_CUDA(cudaMemcpyAsync(h.data(), sc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    PDFX_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int j = 0; j < a.C; ++j) any |= h[static_cast<size_t>(j) * kPcgScalars + kPcgActive] != 0.0;
    if (!any) break;
    if (done >= max_iter) return PDFX_ERR_SOLVE;
    if (!chunk) PDFX_TRY(pcg_graph(c, a, &chunk));
    PDFX_CUDA(cudaGraphLaunch(chunk, s));
    c.launches += 2 * kPcgChunk;
    done += kPcgChunk;
  }
  int32_t most = 0;
  for (int j = 0; j < a.C; ++j)
    most = std::max(most, static_cast<int32_t>(h[static_cast<size_t>(j) * kPcgScalars + kPcgIters]));
  if (most > max_iter) return PDFX_ERR_SOLVE;
  if (iters) *iters = most;
  return PDFX_OK;
}

int read_flag(Ctx& c, cudaStream_t s) {
  int flag = 0;
  PDFX_CUDA(cudaMemcpyAsync(&flag, c.eflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  PDFX_CUDA(cudaStreamSynchronize(s));
  return flag ? PDFX_ERR_ARG : PDFX_OK;
}

// Eq. 12 from w.rhs, w.L and the initial guess in w.x (Dirichlet values set here).
template <typename T>
int wp_solve_dev(Ctx& c, const EWork& w, double tol, int32_t max_iter, int32_t* iters, cudaStream_t s) {
  const WpConst k = wp_const(c);
  PDFX_CUDA(cudaMemsetAsync(c.eflag, 0, sizeof(int), s));
  launch_wp_bc<T>(static_cast<const T*>(c.fields), c.nn, k, c.fem.ncls, c.fem.nrm, c.efixed, w.x, c.eflag, s);
  launch_assemble_wp(c.fem, w.L, w.aval, w.adiag, s);
  launch_spmv(c.fem, c.fem.mval, 9, w.rhs, w.b, s);
  c.launches += 4;
  PDFX_TRY(read_flag(c, s));
  PcgArgs a;
  a.C = 9; a.val = w.aval; a.diag = w.adiag; a.fixed = c.efixed; a.b = w.b;
  a.x = w.x; a.r = w.r; a.z = w.z; a.d = w.d; a.q = w.q; a.d2 = w.d2; a.ticket = w.ticket;
  a.scratch = w.pcg; a.tol = tol;
  return run_pcg(c, a, max_iter, iters, s);
}

template <typename T>
int wp_rhs_dev(Ctx& c, const EWork& w, cudaStream_t s) {
  PDFX_CUDA(cudaMemsetAsync(c.eflag, 0, sizeof(int), s));
  launch_wp_rhs<T>(static_cast<const T*>(c.fields), c.nn, wp_const(c), w.rhs, w.L, c.eflag, s);
  c.launches++;
  return read_flag(c, s);
}

// The fields' wp_ij: right-hand side and length scale from the fields, solved from slots
// 14-22 and written back there.
template <typename T>
int update_wp_dev(Ctx& c, const EWork& w, double tol, int32_t max_iter, int32_t* iters, cudaStream_t s) {
  PDFX_TRY(wp_rhs_dev<T>(c, w, s));
  launch_read_wp<T>(c.nn, static_cast<const T*>(c.fields), w.x, s);
  c.launches++;
  PDFX_TRY(wp_solve_dev<T>(c, w, tol, max_iter, iters, s));
  launch_write_wp<T>(c.nn, w.x, static_cast<T*>(c.fields), s);
  c.launches++;
  return cerr(cudaGetLastError());
}

// Eq. 33 from w.src and w.flux into x (initial guess in), zero integral.
int pressure_dev(Ctx& c, const EWork& w, double* x, double tol, int32_t max_iter, int32_t* iters,
                 cudaStream_t s) {
  launch_pressure_load(c.fem, w.src, w.flux, w.b, w.red, s);
  c.launches += 4;
  PcgArgs a;
  a.C = 1; a.val = c.fem.kval; a.diag = c.fem.kdiag; a.fixed = nullptr; a.b = w.b;
  a.x = x; a.r = w.r; a.z = w.z; a.d = w.d; a.q = w.q; a.d2 = w.d2; a.ticket = w.ticket;
  a.scratch = w.pcg; a.tol = tol;
  PDFX_TRY(run_pcg(c, a, max_iter, iters, s));
  launch_zero_mean(c.fem, x, w.red, s);
  c.launches += 3;
  return cerr(cudaGetLastError());
}

template <typename T>
int do_coupled_step(Ctx& c, double dt, double Cp, double tol, int32_t max_iter, int32_t* iters, cudaStream_t s) {
  const EWork w = ework(c);
  int32_t iw = 0, ip = 0;
  PDFX_TRY(update_wp_dev<T>(c, w, tol, max_iter, &iw, s));
  PDFX_TRY(do_step<T>(c, dt, s));   // prediction (Eq. 27 and the other equations), control, statistics
  T* fields = static_cast<T*>(c.fields);
  launch_pressure_rhs<T>(c.fem, c.ne_off, c.ne_list, c.nmom, kNS, 1, c.P, fields, c.prm.nu, dt, Cp, w.prs,
                         w.src, w.flux, s);
  c.launches += 7;
  PDFX_TRY(pressure_dev(c, w, c.dP, tol, max_iter, &ip, s));
  const ElemGeo<T>* geo = static_cast<const ElemGeo<T>*>(c.geo);
  // Eq. 31: U -= dt grad(dP), one vector per element.  It shifts the particles of an element
  // together, so the statistics follow by shifting the element means (central moments,
  // conditioning order and conditional means stay) and averaging at the nodes; the
  // particles take it as the next advance reads them (or before any other reader).
  launch_correction_field<T>(geo, c.topo, c.ne, c.prm.period_x, nullptr, nullptr, c.dP, dt, c.corr, s);
  launch_shift_means(c.ne, c.corr, c.emom, s);
  launch_node_average(c.emom, c.ne_off, c.ne_list, c.nn, c.nmom, s);
  c.corr_pending = true;
  c.launches += 4;
  launch_add(c.nn, c.dP, c.P, s);
  launch_derive_fields<T>(geo, c.topo, c.ne, c.prm.period_x, nullptr, nullptr, c.ne_off, c.ne_list, c.nn,
                          c.nmom, w.big, fields, s);
  launch_write_pgrad<T>(c.fem, c.ne_off, c.ne_list, c.P, w.big, w.big + 2 * static_cast<size_t>(c.ne),
                        fields, s);
  c.launches += 9;
  drop_graph(c);
  if (iters) { iters[0] = iw; iters[1] = ip; }
  return cerr(cudaGetLastError());
}

// [nn][9] host <-> [9][nn] device.
int upload_9(const double* h, double* d, int nn, cudaStream_t s) {
  std::vector<double> t(9 * static_cast<size_t>(nn));
  for (int n = 0; n < nn; ++n)
    for (int j = 0; j < 9; ++j) t[static_cast<size_t>(j) * nn + n] = h[9 * static_cast<size_t>(n) + j];
  PDFX_CUDA(cudaMemcpyAsync(d, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, s));
  return cerr(cudaStreamSynchronize(s));
}
int download_9(const double* d, double* h, int nn, cudaStream_t s) {
  std::vector<double> t(9 * static_cast<size_t>(nn));
  PDFX_CUDA(cudaMemcpyAsync(t.data(), d, sizeof(double) * t.size(), cudaMemcpyDeviceToHost, s));
  PDFX_CUDA(cudaStreamSynchronize(s));
  for (int n = 0; n < nn; ++n)
    for (int j = 0; j < 9; ++j) h[9 * static_cast<size_t>(n) + j] = t[static_cast<size_t>(j) * nn + n];
  return PDFX_OK;
}
int upload_n(const double* h, double* d, size_t n, cudaStream_t s) {
  PDFX_CUDA(cudaMemcpyAsync(d, h, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  return cerr(cudaStreamSynchronize(s));
}
int download_n(const double* d, double* h, size_t n, cudaStream_t s) {
  PDFX_CUDA(cudaMemcpyAsync(h, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  return cerr(cudaStreamSynchronize(s));
}

// Common checks of the Eulerian entry points.
int eulerian_ready(Ctx* c, bool need_fields) {
  if (!c) return PDFX_ERR_ARG;
  if (!c->have_grid || (need_fields && !c->have_fields)) return PDFX_ERR_ORDER;
  if (c->K > 1) return PDFX_ERR_ARG;
  return ensure_fem(*c);
}

bool solve_args_ok(double tol, int32_t max_iter) {
  return tol > 0.0 && std::isfinite(tol) && max_iter >= 0;
}

}  // namespace
}  // namespace pdfx

using namespace pdfx;

extern "C" {

void pdfx_default_params(pdfx_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  // Table 4
  p->C1 = 1.85; p->C2 = 0.63; p->C3 = 5.0; p->C4 = 0.25; p->CT = 6.0; p->CL = 0.134;
  p->Ceta = 72.0; p->Cv = 1.4; p->gamma5 = 0.1; p->Cw1 = 0.5; p->Cw2 = 0.73;
  p->nu = 1e-4;
  p->c0_mode = 0; p->C0 = 3.5;
  p->tm_mode = 0; p->Cs = 0.02; p->Ct = 0.7; p->Cphi = 2.0;
  p->src_x = 0.5; p->src_y = 0.5; p->src_r = 0.02;
  p->bins[0] = p->bins[1] = p->bins[2] = 4;
  p->cond_mode = 0;
  p->fox_bins = 5;
  p->model = 0;
  p->alpha = 0.5;
  p->cfl = 0.7;
  p->min_per_bin = 2;
  p->minnpel = 0;
  p->interp_mode = 0;
  p->source_on = 1;
  p->seed = 1;
  p->instance = 0;
  p->period_x = 0.0;
  p->precision = 0;
  p->sort_every = 8;
}

int pdfx_create(const pdfx_params* p, const pdfx_allocator* alloc, void** out) {
  if (!p || !out) return PDFX_ERR_ARG;
  *out = nullptr;
  if (!params_valid(*p)) return PDFX_ERR_ARG;
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return PDFX_ERR_ALLOC;
  c->prm = *p;
  if (alloc && alloc->alloc && alloc->release) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  c->G = p->cond_mode == 1 ? p->fox_bins : p->bins[0] * p->bins[1] * p->bins[2];
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return PDFX_ERR_CUDA;
  }
  {
    bool ok = true;
    for (cudaStream_t& st : c->side.side)
      ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t& e : c->side.ev)
      ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    c->side.ok = ok;
  }
  c->diag = static_cast<unsigned long long*>(dev_alloc(*c, sizeof(unsigned long long) * kDiagCount));
  c->err = static_cast<int*>(dev_alloc(*c, sizeof(int) * 4));
  c->brute_list = static_cast<int32_t*>(dev_alloc(*c, sizeof(int32_t) * kBruteCap));
  c->lost_rec = static_cast<double*>(dev_alloc(*c, sizeof(double) * 4 * kLostRecords));
  c->dstep = static_cast<uint32_t*>(dev_alloc(*c, sizeof(uint32_t)));
  if (!c->diag || !c->err || !c->brute_list || !c->lost_rec || !c->dstep) {
    pdfx_destroy(c);
    return PDFX_ERR_ALLOC;
  }
  if (cudaMemset(c->diag, 0, sizeof(unsigned long long) * kDiagCount) != cudaSuccess ||
      cudaMemset(c->err, 0, sizeof(int) * 4) != cudaSuccess ||
      cudaMemset(c->dstep, 0, sizeof(uint32_t)) != cudaSuccess) {
    pdfx_destroy(c);
    return PDFX_ERR_CUDA;
  }
  *out = c;
  return PDFX_OK;
}

void pdfx_destroy(void* ctx) {
  Ctx* c = as_ctx(ctx);
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (Ctx::PcgGraph& g : c->pcg_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  for (cudaStream_t st : c->side.side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : c->side.ev)
    if (e) cudaEventDestroy(e);
  for (auto& o : c->owned) {
    if (c->has_alloc) c->alloc.release(o.first, o.second, c->alloc.user);
    else cudaFree(o.first);
  }
  c->owned.clear();
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (auto& pe : c->ev_pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
  delete c;
}

int pdfx_set_params(void* ctx, const pdfx_params* p) {
  Ctx* c = as_ctx(ctx);
  if (!c || !p || !params_valid(*p)) return PDFX_ERR_ARG;
  if (p->precision != c->prm.precision || p->sort_every != c->prm.sort_every ||
      p->acc64 != c->prm.acc64 || p->cond_mode != c->prm.cond_mode ||
      (p->cond_mode == 1 && p->fox_bins != c->prm.fox_bins) || p->model != c->prm.model ||
      p->bins[0] != c->prm.bins[0] || p->bins[1] != c->prm.bins[1] || p->bins[2] != c->prm.bins[2])
    return PDFX_ERR_ARG;
  if (c->have_grid && p->period_x != c->prm.period_x) return PDFX_ERR_ARG;
  if (c->K > 1) return PDFX_ERR_ARG;   // a batch takes its parameters from pdfx_set_instances
  c->prm = *p;
  drop_graph(*c);
  if (c->np > 0) return upload_inst_any(*c);
  return PDFX_OK;
}

int pdfx_set_instances(void* ctx, int32_t n, const pdfx_params* p, const int32_t* elem_first) {
  Ctx* c = as_ctx(ctx);
  if (!c || n < 1 || !p || !elem_first || elem_first[0] != 0) return PDFX_ERR_ARG;
  for (int32_t k = 0; k < n; ++k) {
    if (elem_first[k + 1] <= elem_first[k] || !params_valid(p[k])) return PDFX_ERR_ARG;
    if (p[k].precision != c->prm.precision || p[k].sort_every != c->prm.sort_every ||
        p[k].bins[0] != c->prm.bins[0] || p[k].bins[1] != c->prm.bins[1] ||
        p[k].bins[2] != c->prm.bins[2] || p[k].min_per_bin != c->prm.min_per_bin ||
        p[k].acc64 != c->prm.acc64 || p[k].cond_mode != c->prm.cond_mode ||
        (p[k].cond_mode == 1 && p[k].fox_bins != c->prm.fox_bins) || p[k].model != c->prm.model)
      return PDFX_ERR_ARG;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return PDFX_ERR_CUDA;
  drop_graph(*c);
  if (n == 1) {
    c->K = 1;
    c->iprm.clear();
    c->prm = p[0];
  } else {
    c->K = n;
    c->iprm.assign(p, p + n);
  }
  c->h_ielem.assign(elem_first, elem_first + n + 1);
  c->h_ippe.clear();
  for (int b = 0; b < 2; ++b) { dev_free(*c, c->pbuf[b]); c->pbuf[b] = nullptr; }
  c->np = 0;
  c->have_grid = false;
  c->have_fields = false;
  return PDFX_OK;
}

int pdfx_instance_ranges(const void* ctx, int32_t* elem_first, int64_t* part_first) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  if (!c) return PDFX_ERR_ARG;
  if (elem_first) for (int k = 0; k <= c->K && k < static_cast<int>(c->h_ielem.size()); ++k) elem_first[k] = c->h_ielem[k];
  if (part_first) for (int k = 0; k <= c->K && k < static_cast<int>(c->h_ip0.size()); ++k) part_first[k] = c->h_ip0[k];
  return c->K;
}

int pdfx_set_grid(void* ctx, int32_t nn, const double* node_xy, int32_t ne, const int32_t* tri,
                  const int8_t* edge_tag) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return PDFX_ERR_CUDA;
  drop_graph(*c);
  return set_grid(*c, nn, node_xy, ne, tri, edge_tag);
}

int pdfx_set_fields(void* ctx, const double* fields, int on_device, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !fields) return PDFX_ERR_ARG;
  if (!c->have_grid) return PDFX_ERR_ORDER;
  const cudaStream_t s = as_stream(stream);
  const size_t n = static_cast<size_t>(c->nn) * kNF;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (c->prm.precision == 1) {
    PDFX_CUDA(cudaMemcpyAsync(c->fields64, fields, sizeof(double) * n, kind, s));
    launch_convert_fields(c->fields64, static_cast<float*>(c->fields), static_cast<int64_t>(n), s);
    c->launches++;
  } else {
    PDFX_CUDA(cudaMemcpyAsync(c->fields, fields, sizeof(double) * n, kind, s));
  }
  c->have_fields = true;
  return cerr(cudaGetLastError());
}

int pdfx_init_particles_batch(void* ctx, const int32_t* ppe, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !ppe) return PDFX_ERR_ARG;
  if (!c->have_grid || !c->have_fields) return PDFX_ERR_ORDER;
  int64_t total = 0;
  for (int k = 0; k < c->K; ++k) {
    const int64_t nk = static_cast<int64_t>(ppe[k]) * (c->h_ielem[k + 1] - c->h_ielem[k]);
    if (ppe[k] <= 0 || nk >= kMaxParticles) return PDFX_ERR_ARG;
    total += nk;
  }
  if (total > kMaxSlots) return PDFX_ERR_ARG;
  drop_graph(*c);
  return c->prm.precision == 1 ? do_init<float>(*c, ppe, as_stream(stream))
                               : do_init<double>(*c, ppe, as_stream(stream));
}

int pdfx_init_particles(void* ctx, int32_t ppe, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || ppe <= 0) return PDFX_ERR_ARG;
  const std::vector<int32_t> all(static_cast<size_t>(c->K), ppe);
  return pdfx_init_particles_batch(ctx, all.data(), stream);
}

int pdfx_set_particles(void* ctx, int64_t np, const pdfx_soa* s, uint32_t step, int on_device,
                       void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !s || np < 0 || np > kMaxSlots || (c->K <= 1 && np >= kMaxParticles)) return PDFX_ERR_ARG;
  if (np > 0 && (!s->x || !s->y || !s->u || !s->v || !s->w || !s->om || !s->psi || !s->elem))
    return PDFX_ERR_ARG;
  if (!c->have_grid) return PDFX_ERR_ORDER;
  if (!on_device)
    for (int64_t i = 0; i < np; ++i)
      if (s->elem[i] < 0 || s->elem[i] >= c->ne) return PDFX_ERR_ARG;
  if (c->K > 1) {
    // a batch state is given instance by instance (ids restart at each instance)
    if (on_device) return PDFX_ERR_ARG;
    c->h_ip0.assign(static_cast<size_t>(c->K) + 1, 0);
    int prev = 0;
    for (int64_t i = 0; i < np; ++i) {
      const int k = inst_of_element(*c, s->elem[i]);
      if (k < prev) return PDFX_ERR_ARG;
      prev = k;
      c->h_ip0[k + 1]++;
    }
    for (int k = 0; k < c->K; ++k) {
      if (c->h_ip0[k + 1] >= kMaxParticles) return PDFX_ERR_ARG;
      c->h_ip0[k + 1] += c->h_ip0[k];
    }
  } else {
    c->h_ip0 = {0, np};
  }
  drop_graph(*c);
  return c->prm.precision == 1 ? do_set_particles<float>(*c, np, s, step, on_device, as_stream(stream))
                               : do_set_particles<double>(*c, np, s, step, on_device, as_stream(stream));
}

int pdfx_get_particles(void* ctx, pdfx_soa* s, int on_device, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !s) return PDFX_ERR_ARG;
  if (!c->pbuf[0]) return PDFX_ERR_ORDER;
  return c->prm.precision == 1 ? do_get_particles<float>(*c, s, on_device, as_stream(stream))
                               : do_get_particles<double>(*c, s, on_device, as_stream(stream));
}

int pdfx_last_dt(const void* ctx, double* dt) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  if (!c || !dt) return PDFX_ERR_ARG;
  *dt = c->last_dt;
  return PDFX_OK;
}

int64_t pdfx_num_particles(const void* ctx) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  return c ? c->np : 0;
}

uint32_t pdfx_step_index(const void* ctx) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  return c ? c->step : 0;
}

int pdfx_step_many(void* ctx, double dt, int32_t nsteps, int use_graph, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || nsteps < 0 || !model_fits_grid(*c) || std::isnan(dt)) return PDFX_ERR_ARG;
  if (!c->pbuf[0] || !c->have_fields) return PDFX_ERR_ORDER;
  if (!(dt > 0.0)) {   // Eq. 26 at every step: plain steps
    for (int32_t i = 0; i < nsteps; ++i) PDFX_TRY(pdfx_step(ctx, dt, stream));
    return PDFX_OK;
  }
  return c->prm.precision == 1 ? do_step_many<float>(*c, dt, nsteps, use_graph, as_stream(stream))
                               : do_step_many<double>(*c, dt, nsteps, use_graph, as_stream(stream));
}

int pdfx_autotune(void* ctx, double dt, int32_t* adv_block, int32_t* sort_every, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !(dt > 0.0) || !model_fits_grid(*c)) return PDFX_ERR_ARG;
  if (!c->pbuf[0] || !c->have_fields || c->np <= 0) return PDFX_ERR_ORDER;
  return c->prm.precision == 1 ? do_autotune<float>(*c, dt, as_stream(stream), adv_block, sort_every)
                               : do_autotune<double>(*c, dt, as_stream(stream), adv_block, sort_every);
}

int pdfx_get_launch_shapes(const void* ctx, int32_t* adv_block, int32_t* sort_every, int32_t* tile_split) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  if (!c) return PDFX_ERR_ARG;
  if (adv_block) *adv_block = c->adv_block;
  if (sort_every) *sort_every = c->prm.sort_every;
  if (tile_split) *tile_split = c->tile_split;
  return PDFX_OK;
}

int pdfx_set_launch_shapes(void* ctx, int32_t adv_block, int32_t sort_every, int32_t tile_split) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  if (adv_block >= 0 && adv_block != 128 && adv_block != 256) return PDFX_ERR_ARG;
  if (tile_split > kTileSplit) return PDFX_ERR_ARG;
  if (adv_block >= 0) c->adv_block = adv_block;
  if (sort_every >= 0) c->prm.sort_every = sort_every;
  if (tile_split >= 0) c->tile_split = tile_split;
  drop_graph(*c);
  return PDFX_OK;
}

int pdfx_step(void* ctx, double dt, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !model_fits_grid(*c) || std::isnan(dt)) return PDFX_ERR_ARG;
  if (!c->pbuf[0] || !c->have_fields) return PDFX_ERR_ORDER;
  if (!(dt > 0.0)) PDFX_TRY(cfl_dt(*c, as_stream(stream), &dt));
  return c->prm.precision == 1 ? do_step<float>(*c, dt, as_stream(stream))
                               : do_step<double>(*c, dt, as_stream(stream));
}

int pdfx_batch_step(void* const* ctxs, int32_t n, double dt, void* stream) {
  if (!ctxs || n < 1) return PDFX_ERR_ARG;
  for (int32_t i = 0; i < n; ++i) {
    if (!ctxs[i]) return PDFX_ERR_ARG;
    for (int32_t j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return PDFX_ERR_ARG;
  }
  for (int32_t i = 0; i < n; ++i) {
    const int rc = pdfx_step(ctxs[i], dt, stream);
    if (rc != PDFX_OK) return rc;
  }
  return PDFX_OK;
}

static int copy_out(void* dst, const void* src, size_t bytes, int on_device, cudaStream_t s) {
  if (!dst) return PDFX_OK;
  if (on_device) return cerr(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
  if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PDFX_ERR_CUDA;
  return cerr(cudaStreamSynchronize(s));
}

int pdfx_get_nodal_stats(void* ctx, double* out, int on_device, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !out) return PDFX_ERR_ARG;
  if (!c->have_grid) return PDFX_ERR_ORDER;
  return copy_out(out, c->nmom, sizeof(double) * kNS * c->nn, on_device, as_stream(stream));
}

int pdfx_derive_fields(void* ctx, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  if (!c->have_grid || !c->have_fields || !c->pbuf[0]) return PDFX_ERR_ORDER;
  const cudaStream_t s = as_stream(stream);
  const size_t n = 18 * (static_cast<size_t>(c->ne) + static_cast<size_t>(c->nn));
  auto* scratch = static_cast<double*>(dev_alloc(*c, sizeof(double) * n));
  if (!scratch) return PDFX_ERR_ALLOC;
  const int32_t* einst = c->K > 1 ? c->einst : nullptr;
  if (c->prm.precision == 1)
    launch_derive_fields<float>(static_cast<const ElemGeo<float>*>(c->geo), c->topo, c->ne,
                                c->prm.period_x, einst, static_cast<const InstDev<float>*>(c->inst),
                                c->ne_off, c->ne_list, c->nn, c->nmom, scratch,
                                static_cast<float*>(c->fields), s);
  else
    launch_derive_fields<double>(static_cast<const ElemGeo<double>*>(c->geo), c->topo, c->ne,
                                 c->prm.period_x, einst, static_cast<const InstDev<double>*>(c->inst),
                                 c->ne_off, c->ne_list, c->nn, c->nmom, scratch,
                                 static_cast<double*>(c->fields), s);
  c->launches += 5;
  int rc = cerr(cudaGetLastError());
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == PDFX_OK) rc = PDFX_ERR_CUDA;
  dev_free(*c, scratch);
  drop_graph(*c);
  return rc;
}

int pdfx_correct_velocity(void* ctx, const double* dp, double dt, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !dp || !(dt > 0.0) || !std::isfinite(dt)) return PDFX_ERR_ARG;
  if (!c->have_grid || !c->pbuf[0]) return PDFX_ERR_ORDER;
  const cudaStream_t s = as_stream(stream);
  const size_t nn = static_cast<size_t>(c->nn), ne = static_cast<size_t>(c->ne);
  auto* scratch = static_cast<double*>(dev_alloc(*c, sizeof(double) * (nn + 2 * ne)));
  if (!scratch) return PDFX_ERR_ALLOC;
  const int32_t* einst = c->K > 1 ? c->einst : nullptr;
  apply_pending_correction_any(*c, s);
  int rc = cerr(cudaMemcpyAsync(scratch, dp, sizeof(double) * nn, cudaMemcpyHostToDevice, s));
  if (rc == PDFX_OK) {
    if (c->prm.precision == 1)
      launch_correct_velocity<float>(static_cast<const ElemGeo<float>*>(c->geo), c->topo, c->ne,
                                     c->prm.period_x, einst, static_cast<const InstDev<float>*>(c->inst),
                                     scratch, scratch + nn, carve<float>(c->pbuf[c->cur], c->np), c->np,
                                     dt, s);
    else
      launch_correct_velocity<double>(static_cast<const ElemGeo<double>*>(c->geo), c->topo, c->ne,
                                      c->prm.period_x, einst,
                                      static_cast<const InstDev<double>*>(c->inst), scratch,
                                      scratch + nn, carve<double>(c->pbuf[c->cur], c->np), c->np, dt, s);
    c->launches += 2;
    rc = cerr(cudaGetLastError());
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == PDFX_OK) rc = PDFX_ERR_CUDA;
  dev_free(*c, scratch);
  return rc;
}

int pdfx_get_fields(void* ctx, double* out, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !out) return PDFX_ERR_ARG;
  if (!c->have_fields) return PDFX_ERR_ORDER;
  const size_t n = static_cast<size_t>(kNF) * c->nn;
  const cudaStream_t s = as_stream(stream);
  if (c->prm.precision == 1) {
    std::vector<float> h(n);
    PDFX_TRY(copy_out(h.data(), c->fields, sizeof(float) * n, 0, s));
    for (size_t i = 0; i < n; ++i) out[i] = static_cast<double>(h[i]);
    return PDFX_OK;
  }
  return copy_out(out, c->fields, sizeof(double) * n, 0, s);
}

int pdfx_get_element_stats(void* ctx, double* out, int32_t* counts, int on_device, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  if (!c->have_grid) return PDFX_ERR_ORDER;
  const cudaStream_t s = as_stream(stream);
  PDFX_TRY(copy_out(out, c->emom, sizeof(double) * kNS * c->ne, on_device, s));
  if (counts) {
    // counts of the last statistics pass: the element moments' first column
    std::vector<double> tmp;
    if (on_device) return PDFX_ERR_ARG;
    tmp.resize(static_cast<size_t>(kNS) * c->ne);
    PDFX_TRY(copy_out(tmp.data(), c->emom, sizeof(double) * tmp.size(), 0, s));
    for (int32_t e = 0; e < c->ne; ++e) counts[e] = static_cast<int32_t>(tmp[kNS * e]);
  }
  return PDFX_OK;
}

int pdfx_get_bins(void* ctx, double* vcce, int32_t* g, int on_device, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  if (!c->have_grid) return PDFX_ERR_ORDER;
  const cudaStream_t s = as_stream(stream);
  PDFX_TRY(copy_out(vcce, c->vcce, sizeof(double) * c->G * c->ne, on_device, s));
  return copy_out(g, c->gbin, sizeof(int32_t) * 3 * c->ne, on_device, s);
}

int pdfx_scalar_stats(void* ctx, int32_t n, const int32_t* elems, int32_t nb, int32_t* count,
                      double* phit, double* cdiff, double* cdiss, double* mom, int on_device,
                      void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || n < 1 || !elems || nb < 1 || nb > PDFX_MAX_SCALAR_BINS) return PDFX_ERR_ARG;
  if (!c->pbuf[0] || !c->have_grid) return PDFX_ERR_ORDER;
  std::vector<int32_t> probe(static_cast<size_t>(c->ne), -1);
  for (int32_t j = 0; j < n; ++j) {
    if (elems[j] < 0 || elems[j] >= c->ne || probe[elems[j]] >= 0) return PDFX_ERR_ARG;
    probe[elems[j]] = j;
  }
  const cudaStream_t s = as_stream(stream);
  const size_t B = static_cast<size_t>(n) * nb, N = static_cast<size_t>(n), E = probe.size();
  // one scratch block: the probe map, the accumulators, the outputs
  const size_t bytes = 4 * E + 4 * B + 8 * 2 * B + 4 * N + 8 * 6 * N + 4 * B + 8 * 3 * B +
                       8 * 6 * N + 16 * 16;
  auto* base = static_cast<unsigned char*>(dev_alloc(*c, bytes));
  if (!base) return PDFX_ERR_ALLOC;
  unsigned char* ptr = base;
  auto take = [&](size_t b) { unsigned char* r = ptr; ptr += (b + 15) & ~size_t(15); return r; };
  auto* dprobe = reinterpret_cast<int32_t*>(take(4 * E));
  ScalarAcc acc;
  acc.count = reinterpret_cast<int32_t*>(take(4 * B));
  acc.sc = reinterpret_cast<unsigned long long*>(take(8 * B));
  acc.sd = reinterpret_cast<unsigned long long*>(take(8 * B));
  acc.n = reinterpret_cast<int32_t*>(take(4 * N));
  acc.s1 = reinterpret_cast<unsigned long long*>(take(8 * N));
  acc.m = reinterpret_cast<unsigned long long*>(take(8 * 3 * N));
  acc.lo = reinterpret_cast<unsigned long long*>(take(8 * N));
  acc.hi = reinterpret_cast<unsigned long long*>(take(8 * N));
  ScalarOut out;
  out.count = reinterpret_cast<int32_t*>(take(4 * B));
  out.phit = reinterpret_cast<double*>(take(8 * B));
  out.cdiff = reinterpret_cast<double*>(take(8 * B));
  out.cdiss = reinterpret_cast<double*>(take(8 * B));
  out.mom = reinterpret_cast<double*>(take(8 * 6 * N));
  int rc = PDFX_OK;
  auto run = [&]() -> int {
    PDFX_CUDA(cudaMemcpyAsync(dprobe, probe.data(), 4 * E, cudaMemcpyHostToDevice, s));
    PDFX_CUDA(cudaMemsetAsync(acc.count, 0, static_cast<size_t>(reinterpret_cast<unsigned char*>(acc.lo) -
                                                                reinterpret_cast<unsigned char*>(acc.count)), s));
    PDFX_CUDA(cudaMemsetAsync(acc.lo, 0xff, 8 * N, s));
    PDFX_CUDA(cudaMemsetAsync(acc.hi, 0, 8 * N, s));
    if (c->prm.precision == 1)
      launch_scalar_stats<float>(carve<float>(c->pbuf[c->cur], c->np), c->np, dprobe, c->vcce, c->G,
                                 n, nb, acc, out, c->num_sms, s);
    else
      launch_scalar_stats<double>(carve<double>(c->pbuf[c->cur], c->np), c->np, dprobe, c->vcce,
                                  c->G, n, nb, acc, out, c->num_sms, s);
    c->launches += c->np > 0 ? 3 : 1;
    PDFX_CUDA(cudaGetLastError());
    PDFX_TRY(copy_out(count, out.count, 4 * B, on_device, s));
    PDFX_TRY(copy_out(phit, out.phit, 8 * B, on_device, s));
    PDFX_TRY(copy_out(cdiff, out.cdiff, 8 * B, on_device, s));
    PDFX_TRY(copy_out(cdiss, out.cdiss, 8 * B, on_device, s));
    PDFX_TRY(copy_out(mom, out.mom, 8 * 6 * N, on_device, s));
    return cerr(cudaStreamSynchronize(s));
  };
  rc = run();
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == PDFX_OK) rc = PDFX_ERR_CUDA;
  dev_free(*c, base);
  return rc;
}

int pdfx_bins_capacity(const void* ctx) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  return c ? c->G : 0;
}

int pdfx_get_diag(void* ctx, pdfx_diag* d, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !d) return PDFX_ERR_ARG;
  unsigned long long h[kDiagCount];
  int err = 0;
  const cudaStream_t s = as_stream(stream);
  PDFX_CUDA(cudaMemcpyAsync(h, c->diag, sizeof(h), cudaMemcpyDeviceToHost, s));
  PDFX_CUDA(cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PDFX_CUDA(cudaStreamSynchronize(s));
  std::memset(d, 0, sizeof(*d));
  d->steps = c->steps_done;
  d->hops_total = static_cast<int64_t>(h[kDiagHops]);
  d->walk_fallback = static_cast<int64_t>(h[kDiagFallback]);
  d->walk_brute = static_cast<int64_t>(h[kDiagBrute]);
  d->lost = static_cast<int64_t>(h[kDiagLost]);
  d->wall_hits = static_cast<int64_t>(h[kDiagWall]);
  d->freeslip_hits = static_cast<int64_t>(h[kDiagFreeSlip]);
  d->omega_reflect = static_cast<int64_t>(h[kDiagOmegaReflect]);
  d->c0_clamp = static_cast<int64_t>(h[kDiagC0Clamp]);
  d->gamma_exhausted = static_cast<int64_t>(h[kDiagGammaExhausted]);
  d->moves = static_cast<int64_t>(h[kDiagMoves]);
  d->source_hits = static_cast<int64_t>(h[kDiagSource]);
  d->capacity_overflow = static_cast<int64_t>(h[kDiagCapacity]);
  d->nonfinite = static_cast<int64_t>(h[kDiagNonFinite]);
  int64_t moved = 0;
  for (int b = 1; b < 8; ++b) {
    d->hop_hist[b] = static_cast<int64_t>(h[kDiagHopHist0 + b]);
    moved += d->hop_hist[b];
  }
  d->hop_hist[0] = c->steps_done * c->np - moved;
  d->error = err;
  const int nrec = static_cast<int>(h[kDiagLostRecord] < kLostRecords ? h[kDiagLostRecord] : kLostRecords);
  if (nrec > 0) {
    PDFX_CUDA(cudaMemcpy(d->lost_xy, c->lost_rec, sizeof(double) * 4 * nrec, cudaMemcpyDeviceToHost));
  }
  d->lost_records = nrec;
  d->bad_element = static_cast<int64_t>(h[kDiagBadElement]);
  return PDFX_OK;
}

int pdfx_reset_diag(void* ctx, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  const cudaStream_t s = as_stream(stream);
  PDFX_CUDA(cudaMemsetAsync(c->diag, 0, sizeof(unsigned long long) * kDiagCount, s));
  PDFX_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), s));
  c->steps_done = 0;
  return PDFX_OK;
}

int pdfx_check(void* ctx, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  int err = 0;
  const cudaStream_t s = as_stream(stream);
  PDFX_CUDA(cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PDFX_CUDA(cudaStreamSynchronize(s));
  return err;
}

int pdfx_set_profiling(void* ctx, int on) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  c->profiling = on != 0;
  return PDFX_OK;
}

int pdfx_stage_times(void* ctx, double* ms, int64_t* launches, int n, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c) return PDFX_ERR_ARG;
  PDFX_CUDA(cudaStreamSynchronize(as_stream(stream)));
  collect_times(*c);
  for (int i = 0; i < n && i < Ctx::kStages; ++i) {
    if (ms) ms[i] = c->stage_ms[i];
    if (launches) launches[i] = c->stage_n[i];
  }
  for (int i = 0; i < Ctx::kStages; ++i) { c->stage_ms[i] = 0; c->stage_n[i] = 0; }
  return Ctx::kStages;
}

int64_t pdfx_kernel_launches(const void* ctx) {
  const Ctx* c = static_cast<const Ctx*>(ctx);
  return c ? c->launches : 0;
}

int pdfx_wp_rhs(void* ctx, double* rhs, double* L, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !rhs || !L) return PDFX_ERR_ARG;
  PDFX_TRY(eulerian_ready(c, true));
  const cudaStream_t s = as_stream(stream);
  const EWork w = ework(*c);
  PDFX_TRY(c->prm.precision == 1 ? wp_rhs_dev<float>(*c, w, s) : wp_rhs_dev<double>(*c, w, s));
  PDFX_TRY(download_9(w.rhs, rhs, c->nn, s));
  return download_n(w.L, L, static_cast<size_t>(c->nn), s);
}

int pdfx_wp_solve(void* ctx, const double* rhs, const double* L, double* wp, double tol, int32_t max_iter,
                  int32_t* iters, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !rhs || !L || !wp || !solve_args_ok(tol, max_iter)) return PDFX_ERR_ARG;
  PDFX_TRY(eulerian_ready(c, true));
  const cudaStream_t s = as_stream(stream);
  const EWork w = ework(*c);
  PDFX_TRY(upload_9(rhs, w.rhs, c->nn, s));
  PDFX_TRY(upload_9(wp, w.x, c->nn, s));
  PDFX_TRY(upload_n(L, w.L, static_cast<size_t>(c->nn), s));
  PDFX_TRY(c->prm.precision == 1 ? wp_solve_dev<float>(*c, w, tol, max_iter, iters, s)
                                 : wp_solve_dev<double>(*c, w, tol, max_iter, iters, s));
  return download_9(w.x, wp, c->nn, s);
}

int pdfx_update_wp(void* ctx, double tol, int32_t max_iter, int32_t* iters, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !solve_args_ok(tol, max_iter)) return PDFX_ERR_ARG;
  PDFX_TRY(eulerian_ready(c, true));
  const cudaStream_t s = as_stream(stream);
  const EWork w = ework(*c);
  drop_graph(*c);
  return c->prm.precision == 1 ? update_wp_dev<float>(*c, w, tol, max_iter, iters, s)
                               : update_wp_dev<double>(*c, w, tol, max_iter, iters, s);
}

int pdfx_pressure_rhs(void* ctx, const double* ustar, const double* P, double dt, double Cp, double* src,
                      double* flux, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !ustar || !P || !src || !flux || !(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(Cp))
    return PDFX_ERR_ARG;
  PDFX_TRY(eulerian_ready(c, true));
  const cudaStream_t s = as_stream(stream);
  const EWork w = ework(*c);
  const size_t nn = static_cast<size_t>(c->nn);
  PDFX_TRY(upload_n(ustar, w.q, 3 * nn, s));
  PDFX_TRY(upload_n(P, w.r, nn, s));
  if (c->prm.precision == 1)
    launch_pressure_rhs<float>(c->fem, c->ne_off, c->ne_list, w.q, 3, 0, w.r,
                               static_cast<const float*>(c->fields), c->prm.nu, dt, Cp, w.prs, w.src, w.flux, s);
  else
    launch_pressure_rhs<double>(c->fem, c->ne_off, c->ne_list, w.q, 3, 0, w.r,
                                static_cast<const double*>(c->fields), c->prm.nu, dt, Cp, w.prs, w.src, w.flux, s);
  c->launches += 7;
  PDFX_TRY(cerr(cudaGetLastError()));
  PDFX_TRY(download_n(w.src, src, nn, s));
  return download_n(w.flux, flux, nn, s);
}

int pdfx_pressure_solve(void* ctx, const double* src, const double* flux, double* dP, double tol,
                        int32_t max_iter, int32_t* iters, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !src || !flux || !dP || !solve_args_ok(tol, max_iter)) return PDFX_ERR_ARG;
  PDFX_TRY(eulerian_ready(c, false));
  const cudaStream_t s = as_stream(stream);
  const EWork w = ework(*c);
  const size_t nn = static_cast<size_t>(c->nn);
  PDFX_TRY(upload_n(src, w.src, nn, s));
  PDFX_TRY(upload_n(flux, w.flux, nn, s));
  PDFX_TRY(upload_n(dP, w.x, nn, s));
  PDFX_TRY(pressure_dev(*c, w, w.x, tol, max_iter, iters, s));
  return download_n(w.x, dP, nn, s);
}

int pdfx_set_pressure(void* ctx, const double* P, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || !P) return PDFX_ERR_ARG;
  PDFX_TRY(eulerian_ready(c, false));
  const cudaStream_t s = as_stream(stream);
  PDFX_TRY(upload_n(P, c->P, static_cast<size_t>(c->nn), s));
  PDFX_CUDA(cudaMemsetAsync(c->dP, 0, sizeof(double) * c->nn, s));
  return cerr(cudaStreamSynchronize(s));
}

int pdfx_get_pressure(void* ctx, double* P, double* dP, void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || (!P && !dP)) return PDFX_ERR_ARG;
  PDFX_TRY(eulerian_ready(c, false));
  const cudaStream_t s = as_stream(stream);
  if (P) PDFX_TRY(download_n(c->P, P, static_cast<size_t>(c->nn), s));
  if (dP) PDFX_TRY(download_n(c->dP, dP, static_cast<size_t>(c->nn), s));
  return PDFX_OK;
}

int pdfx_coupled_step(void* ctx, double dt, double Cp, double tol, int32_t max_iter, int32_t* iters,
                      void* stream) {
  Ctx* c = as_ctx(ctx);
  if (!c || std::isnan(dt) || !std::isfinite(Cp) || !solve_args_ok(tol, max_iter)) return PDFX_ERR_ARG;
  if (!model_fits_grid(*c)) return PDFX_ERR_ARG;
  if (!c->pbuf[0] || !c->have_fields) return PDFX_ERR_ORDER;
  PDFX_TRY(eulerian_ready(c, true));
  const cudaStream_t s = as_stream(stream);
  if (!(dt > 0.0)) PDFX_TRY(cfl_dt(*c, s, &dt));
  return c->prm.precision == 1 ? do_coupled_step<float>(*c, dt, Cp, tol, max_iter, iters, s)
                               : do_coupled_step<double>(*c, dt, Cp, tol, max_iter, iters, s);
}

const char* pdfx_strerror(int code) {
  switch (code) {
    case PDFX_OK: return "ok";
    case PDFX_ERR_ARG: return "invalid argument";
    case PDFX_ERR_MESH: return "invalid grid";
    case PDFX_ERR_ORDER: return "call made before the state it needs exists";
    case PDFX_ERR_CUDA: return "CUDA runtime error";
    case PDFX_ERR_ALLOC: return "device allocation failed";
    case PDFX_ERR_LOST_PARTICLE: return "a particle was found in no element";
    case PDFX_ERR_CAPACITY: return "an element exceeded the per-element capacity";
    case PDFX_ERR_NONFINITE: return "a particle state became non-finite";
    case PDFX_ERR_SOLVE: return "an iterative solve did not converge within its iteration limit";
    case PDFX_ERR_ELEMENT: return "a particle's element id lies outside the grid";
    default: return "unknown error";
  }
}

}  // extern "C"
