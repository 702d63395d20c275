// Host-side context of one pdfx instance and the kernel launch interface.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pdfx.h"
#include "eulerian_ops.h"
#include "pdfx_device.cuh"

namespace pdfx {

// Model constants in the working precision, passed by value to the advance kernel.
template <typename T>
struct Model {
  T C1, C2, C3, C4, CT, Cw1, Cw2, nu, C0, Cs, Ct, Cphi, src_x, src_y, src_r, period_x;
  T src_xl, src_yl;  // FP32 form: the source centre's trailing parts (hi + lo pairs)
  T nuCT2;      // nu C_T^2 (Eq. 18)
  T s2nu;       // sqrt(2 nu) (Eqs. 7, 27)
  T cs_r2;      // C_s r0^(2/3) (Eq. 25)
  int c0_mode, tm_mode, interp_mode, source_on;
  int model;    // 0 full model; 1 Eqs. 46-47
  T alpha;      // Eq. 47
};

// One instance of a batch (a grid of the union, its particles and its parameters).  A
// context without instances is a batch of one.
template <typename T>
struct InstDev {
  Model<T> m;
  uint32_t k0, k1;       // Philox key (seed, instance)
  int32_t e0, e1;        // element range in the union grid
  int64_t p0, np;        // particle slot range
  int32_t ppe, minnpel;
};

// Particle storage (structure of arrays) in the working precision.  The FP32 form holds the
// position as hi + lo pairs: x, y the leading parts, xl, yl the trailing ones (nullptr in
// the FP64 form).
template <typename T>
struct Particles {
  T *x = nullptr, *y = nullptr, *u = nullptr, *v = nullptr, *w = nullptr, *om = nullptr,
    *psi = nullptr;
  uint32_t* pid = nullptr;
  int32_t* elem = nullptr;
  uint8_t* cp = nullptr;
  T *xl = nullptr, *yl = nullptr;
};

__device__ __forceinline__ Pos<double> load_pos(const Particles<double>& p, int64_t i) {
  return {p.x[i], p.y[i]};
}
__device__ __forceinline__ Pos<float> load_pos(const Particles<float>& p, int64_t i) {
  return {p.x[i], p.xl[i], p.y[i], p.yl[i]};
}
__device__ __forceinline__ void store_pos(const Particles<double>& p, int64_t i, const Pos<double>& P) {
  p.x[i] = P.x;
  p.y[i] = P.y;
}
__device__ __forceinline__ void store_pos(const Particles<float>& p, int64_t i, const Pos<float>& P) {
  p.x[i] = P.xh;
  p.xl[i] = P.xl;
  p.y[i] = P.yh;
  p.yl[i] = P.yl;
}

// Arguments of the advance kernel (Eqs. 7, 27, 19, 24; Sect. 3.8; Sect. 3.6).
template <typename T>
struct AdvanceArgs {
  Particles<T> p;
  int64_t np;
  const ElemGeo<T>* geo;
  const ElemTopo* topo;
  const Line<T>* walls;
  const int32_t* wall2;    // [ne] second no-slip line of the element (a corner), -1 none
  const Line<T>* fslines;
  const Line<T>* fsedges;  // lines of the free-slip boundary edges (topology -2 - j)
  const int32_t* ne_off;
  const int32_t* ne_list;
  int32_t ne;
  const T* fields;
  const double* vcce;
  int G;
  const double* nmom;      // [nn][13] nodal statistics of the previous pass (model 1)
  int32_t* cnt;
  unsigned long long* diag;
  int* err;
  int32_t* brute_list;   // slots that need the brute-force search
  int* brute_count;
  int brute_cap;
  double* lost_rec;      // [kLostRecords][4]
  Model<T> m;
  T dt, sdt;    // time step and its square root
  const uint32_t* stepc;   // step counter (Philox counter word) in device memory
  const double* corr;      // [ne][2] Eq. 31 correction of the last coupled step still to be
                           // applied to the velocities as they are read (nullptr: none)
  uint32_t k0, k1;
  // batches: per-instance parameters (m, k0, k1 above are unused) and element -> instance
  const InstDev<T>* inst;
  const int32_t* einst;
};

// Arguments of the statistics / conditional-mean kernels.
template <typename T>
struct StatsArgs {
  Particles<T> p;       // current state
  Particles<T> out;     // re-ordered state (written when resort != 0)
  int resort;
  const int32_t* cnt;   // particles per element after advance (list segment sizes)
  const int32_t* off;   // list offsets
  const int32_t* idx;   // element lists of particle slots (-1 = moved out)
  const int32_t* fin;   // final counts after redistribution
  const int32_t* foff;  // exclusive scan of fin
  const int32_t* gain;  // particles received per element
  const int32_t* goff;  // offsets into movers of received particles
  const int32_t* movers;
  const int32_t* big_list;
  const int32_t* tiles;  // tile-class element lists (scal 6 from the front, scal 7 from the back)
  const int32_t* tiles_mid;  // the middle tile class (scal 8 from the front)
  const int32_t* einst;  // element -> instance (nullptr: one instance)
  const int32_t* ielem;  // [K + 1] first element of each instance
  int K;                 // instances (plan scalars scal[16 k ...] per instance)
  const int32_t* scal;  // plan scalars: 0 moves, 3 number of large elements
  int32_t ne;
  int64_t np;
  int bins[3];
  int min_per_bin;
  int G;
  double* emom;
  double* vcce;
  int32_t* gbin;
  uint32_t* step_inc;    // stepping: the step counter, advanced once after this step's reads
  int acc64;             // FP32 form: accumulate moments and conditional means in FP64
  int prior;             // emom holds the previous statistics pass of the same grid (the
                         // binning takes its bucket scales from them; results do not depend
                         // on it)
  int cond_mode;         // 0 hierarchical bins (Sect. 3.5); 1 Fox's projection (Eqs. 64-66)
  int fox_bins;          // intervals of the projected velocity (cond_mode 1)
  unsigned long long* diag;
  int* err;
};

// Scratch of the statistics pipeline (device).
struct Plan {
  int32_t* cnt = nullptr;      // [ne]
  int32_t* off = nullptr;      // [ne + 1]
  int32_t* cursor = nullptr;   // [ne]
  int32_t* fin = nullptr;      // [ne]
  int32_t* foff = nullptr;     // [ne + 1]
  int32_t* gain = nullptr;     // [ne]
  int32_t* goff = nullptr;     // [ne + 1]
  int32_t* loss = nullptr;     // [ne]
  int32_t* doff = nullptr;     // [ne + 1]
  int32_t* recips = nullptr;   // [ne] elements that receive
  int32_t* donors = nullptr;   // [ne] elements that give
  int32_t* big_list = nullptr; // [ne] elements above the small binning capacity
  int32_t* tiles = nullptr;    // [ne] elements of up to kTileSplit particles from the front,
                               // kTileMid + 1 .. kSmallCap from the back
  int32_t* tiles_mid = nullptr;  // [ne] elements of kTileSplit + 1 .. kTileMid particles
  int32_t* scal = nullptr;     // [16 K]: per instance 0 T, 1 n_recips, 2 n_donors, 3 n_big,
                               // 4 min, 5 max, 6 / 7 / 8 tile-class counts (front, back,
                               // middle); lists of instance k
                               // live in its element range, its moves in its slot range
  const int32_t* ielem = nullptr;    // [K + 1] first element of each instance (nullptr: one)
  const int64_t* ip0 = nullptr;      // [K + 1] first particle slot of each instance
  const int32_t* iminnpel = nullptr; // [K] MINNPEL of each instance
  int64_t* hist = nullptr;     // [K][2 (kHistCap + 1)] prefix sums for the closed form
  int32_t* idx = nullptr;      // [np] element lists
  int32_t* movers = nullptr;   // [np] particle slots that move (by move index)
  int32_t* mrecip = nullptr;   // [np] recipient element per move
  double* mvals = nullptr;     // [np][7] new values per move
  int tile_split = 256;        // elements of up to this many particles take the tile of
                               // kTileSplit (bucket ranks; chunk sorts for Fox's
                               // projection); larger ones up to kTileMid the tile of kTileMid
};

constexpr int kHistCap = 8192;      // counts above this are clipped for the closed form
constexpr int kSmallCap = 768;      // binning capacity of the block-per-element tile kernels
constexpr int kTileBig = 1024;      // the large-element list's entries up to this size take a bucket-rank tile
constexpr int kTileSplit = 256;     // tile classes: up to the split, at most 256 particles,
constexpr int kTileMid = 512;       // 257 .. 512 and 513 .. kSmallCap (bucket-rank tiles)
constexpr int64_t kMaxParticles = int64_t(1) << 28;   // particle ids fit the 28-bit sort key field
constexpr int64_t kMaxSlots = (int64_t(1) << 31) - 1;  // particle slots of a batch (int32 lists)
constexpr int kBigCap = 4096;       // binning capacity of the large-element kernel

// Eulerian solves of the coupled loop (k_eulerian.cu), FP64.
// Galerkin FEM data of a grid with linear triangles (Sect. 3.2), built on the host once.
struct FemDev {
  int32_t nn = 0, ne = 0, nnz = 0;
  int32_t* row = nullptr;    // [nn + 1] CSR rows: each node's neighbours and itself
  int32_t* col = nullptr;    // [nnz] ascending within a row
  int32_t* dpos = nullptr;   // [nn] position of each row's diagonal entry
  int32_t* cptr = nullptr;   // [nnz + 1] element contributions of each entry
  int32_t* clist = nullptr;  // [9 ne] 9 e + 3 a + b (local row a, column b), ascending e
  int32_t* tri = nullptr;    // [ne][3]
  double* fe = nullptr;      // [ne][7] dN/dx (3), dN/dy (3), area (Eq. 40, element frame)
  double* mval = nullptr;    // [nnz] consistent mass matrix
  double* kval = nullptr;    // [nnz] stiffness of the laplacian
  double* kdiag = nullptr;   // [nn] its diagonal
  double* mlump = nullptr;   // [nn] integral of each shapefunction
  double area = 0.0;         // domain area
  int8_t* ncls = nullptr;    // [nn] 0 interior, 1 no-slip, 2 free-slip (no-slip wins)
  double* nrm = nullptr;     // [nn][2] outward unit normal of no-slip nodes (corner: bisector)
  int32_t* boff = nullptr;   // [nn + 1] no-slip edges at each node
  int32_t* bnb = nullptr;    // [.] the edge's other node
  double* blen = nullptr;    // [.] the edge's length
  double cxi = 1.0;
};
// Jacobi-PCG over C systems sharing one matrix; vectors [C][nn].
struct PcgArgs {
  int C = 1;
  const double* val = nullptr;     // [nnz]
  const double* diag = nullptr;    // [nn]
  const uint8_t* fixed = nullptr;  // [C][nn] Dirichlet mask (NULL: none)
  const double* b = nullptr;       // [C][nn] load
  double* x = nullptr;             // [C][nn] initial guess (Dirichlet values set) in, solution out
  double* r = nullptr;
  double* z = nullptr;
  double* d = nullptr;
  double* q = nullptr;
  double* d2 = nullptr;            // [C][nn] the second direction buffer (two-kernel iterations)
  unsigned* ticket = nullptr;      // [C] zeroed counters of the last-block reductions
  double* scratch = nullptr;       // pcg_scratch_doubles(nn, C)
  double tol = 0.0;
};
constexpr int kPcgScalars = eops::kPcgScalars;   // per component: rz, |b|, zz, alpha, beta, active, iterations
constexpr int kRedBlocks = 256;                  // blocks of the solvers' reduction passes, at most
constexpr int kPcgActive = eops::S_ACTIVE;
constexpr int kPcgIters = eops::S_ITERS;

// Two streams and three events for the statistics tiles' size classes, which are independent
// (disjoint elements and outputs) and run as parallel branches of the step: fork after the
// lists, join before the large-element kernel.  Captured into a graph they become parallel
// nodes.  Created with the context, outside any capture; ok is false when creation failed
// (the classes then run one after another on the caller's stream).
struct SideStreams {
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool ok = false;
};

struct Ctx {
  pdfx_params prm{};
  pdfx_allocator alloc{};
  bool has_alloc = false;
  int device = 0;
  int num_sms = 0;
  // grid
  int32_t nn = 0, ne = 0;
  void* geo = nullptr;          // ElemGeo<T>[ne]
  ElemTopo* topo = nullptr;     // [ne]
  int32_t* wall2 = nullptr;     // [ne] second no-slip line index (-1 none)
  void* walls = nullptr;        // Line<T>[n_walls]
  void* fsedges = nullptr;      // Line<T>[]: each free-slip boundary edge's own line
  int n_wall_lines = 0;         // no-slip wall lines of the grid
  double min_sqrt_an = 0.0;     // min over nodes of sqrt(mean area of the elements around it)
  double last_dt = 0.0;         // the time step of the last step
  double* dnorm = nullptr;      // device scalar: max nodal ||<Z>|| (Eq. 26)
  void* fslines = nullptr;      // Line<T>[n_fs]
  int32_t* ne_off = nullptr;    // [nn + 1]
  int32_t* ne_list = nullptr;   // [3 ne]
  std::vector<int32_t> h_ne_off, h_ne_list;
  bool have_grid = false;
  // fields
  void* fields = nullptr;       // T[nn][32]
  double* fields64 = nullptr;   // staging for the FP32 conversion
  bool have_fields = false;
  // particles (double buffered for re-ordering)
  int64_t np = 0;
  int cur = 0;
  void* pbuf[2] = {nullptr, nullptr};  // one allocation per buffer
  size_t pbuf_bytes = 0;
  uint32_t step = 0;             // host mirror of the device step counter
  int steps_since_sort = 0;
  uint32_t* dstep = nullptr;     // device step counter (read by the kernels of a step)
  // CUDA graph of a cycle of steps (2 sort_every steps, so the buffer roles repeat)
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  SideStreams side;               // branches of the statistics tiles
  double g_dt = 0.0;
  int g_steps = 0;
  const void* g_buf = nullptr;
  int64_t g_np = -1;
  int64_t g_launches = 0;
  // launch shapes (pdfx_autotune)
  int adv_block = 256;
  int tile_split = kTileSplit;  // the binning's size-class split (Plan::tile_split)
  // instances of a batch (K = 1: the whole grid)
  int K = 1;
  std::vector<pdfx_params> iprm;        // [K] parameters (K > 1 only)
  std::vector<int32_t> h_ielem;         // [K + 1]
  std::vector<int64_t> h_ip0;           // [K + 1]
  std::vector<int32_t> h_ippe;          // [K]
  std::vector<int32_t> h_nb;            // [3 ne] neighbours (host copy for batch checks)
  int32_t* einst = nullptr;             // [ne] (K > 1 only)
  int32_t* ielem = nullptr;             // [K + 1]
  int64_t* ip0 = nullptr;               // [K + 1]
  int32_t* iminnpel = nullptr;          // [K]
  void* inst = nullptr;                 // InstDev<T>[K]
  int inst_cap = 0;                     // capacity of the instance tables
  // statistics
  Plan plan;
  double* emom = nullptr;       // [ne][13]
  double* nmom = nullptr;       // [nn][13]
  double* vcce = nullptr;       // [ne][G]
  int32_t* gbin = nullptr;      // [ne][3]
  int G = 1;
  // diagnostics
  unsigned long long* diag = nullptr;  // [kDiagCount]
  int* err = nullptr;                  // [0] error word, [1] brute-force list length
  int32_t* brute_list = nullptr;       // [kBruteCap]
  double* lost_rec = nullptr;          // [kLostRecords][4]
  int64_t steps_done = 0;
  int64_t launches = 0;
  // profiling
  bool profiling = false;
  static constexpr int kStages = 6;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double stage_ms[kStages] = {0};
  int64_t stage_n[kStages] = {0};
  // Eulerian solves of the coupled loop: host copies of the grid, the FEM data (built on
  // the first Eulerian call after pdfx_set_grid) and their device work arrays
  std::vector<int32_t> h_tri;
  std::vector<int8_t> h_tag;
  std::vector<double> h_vx, h_vy, h_area2;   // [ne][3] vertices unwrapped toward vertex A
  FemDev fem;
  bool fem_ready = false;
  double* ew = nullptr;         // work: 7 [9][nn] vectors, rhs, L, matrix, scratch
  uint8_t* efixed = nullptr;    // [9][nn] Dirichlet masks
  int* eflag = nullptr;         // [1] eps <= 0 at a node
  double* P = nullptr;          // [nn] nodal mean pressure (rho = 1)
  double* corr = nullptr;       // [ne][2] Eq. 31: dt grad(dP) per element of the last coupled step
  // conjugate-gradient iterations replayed from CUDA graphs (16 iterations each), one per
  // solve configuration (components, arrays, tolerance)
  struct PcgGraph {
    cudaGraphExec_t exec = nullptr;
    int C = 0;
    const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
    double tol = 0.0;
  };
  PcgGraph pcg_graphs[4];
  bool corr_pending = false;    // corr not yet applied to the particles (the next advance does)
  double* dP = nullptr;         // [nn] last pressure increment (the next initial guess)
  // allocations to release
  std::vector<std::pair<void*, size_t>> owned;
};

template <typename T>
Particles<T> particles_of(Ctx& c, int which);

// Kernel attributes are per device: a flag per device records that a kernel's attributes
// were set on it (setting them twice from racing host threads is harmless).  True on the
// first call for the current device (and whenever the device cannot be told).
constexpr int kMaxDevices = 64;
inline bool first_use_on_device(bool (&flags)[kMaxDevices]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return true;
  if (flags[dev]) return false;
  flags[dev] = true;
  return true;
}

// Kernel launchers (defined in the .cu files).
template <typename T>
void launch_advance(const AdvanceArgs<T>& a, int num_sms, int block, cudaStream_t s);   // block <= 256
template <typename T>
void launch_init(Particles<T> p, int32_t ne, int32_t ppe, const ElemGeo<T>* geo,
                 const ElemTopo* topo, const T* fields, Model<T> m, uint32_t k0, uint32_t k1,
                 unsigned long long* diag, cudaStream_t s);
// Batches: every instance k gets ppe_k particles per element in slots [p0_k, p0_k + np_k).
template <typename T>
void launch_init_batch(Particles<T> p, int64_t np, int K, const InstDev<T>* inst,
                       const int64_t* ip0, const ElemGeo<T>* geo, const ElemTopo* topo,
                       const T* fields, unsigned long long* diag, cudaStream_t s);
// Counts per element; ids outside 0 .. ne - 1 are skipped, counted and raise PDFX_ERR_ELEMENT.
void launch_count(const int32_t* elem, int64_t np, int32_t ne, int32_t* cnt, unsigned long long* diag,
                  int* err, cudaStream_t s);
int launch_plan(Plan& pl, int32_t ne, int K, int minnpel, int allow_moves, cudaStream_t s);   // kernels launched
// Element lists (ids outside 0 .. ne - 1 are skipped; launch_count reports them).
void launch_scatter(const int32_t* elem, int64_t np, int32_t ne, Plan& pl, cudaStream_t s);
template <typename T>
void launch_redistribute(Particles<T> p, Plan& pl, int K, const InstDev<T>* inst, int32_t ne,
                         int64_t np, const ElemGeo<T>* geo, const ElemTopo* topo, const uint32_t* stepc,
                         int num_sms, unsigned long long* diag, int* err, cudaStream_t s);
template <typename T>
void launch_stats(const StatsArgs<T>& a, int num_sms, cudaStream_t s, const SideStreams* side);
// The tile classes of up to 256, 257..512 and 513..768 particles on s_small, s_mid and
// s_large (k_bins_f32.cu / k_bins_f64.cu).
template <typename T>
void launch_stats_tiles(const StatsArgs<T>& a, int num_sms, cudaStream_t s_small, cudaStream_t s_mid,
                        cudaStream_t s_large);
void launch_node_average(const double* emom, const int32_t* ne_off, const int32_t* ne_list,
                         int32_t nn, double* nmom, cudaStream_t s);
// Eq. 26: max over nodes of ||(<U>, <V>, <W>, <omega>, <psi>)||_2 into out[0] (one block).
void launch_cfl_norm(const double* nmom, int32_t nn, double* out, cudaStream_t s);
// Eq. 31 (rho = 1): U -= dt grad(dP) with the element-constant gradient of the nodal dP[nn];
// egrad is scratch of 2 ne doubles.
template <typename T>
void launch_correct_velocity(const ElemGeo<T>* geo, const ElemTopo* topo, int32_t ne, double period_x,
                             const int32_t* einst, const InstDev<T>* inst, const double* dp,
                             double* egrad, Particles<T> p, int64_t np, double dt, cudaStream_t s);
// The same in parts: corr[ne][2] = dt grad(dP) per element; U -= corr on each particle;
// the element means of U and V shifted by corr (elements that hold particles).
template <typename T>
void launch_correction_field(const ElemGeo<T>* geo, const ElemTopo* topo, int32_t ne, double period_x,
                             const int32_t* einst, const InstDev<T>* inst, const double* dp, double dt,
                             double* corr, cudaStream_t s);
template <typename T>
void launch_apply_correction(Particles<T> p, int64_t np, const double* corr, cudaStream_t s);
void launch_shift_means(int32_t ne, const double* corr, double* emom, cudaStream_t s);
// Sect. 3.4: the nodal fields the statistics provide (slots 0-2, 5-13, 23-29) from nmom;
// scratch holds 18 (ne + nn) doubles.
template <typename T>
void launch_derive_fields(const ElemGeo<T>* geo, const ElemTopo* topo, int32_t ne, double period_x,
                          const int32_t* einst, const InstDev<T>* inst, const int32_t* ne_off,
                          const int32_t* ne_list, int32_t nn, const double* nmom, double* scratch,
                          T* fields, cudaStream_t s);

// Eulerian solves of the coupled loop (k_eulerian.cu): launchers.
int pcg_blocks(int nn);
size_t pcg_scratch_doubles(int nn, int C);
const double* pcg_scalars(const PcgArgs& a, int nn);   // [C][kPcgScalars], device
template <typename T>
void launch_wp_rhs(const T* fields, int nn, const WpConst& k, double* rhs, double* L, int* err, cudaStream_t s);
template <typename T>
void launch_read_wp(int nn, const T* fields, double* x, cudaStream_t s);
template <typename T>
void launch_wp_bc(const T* fields, int nn, const WpConst& k, const int8_t* ncls, const double* nrm,
                  uint8_t* fixed, double* x, int* err, cudaStream_t s);
void launch_assemble_wp(const FemDev& m, const double* L, double* aval, double* adiag, cudaStream_t s);
void launch_spmv(const FemDev& m, const double* val, int C, const double* x, double* y, cudaStream_t s);
void launch_pcg_setup(const FemDev& m, const PcgArgs& a, cudaStream_t s);
void launch_pcg_iteration(const FemDev& m, const PcgArgs& a, cudaStream_t s);
void launch_pcg_two_iterations(const FemDev& m, const PcgArgs& a, cudaStream_t s);
void launch_node_gradients(const FemDev& m, const int32_t* ne_off, const int32_t* ne_list, int nq,
                           const double* q, double* eg, double* gn, cudaStream_t s);
size_t pressure_rhs_scratch_doubles(int nn, int ne);
template <typename T>
void launch_pressure_rhs(const FemDev& m, const int32_t* ne_off, const int32_t* ne_list, const double* ustar,
                         int ustride, int uoff, const double* P, const T* fields, double nu, double dt,
                         double Cp, double* work, double* src, double* flux, cudaStream_t s);
void launch_pressure_load(const FemDev& m, const double* src, const double* flux, double* b, double* red,
                          cudaStream_t s);
void launch_zero_mean(const FemDev& m, double* x, double* red, cudaStream_t s);
template <typename T>
void launch_write_wp(int nn, const double* x, T* fields, cudaStream_t s);
template <typename T>
void launch_write_pgrad(const FemDev& m, const int32_t* ne_off, const int32_t* ne_list, const double* P,
                        double* eg, double* gp, T* fields, cudaStream_t s);
void launch_add(int nn, const double* a, double* b, cudaStream_t s);

// Accumulators of the scalar statistics of n probe elements over nb psi bins (fixed-point
// sums in two's complement; lo and hi hold order-preserving images of doubles).
struct ScalarAcc {
  int32_t* count;              // [n][nb] particles per bin
  unsigned long long* sc;      // [n][nb] sums of <phi|V>
  unsigned long long* sd;      // [n][nb] sums of psi - <phi|V>
  int32_t* n;                  // [n] particles per element
  unsigned long long* s1;      // [n] sums of psi
  unsigned long long* m;       // [n][3] sums of (psi - <phi>)^2, ^3, ^4
  unsigned long long* lo;      // [n] minimum of psi
  unsigned long long* hi;      // [n] maximum of psi
};
struct ScalarOut {
  int32_t* count;              // [n][nb]
  double* phit;                // [n][nb] Eq. 68
  double* cdiff;               // [n][nb] t_m <Gamma lap phi | psi>
  double* cdiss;               // [n][nb] t_m <2 Gamma (grad phi)^2 | psi>, Eq. 67
  double* mom;                 // [n][6] <phi>, <phi'^2>, <phi'^3>, <phi'^4>, min, max
};
// probe: [ne] index of the element among the probes, -1 for the others.
template <typename T>
void launch_scalar_stats(const Particles<T>& p, int64_t np, const int32_t* probe, const double* vcce,
                         int G, int n, int nb, const ScalarAcc& acc, const ScalarOut& out,
                         int num_sms, cudaStream_t s);   // k_scalar.cu
// Particle order of the caller's arrays: by (instance, id), i.e. index p0_k + id (einst and
// ip0 nullptr: one instance, index = id).
template <typename T>
void launch_gather_by_pid(Particles<T> p, int64_t np, const int32_t* einst, const int64_t* ip0,
                          double* x, double* y, double* u, double* v, double* w, double* om,
                          double* psi, int32_t* elem, uint8_t* cp, cudaStream_t s);
template <typename T>
void launch_load_state(Particles<T> p, int64_t np, const int32_t* einst, const int64_t* ip0,
                       const double* x, const double* y, const double* u, const double* v,
                       const double* w, const double* om, const double* psi, const int32_t* elem,
                       int32_t ne, unsigned long long* diag, int* err, cudaStream_t s);
void launch_convert_fields(const double* in, float* out, int64_t n, cudaStream_t s);
template <typename T>
void launch_check_finite(Particles<T> p, int64_t np, unsigned long long* diag, int* err,
                         cudaStream_t s);

}  // namespace pdfx
