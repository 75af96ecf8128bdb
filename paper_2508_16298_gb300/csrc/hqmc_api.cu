// C ABI of the HQMC library: configuration, workspace, argument checking and
// the host-side orchestration of the kernels (CG loop, force, leapfrog,
// trajectory).  Declarations and contracts are in include/hqmc.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>

#include "hqmc.h"
#include "kernels.h"
#include "multi_shape.h"

using namespace hqmc;

namespace {

// NVTX range over a scope (CG solve, force, leapfrog, trajectory, estimate), so
// that a profiler's timeline shows the path's phases; free when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxL = 68;             // 3 complex-double slices must fit in 227 KB of shared memory
constexpr int kBodyIters64 = 16;      // FP64 CG iterations per loop body
constexpr int kMaxMultiRhs = 1024;  // systems of one multi-system workspace (hqmc_set_multi_rhs)
constexpr int kDefaultReliable = 50;  // mixed solver residual-update period (iterations per body)
constexpr int kMaxBreakdowns = 8;     // mixed solver: FP32 breakdown restarts before the FP64 fallback
constexpr size_t kMaxLineSmem = 227 * 1024;  // tau-line preconditioner tile: opt-in shared memory per block
constexpr long long kFuseMaxSites = 2000000;  // fused preconditioned update by default up to this size
constexpr double kLineTruncation = 1e-3;  // entries of the factor's inverse below this are dropped (Methods)
constexpr size_t kMaxGraphs = 8;      // cached solve graphs per config

struct TimerClass {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs;
  size_t used = 0;
};

// An instantiated CG loop (WHILE node around one loop body) for fixed operands.
struct SolveGraph {
  const void* phi;
  void* x;
  int solver;
  long long net_version;  // flexible CG: the net weights captured by value in the body
  int body_kernels;  // kernels per body, including the loop-condition kernel
  cudaGraphExec_t exec;
};

// Systems solved together on one field (hqmc_set_multi_rhs): `cap` systems stored
// back to back, system k at offset k n of every vector, k pstride of part_w,
// part_ew and part_rz, k rstride of part_res, 2 k of report.
struct MultiWs {
  int cap = 0;
  int pstride = 0;  // doubles per system: walk partials (<= Ntau), update partials, preconditioner partials
  int rstride = 0;  // doubles per system of the FP64 residual partials (two sums per slot)
  int nlt = 0;      // preconditioner tiles per system
  int ublocks = 0;  // blocks per system of the batched update (= its partials of <r, r>)
  int rC = 1;       // cluster size (slices per tile) of the batched FP64 residual
  int rnt = 0;      // FP64 residual tiles per system
  int rslots = 0;   // FP64 residual partial slots per system (rnt rC)
  float2 *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr, *z = nullptr, *xh = nullptr;
  double2 *eta = nullptr, *xw = nullptr, *xiw = nullptr;  // estimate: R_k, X_k and xi_k when the caller keeps none
  double *part_w = nullptr, *part_ew = nullptr, *part_rz = nullptr, *part_res = nullptr, *report = nullptr;
  CgState* st = nullptr;
  CgState** d_states = nullptr;
  LineBatchDesc<float>* d_line = nullptr;
  int4* d_ltiles = nullptr;            // (system, bx, by) of the batched preconditioner
  MdagmArgs<double>* d_res = nullptr;  // per call: [0, cap) start residuals, [cap, 2 cap) reliable updates
  FinArgs* d_fin = nullptr;
  int2* d_rtiles = nullptr;            // (system, slice) of the FP64 residual
  CgState* st_h = nullptr;             // pinned mirrors
  double* report_h = nullptr;
  void* h_stage = nullptr;             // pinned staging of the per-call descriptors
  size_t stage_bytes = 0;
  std::vector<void*> allocs;           // device buffers above (freed when the workspace grows)
  struct Graph {
    int nsys, pc, granges;
    void* x;
    int body_kernels;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
};

}  // namespace

struct hqmc_config {
  hqmc_params p{};
  int device = 0;
  Geo g{};
  long long n = 0;  // sites
  double a = 0, t1 = 0, t2 = 0, cB = 0;
  BosonParams bp{};
  SliceLaunch sl{};    // fused M^dagger M in FP64
  SliceLaunch sl32{};  // fused M^dagger M in FP32 (same grid and clusters, own block shape)
  SliceLaunch slb64{}; // register-blocked fused M^dagger M, FP64 (nby = 0: not available)
  SliceLaunch slb32{}; // register-blocked fused M^dagger M, FP32 (nby = 0: not available)
  SliceLaunch slw32{}; // tau-walking fused M^dagger M, FP32 (walk = 0: not available)
  SliceLaunch slw32h[3]{};  // every strip height whose walk block fits (walk = 0: unused), for the autotuner
  int num_sms = 0;
  // tau-line preconditioner: coefficients from the pi-flux field, launch shape, workspace
  double pc_a = 0, pc_b = 0;
  LineCoef lc{};
  LineLaunch ll64{}, ll32{};    // separate tau-line preconditioner (FP32 tile height tuned per config)
  LineLaunch llu64{}, llu32{};  // fused update and preconditioner
  size_t smem_per_sm = 0;
  double2* z64 = nullptr;
  float2* z32 = nullptr;
  double2* r64b = nullptr;  // second residual buffers of the fused preconditioned update
  float2* r32b = nullptr;
  int fuse_pc64 = 1, fuse_pc32 = 1;  // preconditioned update fused with the preconditioner (autotuned;
                                     // default: fused below kFuseMaxSites, where it measured faster)
  double* part_rz = nullptr;
  SliceLaunch fused64{}, fused32{};  // shapes used for APPLY / CG direction (nby > 0: register-blocked)
  float tuned_us64 = 0.f, tuned_us32 = 0.f;  // autotuner: time of one FP64 / FP32 apply (0: not tuned)
  SliceLaunch sl1{};   // apply_M and force (one CTA per slice, no cluster)
  int ew_grid = 0;    // CG update grid (= number of <r,r> partials)
  int n_part_ew = 0;  // slots of part_ew: the update's or the fused preconditioned update's partials
  int act_grid = 0;
  int reliable = kDefaultReliable;

  // device workspace
  double2* U64 = nullptr;
  float2* U32 = nullptr;
  float2* th32 = nullptr;
  double2 *r64 = nullptr, *p64[2] = {nullptr, nullptr}, *q64 = nullptr;
  float2 *r32 = nullptr, *p32[2] = {nullptr, nullptr}, *q32 = nullptr, *xh32 = nullptr;
  double2 *eta = nullptr, *Xw = nullptr, *Rw = nullptr, *vscratch = nullptr;
  double *dSf = nullptr, *F = nullptr, *th0 = nullptr, *pm = nullptr;
  double *part_mdagm = nullptr, *part_ew = nullptr, *part_resid = nullptr, *part_act = nullptr;
  double *terms = nullptr, *report = nullptr;
  CgState* st = nullptr;
  int* dev_err = nullptr;    // device error word: 1 after a bounded device-side wait gave up
  int* dev_err_h = nullptr;  // its pinned host mirror (read with the CG state)
  // pinned host mirrors
  CgState* st_h = nullptr;
  double* terms_h = nullptr;
  double* report_h = nullptr;

  // learned preconditioner: attached net and its workspace (allocated when a net
  // is first attached with hqmc_set_preconditioner, kept until the config is freed)
  struct hqmc_net* net = nullptr;
  float2* net_h[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // activations (1, 16, 16, 16, 1 channels)
  float2* net_d[2] = {nullptr, nullptr};                               // back-propagated gradients (16 channels)
  double* net_part = nullptr;                                          // weight-gradient and loss partials
  float2* r_old32 = nullptr;                                           // flexible CG: residual before the update
  double *part_fz = nullptr, *part_fx = nullptr;                       // flexible CG: <r, z>, <r_old, z> partials
  int net_interval = 1;                                                // flexible CG: net on iterations c % k == 0
  int net_tc = 1;                                                      // inference 16 -> 16 layers on tensor cores
  // learned guess inside a leapfrog integration with the chronological guess:
  // consecutive tries that did not halve the residual, and whether the last solve tried it
  int net_adaptive = 0, net_rejects = 0, net_tried = 0;
  // chronological initial guess of leapfrog solves (hqmc_set_guess_history): the
  // last guess_k solutions of the current integration and an orthonormal basis
  double2* hist = nullptr;                                             // guess_k vectors, contiguous
  double2* qbasis = nullptr;                                           // guess_k vectors, contiguous
  int guess_k = 0, guess_cap = 0;                                      // in use, allocated
  int hist_n = 0, hist_next = 0;                                       // stored solutions, next ring slot
  double* net_scal = nullptr;                                          // device scalars (norms)

  MultiWs mw;  // systems solved together on one field (hqmc_set_multi_rhs)
  int multi_ranges = 0;  // slice ranges per system of their walk launch (0: the launch-time model)

  int timing = 0;
  long long launches = 0;  // kernels enqueued by this config
  int capturing = 0;       // inside a stream capture: launches are counted when the graph runs
  int graphs_ok = 1;       // cleared if this device cannot build the device-side CG loop
  cudaStream_t cap = nullptr;
  std::vector<SolveGraph> graphs;
  TimerClass timers[HQMC_TIMER_COUNT];
  std::vector<void*> allocs;
  char err[512] = {0};
};

namespace {

int fail(hqmc_config* cfg, int code, const char* fmt, ...) {
  if (cfg) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(cfg->err, sizeof(cfg->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(cfg, HQMC_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                        \
  } while (0)

#define RET(call)                 \
  do {                            \
    int rc_ = (call);             \
    if (rc_ != HQMC_OK) return rc_; \
  } while (0)

// Kernel launches are made through LK so that the config can report how many
// of its kernels it enqueued (launch_action_terms enqueues two).
#define LK(n, call)                          \
  do {                                       \
    if (!cfg->capturing) cfg->launches += (n); \
    CK(call);                                \
  } while (0)

bool aligned16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

template <class T>
int dalloc(hqmc_config* cfg, T** ptr, size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(cfg, HQMC_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  cfg->allocs.push_back(p);
  *ptr = (T*)p;
  return HQMC_OK;
}

void multi_release(MultiWs& m) {
  for (auto& g : m.graphs) cudaGraphExecDestroy(g.exec);
  m.graphs.clear();
  for (void* p : m.allocs) cudaFree(p);
  m.allocs.clear();
  if (m.st_h) cudaFreeHost(m.st_h);
  if (m.report_h) cudaFreeHost(m.report_h);
  if (m.h_stage) cudaFreeHost(m.h_stage);
  m = MultiWs{};
}

void release(hqmc_config* cfg) {
  multi_release(cfg->mw);
  for (void* p : cfg->allocs) cudaFree(p);
  cfg->allocs.clear();
  if (cfg->st_h) cudaFreeHost(cfg->st_h);
  if (cfg->terms_h) cudaFreeHost(cfg->terms_h);
  if (cfg->report_h) cudaFreeHost(cfg->report_h);
  if (cfg->dev_err_h) cudaFreeHost(cfg->dev_err_h);
  for (auto& tc : cfg->timers)
    for (auto& pr : tc.pairs) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto& g : cfg->graphs) cudaGraphExecDestroy(g.exec);
  cfg->graphs.clear();
  if (cfg->cap) cudaStreamDestroy(cfg->cap);
  cfg->cap = nullptr;
}

// Event timing around launches of one kernel class.
int timer_begin(hqmc_config* cfg, int cls, cudaStream_t s, int* slot) {
  *slot = -1;
  if (!cfg->timing || cfg->capturing) return HQMC_OK;
  TimerClass& tc = cfg->timers[cls];
  if (tc.used == tc.pairs.size()) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    tc.pairs.emplace_back(a, b);
  }
  *slot = (int)tc.used++;
  CK(cudaEventRecord(tc.pairs[*slot].first, s));
  return HQMC_OK;
}

int timer_end(hqmc_config* cfg, int cls, cudaStream_t s, int slot) {
  if (slot < 0) return HQMC_OK;
  CK(cudaEventRecord(cfg->timers[cls].pairs[slot].second, s));
  return HQMC_OK;
}

int check_device(hqmc_config* cfg) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != cfg->device)
    return fail(cfg, HQMC_EINVAL, "config belongs to device %d but device %d is current", cfg->device, dev);
  return HQMC_OK;
}

// Per-gauge-field tables: the FP64 link table, and for FP32 either the float
// link table (generic kernel) or theta as float (register-blocked kernel).
// need32: tables for the FP32 fused kernel; table32: the float link table itself
// (the FP32 apply of M reads it whatever the fused kernel uses).
int links(hqmc_config* cfg, const double* theta, bool need64, bool need32, cudaStream_t s, bool table32 = false,
          bool theta32 = false) {
  const bool blk32 = need32 && cfg->fused32.nby > 0;
  LK(1, launch_links(cfg->g, theta, cfg->t1, cfg->t2, need64 ? cfg->U64 : nullptr,
                     ((need32 && !blk32) || table32) ? cfg->U32 : nullptr, (blk32 || theta32) ? cfg->th32 : nullptr, s));
  return HQMC_OK;
}

// Fused M^dagger M launch in the kernel variant chosen for this precision.
template <class R>
const SliceLaunch& fused_shape(const hqmc_config* cfg) {
  return sizeof(R) == 8 ? cfg->fused64 : cfg->fused32;
}

template <class R, int MODE>
cudaError_t launch_shape(const SliceLaunch& sh, const MdagmArgs<R>& a, cudaStream_t s) {
  if constexpr (sizeof(R) == 4) {
    if (sh.walk) return launch_mdagm_walk<MODE>(sh, a, s);
  }
  if (sh.nby > 0) return launch_mdagm_block<R, MODE>(sh, a, s);
  return launch_mdagm<R, MODE>(sh, a, s);
}

template <class R, int MODE>
cudaError_t launch_fused(hqmc_config* cfg, const MdagmArgs<R>& a, cudaStream_t s) {
  return launch_shape<R, MODE>(fused_shape<R>(cfg), a, s);
}

template <class R, int MODE>
MdagmArgs<R> mdagm_args(hqmc_config* cfg) {
  MdagmArgs<R> a{};
  a.g = cfg->g;
  a.cB = (R)cfg->cB;
  a.th32 = cfg->th32;
  a.t1 = cfg->t1;
  a.t2 = cfg->t2;
  a.err = cfg->dev_err;
  return a;
}

// r_out = b - O x (FP64) with partials; then the state bookkeeping.
int residual(hqmc_config* cfg, const double2* b, const double2* x, void* r_out, bool r_fp32, int fin_mode,
             double tol, int maxit, int gate, cudaStream_t s) {
  MdagmArgs<double> a = mdagm_args<double, MODE_RESID>(cfg);
  a.U = cfg->U64;
  a.x = x;
  a.b = b;
  a.r_out = r_out;
  a.r_out_fp32 = r_fp32 ? 1 : 0;
  a.part_out = cfg->part_resid;
  a.st = cfg->st;
  a.gate = gate;
  // the autotuned FP64 shape where it is the generic kernel (the residual mode
  // exists only there), else the default generic shape
  const SliceLaunch& rs = (cfg->fused64.nby == 0 && cfg->fused64.mb == cfg->sl.mb) ? cfg->fused64 : cfg->sl;
  int slot;
  RET(timer_begin(cfg, HQMC_TIMER_MDAGM, s, &slot));
  LK(1, (launch_mdagm<double, MODE_RESID>(rs, a, s)));
  RET(timer_end(cfg, HQMC_TIMER_MDAGM, s, slot));
  LK(1, launch_resid_finalize(cfg->part_resid, rs.grid, fin_mode, tol, maxit, cfg->part_ew, cfg->n_part_ew,
                           cfg->st, cfg->report, gate, s));
  return HQMC_OK;
}

// Solver ids: CG64 / MIXED / LEARNED, and the same three with the tau-line
// preconditioner (PCG64 / PMIXED / PLEARNED).
// HQMC_SOLVER_FLEARNED: flexible CG with the net (every net_interval-th iteration)
// and the tau-line preconditioner (the others), after the learned initial guess.
bool solver_fcg(int solver) { return solver == HQMC_SOLVER_FLEARNED; }
bool solver_pc(int solver) { return solver >= HQMC_SOLVER_PCG64; }
int solver_base(int solver) {
  if (solver_fcg(solver)) return HQMC_SOLVER_LEARNED;
  return solver_pc(solver) ? solver - HQMC_SOLVER_PCG64 : solver;
}
bool solver_fp32(int solver) { return solver_base(solver) != HQMC_SOLVER_CG64; }

// z = Otilde^{-1} r and the partials of <r, z>, gated on a running solve
// (st = NULL: always).
template <class R>
int precondition(hqmc_config* cfg, const C2<R>* r, C2<R>* z, const CgState* st, cudaStream_t s) {
  LK(1, launch_line_precond<R>(cfg->g, cfg->lc, sizeof(R) == 8 ? cfg->ll64 : cfg->ll32, r, z, cfg->part_rz, st, s));
  return HQMC_OK;
}

// One CG iteration: the direction step, then the vector update.  Preconditioned:
// with `rb` set, the update is fused with the preconditioner and moves r from
// r to rb (odd iterations of a loop body: from rb back to r); without it, the
// plain update and a separate preconditioner application.
template <class R>
int cg_iteration(hqmc_config* cfg, C2<R>* r, C2<R>* const pbuf[2], C2<R>* q, const C2<R>* U, void* x,
                 bool x_double, bool pc, C2<R>* z, C2<R>* rb, int c, cudaStream_t s) {
  const bool fused = pc && rb != nullptr;
  const LineLaunch& ll = fused ? (sizeof(R) == 8 ? cfg->llu64 : cfg->llu32) : (sizeof(R) == 8 ? cfg->ll64 : cfg->ll32);
  const LineLaunch& lls = sizeof(R) == 8 ? cfg->ll64 : cfg->ll32;
  MdagmArgs<R> a = mdagm_args<R, MODE_CGDIR>(cfg);
  a.U = U;
  a.y = q;
  a.r = pc ? z : r;  // preconditioned CG: the direction is built from z = Otilde^{-1} r
  if (pc) {
    // <r, z> partials: a body's first iteration reads those of the separate
    // preconditioner that closed the previous body (or started the solve)
    const LineLaunch& lz = (fused && c > 0) ? ll : lls;
    a.part_rz = cfg->part_rz;
    a.n_part_rz = lz.gx * lz.gy;
  }
  a.pbuf[0] = pbuf[0];
  a.pbuf[1] = pbuf[1];
  a.part_in = cfg->part_ew;
  a.n_part_in = fused ? ll.gx * ll.gy : cfg->ew_grid;
  a.part_out = cfg->part_mdagm;
  a.st = cfg->st;
  int slot;
  const int tcls = sizeof(R) == 8 ? HQMC_TIMER_MDAGM : HQMC_TIMER_MDAGM32;
  RET(timer_begin(cfg, tcls, s, &slot));
  LK(1, (launch_fused<R, MODE_CGDIR>(cfg, a, s)));
  RET(timer_end(cfg, tcls, s, slot));
  RET(timer_begin(cfg, HQMC_TIMER_CG_UPDATE, s, &slot));
  if (fused) {
    LineUpdArgs<R> u{};
    u.x = reinterpret_cast<C2<R>*>(x);
    u.r_in = (c & 1) ? rb : r;
    u.r_out = (c & 1) ? r : rb;
    u.p0 = pbuf[0];
    u.p1 = pbuf[1];
    u.q = q;
    u.z = z;
    u.part_pq = cfg->part_mdagm;
    u.n_pq = fused_shape<R>(cfg).grid;
    u.part_rr = cfg->part_ew;
    u.part_rz = cfg->part_rz;
    u.st = cfg->st;
    LK(1, launch_line_update<R>(cfg->g, cfg->lc, ll, u, s));
    RET(timer_end(cfg, HQMC_TIMER_CG_UPDATE, s, slot));
    return HQMC_OK;
  }
  LK(1, launch_cg_update<R>(cfg->n, cfg->ew_grid, x, x_double ? 1 : 0, r, pbuf, q, cfg->part_mdagm, fused_shape<R>(cfg).grid,
                         cfg->part_ew, cfg->st, s));
  RET(timer_end(cfg, HQMC_TIMER_CG_UPDATE, s, slot));
  if (pc) {
    RET(timer_begin(cfg, HQMC_TIMER_PRECOND, s, &slot));
    RET(precondition<R>(cfg, r, z, cfg->st, s));
    RET(timer_end(cfg, HQMC_TIMER_PRECOND, s, slot));
  }
  return HQMC_OK;
}

int read_state(hqmc_config* cfg, cudaStream_t s) {
  CK(cudaMemcpyAsync(cfg->st_h, cfg->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(cfg->report_h, cfg->report, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(cfg->dev_err_h, cfg->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return HQMC_OK;
}

// ---------------------------------------------------------------------------
// Learned preconditioner (see net.cu): 4 layers, channels 1 -> 16 -> 16 -> 16 -> 1.

constexpr int kNetLayers = 4;
constexpr int kNetCh = 16;
constexpr int kNetChunks = 304;  // site chunks of the weight-gradient reduction (one block each; 2 per SM)

}  // namespace

struct hqmc_net {
  int cin[kNetLayers] = {1, kNetCh, kNetCh, kNetCh};
  int cout[kNetLayers] = {kNetCh, kNetCh, kNetCh, 1};
  int off[kNetLayers + 1] = {0, 0, 0, 0, 0};
  int total = 0;
  float* w = nullptr;      // FP32 master weights (device)
  float* m = nullptr;      // Adam moments
  float* v = nullptr;
  void* wb = nullptr;      // BF16 weights used by the layers
  void* wt = nullptr;      // BF16 adjoint weights (backward stencil)
  std::vector<float> hw;   // host copy of the BF16 weights as floats (inference launches take them by value)
  int hw_valid = 0;        // cleared when a training step changes the device weights
  long long version = 0;   // bumped whenever the weights change (captured solve loops hold them by value)
  int steps = 0;
  int device = 0;
};

namespace {

// Allocates the net's activation and gradient fields on the config (once).  Called
// only from hqmc_set_preconditioner, so that no solve, apply or training step
// allocates device memory.
bool net_ready(const hqmc_config* cfg) { return cfg->net_scal != nullptr; }  // the last field allocated

int net_workspace(hqmc_config* cfg) {
  if (net_ready(cfg)) return HQMC_OK;
  const size_t n = cfg->n;
  const int ch[5] = {1, kNetCh, kNetCh, kNetCh, 1};
  for (int l = 0; l < 5; ++l) RET(dalloc(cfg, &cfg->net_h[l], n * ch[l]));
  RET(dalloc(cfg, &cfg->net_d[0], n * kNetCh));
  RET(dalloc(cfg, &cfg->net_d[1], n * kNetCh));
  RET(dalloc(cfg, &cfg->net_part, (size_t)kNetChunks * 7 * kNetCh * kNetCh + 4096));
  RET(dalloc(cfg, &cfg->r_old32, n));
  RET(dalloc(cfg, &cfg->part_fz, (size_t)cfg->act_grid));
  RET(dalloc(cfg, &cfg->part_fx, (size_t)cfg->act_grid));
  RET(dalloc(cfg, &cfg->net_scal, 8));
  return HQMC_OK;
}

// z = K(theta) r for complex-double r, z; the float theta table must be current.
// Inference layers take the weights by value from the host copy (refreshed
// from the device after training steps); the training forward pass reads the
// device weights that its Adam steps update.
// Host copy of the BF16 weights as floats, refreshed from the device after
// training steps (a synchronous copy: never called inside a stream capture).
int net_host_weights(hqmc_config* cfg, hqmc_net* net, cudaStream_t s) {
  if (net->hw_valid) return HQMC_OK;
  std::vector<__nv_bfloat16> hb(net->total);
  CK(cudaMemcpyAsync(hb.data(), net->wb, net->total * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  net->hw.resize(net->total);
  for (int e = 0; e < net->total; ++e) net->hw[e] = __bfloat162float(hb[e]);
  net->hw_valid = 1;
  return HQMC_OK;
}

int net_forward(hqmc_config* cfg, hqmc_net* net, const double2* r, double2* z, cudaStream_t s,
                bool host_weights = true) {
  if (host_weights) RET(net_host_weights(cfg, net, s));
  LK(1, launch_net_convert(r, cfg->net_h[0], 1, 1.0, cfg->n, s));
  for (int l = 0; l < kNetLayers; ++l) {
    if (host_weights)
      LK(1, launch_net_layer_host_weights(cfg->g, cfg->th32, net->hw.data() + net->off[l], net->cin[l], net->cout[l],
                                          cfg->net_h[l], cfg->net_h[l + 1], nullptr, s, cfg->net_tc != 0));
    else
      LK(1, launch_net_layer(cfg->g, cfg->th32, (const char*)net->wb + 2 * (size_t)net->off[l], net->cin[l],
                             net->cout[l], cfg->net_h[l], cfg->net_h[l + 1], s));
  }
  if (z) LK(1, launch_net_convert(cfg->net_h[kNetLayers], z, 0, 1.0, cfg->n, s));
  return HQMC_OK;
}

// Flexible CG: z = K(theta) r in complex float, the first layer reading r and the
// last writing z (one channel is the same in every layout); gated on a running
// solve.  The float theta table must be current and the host weights valid.
int net_forward32(hqmc_config* cfg, hqmc_net* net, const float2* r, float2* z, cudaStream_t s) {
  const float2* in = r;
  for (int l = 0; l < kNetLayers; ++l) {
    float2* out = l == kNetLayers - 1 ? z : cfg->net_h[l + 1];
    LK(1, launch_net_layer_host_weights(cfg->g, cfg->th32, net->hw.data() + net->off[l], net->cin[l], net->cout[l],
                                        in, out, cfg->st, s, cfg->net_tc != 0));
    in = out;
  }
  return HQMC_OK;
}

// Flexible CG's preconditioner step for the iteration that follows: z = K r (net)
// or z = Otilde^{-1} r (tau-line), then the partials of Re<r, z> and Re<r_old, z>.
int fcg_precondition(hqmc_config* cfg, bool use_net, cudaStream_t s) {
  int slot;
  RET(timer_begin(cfg, HQMC_TIMER_PRECOND, s, &slot));
  if (use_net) RET(net_forward32(cfg, cfg->net, cfg->r32, cfg->z32, s));
  else RET(precondition<float>(cfg, cfg->r32, cfg->z32, cfg->st, s));
  RET(timer_end(cfg, HQMC_TIMER_PRECOND, s, slot));
  LK(1, launch_fcg_dots(cfg->n, cfg->r32, cfg->r_old32, cfg->z32, cfg->act_grid, cfg->part_fz, cfg->part_fx, cfg->st, s));
  return HQMC_OK;
}

// One flexible-CG iteration c of a mixed loop body (FP32 recurrence, Notay's FCG
// with one kept direction = Polak-Ribiere beta): p = z + beta p_old and q = O p
// (the direction kernel, beta from the <r, z> and <r_old, z> partials), r_old = r,
// x += alpha p, r -= alpha q, then the preconditioner of iteration c + 1 (the net
// when (c + 1) % net_interval == 0).
int fcg_iteration(hqmc_config* cfg, int c, cudaStream_t s) {
  MdagmArgs<float> a = mdagm_args<float, MODE_CGDIR>(cfg);
  a.U = cfg->U32;
  a.y = cfg->q32;
  a.r = cfg->z32;
  a.part_rz = cfg->part_fz;
  a.part_cross = cfg->part_fx;
  a.n_part_rz = cfg->act_grid;
  a.pbuf[0] = cfg->p32[0];
  a.pbuf[1] = cfg->p32[1];
  a.part_in = cfg->part_ew;
  a.n_part_in = cfg->ew_grid;
  a.part_out = cfg->part_mdagm;
  a.st = cfg->st;
  int slot;
  RET(timer_begin(cfg, HQMC_TIMER_MDAGM32, s, &slot));
  LK(1, (launch_fused<float, MODE_CGDIR>(cfg, a, s)));
  RET(timer_end(cfg, HQMC_TIMER_MDAGM32, s, slot));
  CK(cudaMemcpyAsync(cfg->r_old32, cfg->r32, sizeof(float2) * cfg->n, cudaMemcpyDeviceToDevice, s));
  RET(timer_begin(cfg, HQMC_TIMER_CG_UPDATE, s, &slot));
  LK(1, launch_cg_update<float>(cfg->n, cfg->ew_grid, cfg->xh32, 0, cfg->r32, cfg->p32, cfg->q32, cfg->part_mdagm,
                                fused_shape<float>(cfg).grid, cfg->part_ew, cfg->st, s));
  RET(timer_end(cfg, HQMC_TIMER_CG_UPDATE, s, slot));
  return fcg_precondition(cfg, (c + 1) % cfg->net_interval == 0, s);
}

int theta_float(hqmc_config* cfg, const double* theta, cudaStream_t s) {
  LK(1, launch_links(cfg->g, theta, cfg->t1, cfg->t2, nullptr, nullptr, cfg->th32, s));
  return HQMC_OK;
}

// One body of the CG loop: a block of iterations followed by the residual
// check that closes it.  FP64: kBodyIters64 iterations, then (only if the
// recursive residual converged) the true residual and a restart if needed.
// Mixed: reliable_interval FP32 iterations, then the FP64 reliable update
// x += xh, r = phi - O x (whenever the solve is still active).
int enqueue_body(hqmc_config* cfg, int solver, const double2* phi, double2* x, cudaStream_t s, int* nkernels) {
  const bool mixed = solver_fp32(solver);
  const bool pc = solver_pc(solver);
  const int iters = mixed ? cfg->reliable : kBodyIters64;
  if (solver_fcg(solver)) {
    // flexible CG: the reliable update closes the body and the net preconditions
    // the new residual (iteration 0 of the next body)
    int nets = 0;
    for (int c = 0; c < iters; ++c) {
      RET(fcg_iteration(cfg, c, s));
      nets += (c + 1) % cfg->net_interval == 0;
    }
    LK(1, launch_accumulate_correction(cfg->n, x, cfg->xh32, cfg->st, GATE_ACTIVE, s));
    RET(residual(cfg, phi, x, cfg->r32, true, FIN_RELIABLE, 0.0, 0, GATE_ACTIVE, s));
    RET(fcg_precondition(cfg, true, s));
    *nkernels = 3 * iters + 4 * (nets + 1) + (iters - nets) + 3 + 1;
    return HQMC_OK;
  }
  // the fused preconditioned update alternates two residual buffers, so an even
  // number of iterations per body leaves r where the body's residual expects it
  const bool fuse = pc && (iters % 2 == 0) && (mixed ? cfg->fuse_pc32 : cfg->fuse_pc64) && cfg->p.variant != 1;
  for (int c = 0; c < iters; ++c) {
    if (mixed)
      RET(cg_iteration<float>(cfg, cfg->r32, cfg->p32, cfg->q32, cfg->U32, cfg->xh32, false, pc, cfg->z32,
                              fuse ? cfg->r32b : nullptr, c, s));
    else
      RET(cg_iteration<double>(cfg, cfg->r64, cfg->p64, cfg->q64, cfg->U64, x, true, pc, cfg->z64,
                               fuse ? cfg->r64b : nullptr, c, s));
  }
  if (mixed) {
    LK(1, launch_accumulate_correction(cfg->n, x, cfg->xh32, cfg->st, GATE_ACTIVE, s));
    RET(residual(cfg, phi, x, cfg->r32, true, FIN_RELIABLE, 0.0, 0, GATE_ACTIVE, s));
    if (pc) RET(precondition<float>(cfg, cfg->r32, cfg->z32, cfg->st, s));
  } else {
    RET(residual(cfg, phi, x, cfg->r64, false, FIN_RESTART, 0.0, 0, GATE_REC, s));
    // after a restart z must follow the new r; otherwise this recomputes the same z
    if (pc) RET(precondition<double>(cfg, cfg->r64, cfg->z64, cfg->st, s));
  }
  *nkernels = (pc && !fuse ? 3 : 2) * iters + (mixed ? 3 : 2) + (pc ? 1 : 0);
  return HQMC_OK;
}

// Builds (or finds) the graph that runs loop bodies under a WHILE node until
// the CG state leaves RUNNING: the loop condition is decided on the device.
int get_graph(hqmc_config* cfg, int solver, const double2* phi, double2* x, SolveGraph** out) {
  const long long ver = solver_fcg(solver) && cfg->net ? cfg->net->version : 0;
  for (auto& g : cfg->graphs)
    if (g.phi == phi && g.x == x && g.solver == solver && g.net_version == ver) {
      *out = &g;
      return HQMC_OK;
    }
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(cfg, HQMC_ECUDA, "conditional graph node: %s", cudaGetErrorString(e));
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(cfg->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cfg->capturing = 1;
  int nk = 0;
  int rc = enqueue_body(cfg, solver, phi, x, cfg->cap, &nk);
  if (rc == HQMC_OK) {
    cudaError_t le = launch_loop_condition(cfg->st, handle, cfg->cap);
    if (le != cudaSuccess) rc = fail(cfg, HQMC_ECUDA, "loop condition launch: %s", cudaGetErrorString(le));
  }
  cfg->capturing = 0;
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cfg->cap, &captured);
  if (rc == HQMC_OK && e != cudaSuccess) rc = fail(cfg, HQMC_ECUDA, "end capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  if (rc == HQMC_OK) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) rc = fail(cfg, HQMC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  cudaGraphDestroy(graph);
  if (rc != HQMC_OK) {
    cudaGetLastError();
    return rc;
  }
  if (cfg->graphs.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(cfg->graphs.front().exec);
    cfg->graphs.erase(cfg->graphs.begin());
  }
  cfg->graphs.push_back(SolveGraph{phi, x, solver, ver, nk + 1, exec});
  *out = &cfg->graphs.back();
  return HQMC_OK;
}

// Runs loop bodies until the state leaves RUNNING / REC_CONVERGED; the state
// is in cfg->st_h on return.  Uses the device-side loop unless event timing is
// on (per-launch events cannot sit inside a conditional body).
int run_loop(hqmc_config* cfg, int solver, const double2* phi, double2* x, int* loops_seen, cudaStream_t s) {
  if (!cfg->timing && cfg->graphs_ok) {
    SolveGraph* gr = nullptr;
    if (get_graph(cfg, solver, phi, x, &gr) == HQMC_OK) {
      CK(cudaGraphLaunch(gr->exec, s));
      RET(read_state(cfg, s));
      const int loops = cfg->st_h->loops;
      cfg->launches += (long long)(loops - *loops_seen) * gr->body_kernels;
      *loops_seen = loops;
      return HQMC_OK;
    }
    cfg->graphs_ok = 0;  // fall back to host-driven bodies from now on
  }
  for (;;) {
    RET(read_state(cfg, s));
    const int d = cfg->st_h->done;
    if (d != CG_RUNNING && d != CG_REC_CONVERGED) return HQMC_OK;
    int nk = 0;
    RET(enqueue_body(cfg, solver, phi, x, s, &nk));
  }
}

// Solves the Hermitian positive definite k x k system A c = b in place (b -> c) by
// Cholesky; false if a pivot falls below 1e-12 of its diagonal entry (the earlier
// solutions are then too close to linearly dependent for the projection).
bool hermitian_solve(int k, std::vector<double>& A, std::vector<double>& b) {
  // A: k x k complex, row-major, interleaved (re, im); b: k complex
  auto re = [&](int i, int j) -> double& { return A[2 * (i * k + j)]; };
  auto im = [&](int i, int j) -> double& { return A[2 * (i * k + j) + 1]; };
  for (int j = 0; j < k; ++j) {
    double d = re(j, j);
    for (int p = 0; p < j; ++p) d -= re(j, p) * re(j, p) + im(j, p) * im(j, p);
    if (!(d > 1e-12 * std::fabs(re(j, j)))) return false;
    const double ljj = std::sqrt(d);
    re(j, j) = ljj;
    im(j, j) = 0.0;
    for (int i = j + 1; i < k; ++i) {
      double sr = re(i, j), si = im(i, j);
      for (int p = 0; p < j; ++p) {  // - L_ip conj(L_jp)
        sr -= re(i, p) * re(j, p) + im(i, p) * im(j, p);
        si -= im(i, p) * re(j, p) - re(i, p) * im(j, p);
      }
      re(i, j) = sr / ljj;
      im(i, j) = si / ljj;
    }
  }
  for (int i = 0; i < k; ++i) {  // L y = b
    double sr = b[2 * i], si = b[2 * i + 1];
    for (int p = 0; p < i; ++p) {
      sr -= re(i, p) * b[2 * p] - im(i, p) * b[2 * p + 1];
      si -= re(i, p) * b[2 * p + 1] + im(i, p) * b[2 * p];
    }
    b[2 * i] = sr / re(i, i);
    b[2 * i + 1] = si / re(i, i);
  }
  for (int i = k - 1; i >= 0; --i) {  // L^dagger c = y
    double sr = b[2 * i], si = b[2 * i + 1];
    for (int p = i + 1; p < k; ++p) {  // - conj(L_pi) c_p
      sr -= re(p, i) * b[2 * p] + im(p, i) * b[2 * p + 1];
      si -= re(p, i) * b[2 * p + 1] - im(p, i) * b[2 * p];
    }
    b[2 * i] = sr / re(i, i);
    b[2 * i + 1] = si / re(i, i);
  }
  return true;
}

// CG on (M^dagger M) x = phi with the link tables already built for theta.
// HQMC_SOLVER_LEARNED: x <- x + K(theta)(phi - O x) from the attached net, kept
// only if it lowers the FP64 residual, then the mixed solver (plain CG with its
// FP64 true residual stays the judge and the fallback).
// Within one leapfrog integration that has the chronological guess, the learned
// guess is not tried again after kNetMaxRejects consecutive tries that did not cut
// the residual norm at least in half (||r1||^2 >= kNetGainMin ||r0||^2).  A net apply
// costs about as much as eight CG iterations at L = 66, and CG takes about 28
// iterations per decade of residual there, so a try pays only above a 2x cut.
constexpr int kNetMaxRejects = 2;
constexpr double kNetGainMin = 0.25;

int solve(hqmc_config* cfg, const double2* phi, double2* x, double tol, int maxit, int solver,
          hqmc_solve_info* info, cudaStream_t s) {
  NvtxRange nv("hqmc cg solve");
  int net_used = 0;
  const bool pc = solver_pc(solver);
  cfg->net_tried = 0;
  if (solver_base(solver) == HQMC_SOLVER_LEARNED) {
    if (!solver_fcg(solver)) solver = pc ? HQMC_SOLVER_PMIXED : HQMC_SOLVER_MIXED;
    // Inside a leapfrog integration with the chronological guess, the net is not
    // tried again after kNetMaxRejects consecutive tries below the 2x cut (reset per
    // integration).
    if (!(cfg->net_adaptive && cfg->net_rejects >= kNetMaxRejects)) {
      // candidate x + z with z = K r0, r0 = phi - O x.  Both residual norms come from
      // the FP32 fused apply (r1 = r0 - O z): they only decide whether z is kept, and
      // a rejected z then costs no FP64 residual and no copy of x.  The FP64 residual
      // that starts the recurrence is computed afterwards, as for any solve.
      cfg->net_tried = 1;
      MdagmArgs<float> a = mdagm_args<float, MODE_APPLY>(cfg);
      a.U = cfg->U32;
      a.x = cfg->xh32;
      a.y = cfg->q32;
      LK(1, launch_net_convert(x, cfg->xh32, 1, 1.0, cfg->n, s));  // x as float (xh32 is free until the loop)
      LK(1, (launch_fused<float, MODE_APPLY>(cfg, a, s)));
      LK(1, launch_resid_from_fp32(cfg->n, phi, cfg->q32, cfg->vscratch, s));  // r0
      LK(2, launch_cdot(cfg->n, cfg->vscratch, cfg->vscratch, cfg->act_grid, cfg->part_act, cfg->report, s));
      RET(net_forward(cfg, cfg->net, cfg->vscratch, cfg->p64[1], s));  // z = K r0 (reads the host weights first)
      LK(1, launch_net_convert(cfg->p64[1], cfg->xh32, 1, 1.0, cfg->n, s));
      LK(1, (launch_fused<float, MODE_APPLY>(cfg, a, s)));
      LK(1, launch_resid_from_fp32(cfg->n, cfg->vscratch, cfg->q32, cfg->r64, s));  // r1 = r0 - O z (r64 free here)
      LK(2, launch_cdot(cfg->n, cfg->r64, cfg->r64, cfg->act_grid, cfg->part_act, cfg->report + 1, s));
      RET(read_state(cfg, s));
      if (cfg->report_h[1] < cfg->report_h[0]) {
        net_used = 1;
        LK(1, launch_kick(2 * cfg->n, (double*)x, (const double*)cfg->p64[1], 1.0, s));  // x += z
      }
      cfg->net_rejects = (cfg->report_h[1] < kNetGainMin * cfg->report_h[0]) ? 0 : cfg->net_rejects + 1;
    }
  }
  const bool started = false;
  const bool mixed = solver_fp32(solver);
  hqmc_solve_info inf{};
  if (!started)
    RET(residual(cfg, phi, x, mixed ? (void*)cfg->r32 : (void*)cfg->r64, mixed, FIN_START, tol, maxit, GATE_ALWAYS, s));
  if (mixed) CK(cudaMemsetAsync(cfg->xh32, 0, sizeof(float2) * cfg->n, s));
  if (solver_fcg(solver)) {
    RET(net_host_weights(cfg, cfg->net, s));  // outside any capture: the loop bodies take them by value
    RET(fcg_precondition(cfg, true, s));
  } else if (pc) {
    if (mixed) RET(precondition<float>(cfg, cfg->r32, cfg->z32, cfg->st, s));
    else RET(precondition<double>(cfg, cfg->r64, cfg->z64, cfg->st, s));
  }
  int cur = solver, loops_seen = 0, status = HQMC_OK;
  for (;;) {
    RET(run_loop(cfg, cur, phi, x, &loops_seen, s));
    const CgState& st = *cfg->st_h;
    if (st.bb == 0.0) {  // phi = 0: the solution is zero whatever the guess
      CK(cudaMemsetAsync(x, 0, sizeof(double2) * cfg->n, s));
      cfg->report_h[0] = 0.0;
      break;
    }
    if (st.done == CG_CONVERGED) break;
    if ((st.done == CG_BREAKDOWN || st.done == CG_STAGNATED) && solver_fcg(cur)) {
      // the net made Re<r, z> or <p, O p> non-positive, or stalled the recurrence:
      // fold in the correction and continue with the tau-line preconditioned mixed
      // solver from the FP64 residual of x (the fixed-preconditioner fallback)
      inf.restarts++;
      inf.fcg_fallback = 1;
      LK(1, launch_accumulate_correction(cfg->n, x, cfg->xh32, nullptr, GATE_ALWAYS, s));
      cur = HQMC_SOLVER_PMIXED;
      RET(residual(cfg, phi, x, cfg->r32, true, FIN_RESTART, tol, maxit, GATE_ALWAYS, s));
      RET(precondition<float>(cfg, cfg->r32, cfg->z32, cfg->st, s));
      continue;
    }
    if ((st.done == CG_BREAKDOWN || st.done == CG_STAGNATED) && solver_fp32(cur)) {
      // <p, O32 p> <= 0 or a stalled residual: FP32 rounding cannot resolve the
      // lowest modes of this field.  Fold in the correction and restart from the
      // FP64 residual; after repeated breakdowns, or at once on stagnation,
      // finish the solve with the FP64 recurrence.
      inf.restarts++;
      LK(1, launch_accumulate_correction(cfg->n, x, cfg->xh32, nullptr, GATE_ALWAYS, s));
      if (st.done == CG_STAGNATED || inf.restarts > kMaxBreakdowns) {
        cur = pc ? HQMC_SOLVER_PCG64 : HQMC_SOLVER_CG64;
        inf.fp64_fallback = 1;
        RET(residual(cfg, phi, x, cfg->r64, false, FIN_RESTART, tol, maxit, GATE_ALWAYS, s));
        if (pc) RET(precondition<double>(cfg, cfg->r64, cfg->z64, cfg->st, s));
      } else {
        RET(residual(cfg, phi, x, cfg->r32, true, FIN_RESTART, tol, maxit, GATE_ALWAYS, s));
        if (pc) RET(precondition<float>(cfg, cfg->r32, cfg->z32, cfg->st, s));
      }
      continue;
    }
    // MAXIT, NONFINITE, or a breakdown of the FP64 recurrence: report the true residual of x
    status = solve_status(st.done, *cfg->dev_err_h != 0);
    if (solver_fp32(cur)) LK(1, launch_accumulate_correction(cfg->n, x, cfg->xh32, nullptr, GATE_ALWAYS, s));
    RET(residual(cfg, phi, x, cfg->vscratch, false, FIN_REPORT, tol, maxit, GATE_ALWAYS, s));
    RET(read_state(cfg, s));
    break;
  }
  const CgState& st = *cfg->st_h;
  inf.reliable_updates = mixed ? st.loops : 0;
  inf.net_guess_used = net_used;
  inf.status = status;
  inf.iterations = st.k;
  inf.true_residual = st.bb > 0 ? std::sqrt(cfg->report_h[0] / st.bb) : 0.0;
  const double rr_rec = (pc && st.k > st.seg_start) ? st.rr_rec : st.rr[st.k & 1];
  inf.recursive_residual = st.bb > 0 ? std::sqrt(rr_rec / st.bb) : 0.0;
  if (status == HQMC_OK && !(inf.true_residual <= tol)) status = inf.status = HQMC_ENOTCONV;
  if (*cfg->dev_err_h) {  // a bounded wait gave up during this solve (or an apply before it)
    status = inf.status = solve_status(st.done, true);
    *cfg->dev_err_h = 0;
    CK(cudaMemsetAsync(cfg->dev_err, 0, sizeof(int), s));
  }
  if (info) *info = inf;
  return status;
}


int force(hqmc_config* cfg, const double* theta, const double2* X, double* F, double* dSf, cudaStream_t s) {
  NvtxRange nv("hqmc force");
  int slot;
  RET(timer_begin(cfg, HQMC_TIMER_FORCE, s, &slot));
  LK(1, launch_force(cfg->sl1, cfg->cB, cfg->t1, cfg->t2, cfg->U64, X, dSf, s));
  RET(timer_end(cfg, HQMC_TIMER_FORCE, s, slot));
  LK(1, launch_force_finish(cfg->g, cfg->bp, theta, dSf, F, s));
  return HQMC_OK;
}

int merge_status(int a, int b) { return a != HQMC_OK ? a : b; }

// Chronological initial guess (Brower, Ivanenko, Levi, Orginos, "Chronological
// inversion method for the Dirac matrix in hybrid Monte Carlo", 1997): the
// solutions of the last hist_n solves of this integration, at fields a few
// leapfrog steps back, span a space that holds most of the new solution.  The
// guess is the Galerkin solution in that space with the current operator:
// Q = orthonormal basis of the stored solutions (classical Gram-Schmidt, twice),
// G = Q^dagger O Q with O applied in FP32, b = Q^dagger phi, x = Q G^{-1} b.
// Uses the FP32 link tables of the current field and, as scratch, xh32, q32, q64
// and vscratch (free before a solve).  Leaves x unchanged (the previous solution)
// if the basis or G degenerates.
int chrono_guess(hqmc_config* cfg, const double2* phi, double2* x, cudaStream_t s) {
  const int m0 = cfg->hist_n;
  if (m0 < 2) return HQMC_OK;
  const long long n = cfg->n;
  const size_t vb = (size_t)n * sizeof(double2);
  const int grid = cfg->act_grid;
  double* dsc = reinterpret_cast<double*>(cfg->vscratch);  // many-dot partials and results
  double* dout = dsc + 2 * (size_t)grid * cfg->guess_cap;
  std::vector<double> d(2 * (size_t)cfg->guess_cap);
  auto dots = [&](int k, const double2* v) -> int {  // d = (<Q_i, v>)_{i<k}
    LK(2, launch_cdot_many(n, cfg->qbasis, n, k, v, grid, dsc, dout, s));
    CK(cudaMemcpyAsync(d.data(), dout, 2 * (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return HQMC_OK;
  };
  int m = 0;
  for (int j = 0; j < m0; ++j) {
    double2* qj = cfg->qbasis + (size_t)m * n;
    CK(cudaMemcpyAsync(qj, cfg->hist + (size_t)j * n, vb, cudaMemcpyDeviceToDevice, s));
    RET(dots(m + 1, qj));
    const double nrm0 = d[2 * m];
    for (int pass = 0; pass < 2 && m > 0; ++pass) {  // d holds <Q_i, q_j> of the current q_j
      for (int i = 0; i < m; ++i)
        LK(1, launch_caxpy(n, -d[2 * i], -d[2 * i + 1], cfg->qbasis + (size_t)i * n, qj, s));
      RET(dots(m + 1, qj));
    }
    const double nrm = d[2 * m];
    if (!(nrm > 1e-20 * nrm0) || !(nrm > 0.0)) continue;  // (nearly) in the span already: drop it
    LK(1, launch_dscale(n, 1.0 / std::sqrt(nrm), qj, s));
    ++m;
  }
  if (m == 0) return HQMC_OK;
  // G = Q^dagger O Q, column by column: O q_j in FP32, widened to FP64 in q64 (the
  // FP64 direction product, free outside a solve), then one many-dot per column
  std::vector<double> G(2 * (size_t)m * m), b;
  double2* w = cfg->q64;
  for (int j = 0; j < m; ++j) {
    LK(1, launch_net_convert(cfg->qbasis + (size_t)j * n, cfg->xh32, 1, 1.0, n, s));
    MdagmArgs<float> a = mdagm_args<float, MODE_APPLY>(cfg);
    a.U = cfg->U32;
    a.x = cfg->xh32;
    a.y = cfg->q32;
    LK(1, (launch_fused<float, MODE_APPLY>(cfg, a, s)));
    LK(1, launch_net_convert(cfg->q32, w, 0, 1.0, n, s));
    RET(dots(m, w));
    for (int i = 0; i < m; ++i) {
      G[2 * (i * m + j)] = d[2 * i];
      G[2 * (i * m + j) + 1] = d[2 * i + 1];
    }
  }
  for (int i = 0; i < m; ++i)  // Hermitian part (FP32 rounding of O breaks the symmetry slightly)
    for (int j = i; j < m; ++j) {
      const double re = 0.5 * (G[2 * (i * m + j)] + G[2 * (j * m + i)]);
      const double im = 0.5 * (G[2 * (i * m + j) + 1] - G[2 * (j * m + i) + 1]);
      G[2 * (i * m + j)] = re;
      G[2 * (i * m + j) + 1] = im;
      G[2 * (j * m + i)] = re;
      G[2 * (j * m + i) + 1] = -im;
    }
  RET(dots(m, phi));
  b.assign(d.begin(), d.begin() + 2 * m);
  if (!hermitian_solve(m, G, b)) return HQMC_OK;
  CK(cudaMemsetAsync(x, 0, vb, s));
  for (int i = 0; i < m; ++i) LK(1, launch_caxpy(n, b[2 * i], b[2 * i + 1], cfg->qbasis + (size_t)i * n, x, s));
  return HQMC_OK;
}

// Stores a solution of the current integration in the guess history (ring).
int chrono_push(hqmc_config* cfg, const double2* X, cudaStream_t s) {
  if (cfg->guess_k <= 0) return HQMC_OK;
  CK(cudaMemcpyAsync(cfg->hist + (size_t)cfg->hist_next * cfg->n, X, sizeof(double2) * cfg->n,
                     cudaMemcpyDeviceToDevice, s));
  cfg->hist_next = (cfg->hist_next + 1) % cfg->guess_k;
  cfg->hist_n = std::min(cfg->hist_n + 1, cfg->guess_k);
  return HQMC_OK;
}

int leapfrog(hqmc_config* cfg, double* theta, double* p, const double2* phi, double2* X, int nsteps, double dt,
             double tol, int maxit, int solver, hqmc_traj_info* ti, cudaStream_t s) {
  NvtxRange nv("hqmc leapfrog");
  const bool chrono = cfg->guess_k > 0;
  const bool mixed = solver_fp32(solver) || chrono;  // the guess applies O in FP32
  const bool learned = solver_base(solver) == HQMC_SOLVER_LEARNED;
  const long long nb = 2 * cfg->n;
  hqmc_solve_info si;
  int status = HQMC_OK;
  cfg->hist_n = cfg->hist_next = 0;  // a new integration: no earlier solutions
  // the learned guess gives way to the chronological one after repeated rejections
  // (only within this integration: the guard clears the gate on every exit)
  struct AdaptiveGate {
    hqmc_config* c;
    ~AdaptiveGate() { c->net_adaptive = 0; }
  } gate{cfg};
  cfg->net_adaptive = (chrono && learned) ? 1 : 0;
  cfg->net_rejects = 0;
  auto account = [&]() {
    ti->cg_solves++;
    ti->cg_iterations += si.iterations;
    ti->max_true_residual = std::fmax(ti->max_true_residual, si.true_residual);
    ti->net_guesses_tried += cfg->net_tried;
    ti->net_guesses_used += si.net_guess_used;
  };
  RET(links(cfg, theta, true, mixed, s, false, learned));
  int rc = solve(cfg, phi, X, tol, maxit, solver, &si, s);
  if (rc != HQMC_OK && rc != HQMC_ENOTCONV) return rc;
  status = merge_status(status, rc);
  account();
  RET(chrono_push(cfg, X, s));
  RET(force(cfg, theta, X, cfg->F, cfg->dSf, s));
  for (int n = 0; n < nsteps; ++n) {
    LK(1, launch_kick_drift(nb, p, theta, cfg->F, dt / 2, dt, s));
    RET(links(cfg, theta, true, mixed, s, false, learned));
    if (chrono) RET(chrono_guess(cfg, phi, X, s));  // else X is the previous solution
    rc = solve(cfg, phi, X, tol, maxit, solver, &si, s);
    if (rc != HQMC_OK && rc != HQMC_ENOTCONV) return rc;
    status = merge_status(status, rc);
    account();
    RET(chrono_push(cfg, X, s));
    RET(force(cfg, theta, X, cfg->F, cfg->dSf, s));
    LK(1, launch_kick(nb, p, cfg->F, dt / 2, s));
  }
  ti->status = status;
  return status;
}

int check_solver(hqmc_config* cfg, int solver) {
  if (solver < HQMC_SOLVER_CG64 || solver > HQMC_SOLVER_FLEARNED)
    return fail(cfg, HQMC_EINVAL, "unknown solver %d", solver);
  if (solver_base(solver) == HQMC_SOLVER_LEARNED && !cfg->net)
    return fail(cfg, HQMC_EINVAL, "the learned solver needs a net attached with hqmc_set_preconditioner");
  return HQMC_OK;
}

// ---------------------------------------------------------------------------
// Coefficients of the tau-line preconditioner (Methods, "CG method and
// preconditioner"), once per config, from the pi-flux field: one column of B
// gives b = B_ss and a = 1 + sum_j |B_js|^2 (every site is equivalent there);
// rho + 1/rho = a/b is the bulk Cholesky ratio of a - b (S + S^dagger), and the
// Neumann series of its factor keeps the powers whose entries sqrt(rho/b) rho^m
// are >= 1e-3.  (M e)_1 = -B_0 e_0 for the unit vector e at slice 0, site 0.
int line_coefficients(hqmc_config* cfg) {
  const Geo& g = cfg->g;
  LK(1, launch_pi_flux(g, cfg->th0, 0));
  CK(cudaMemset(cfg->p64[0], 0, sizeof(double2) * cfg->n));
  const double2 one = make_double2(1.0, 0.0);
  CK(cudaMemcpy(cfg->p64[0], &one, sizeof(double2), cudaMemcpyHostToDevice));
  LK(1, launch_links(g, cfg->th0, cfg->t1, cfg->t2, cfg->U64, nullptr, nullptr, 0));
  LK(1, launch_apply_M<double>(cfg->sl1, cfg->cB, cfg->U64, cfg->p64[0], cfg->q64, 0, 0));
  std::vector<double2> col(g.V);
  CK(cudaMemcpy(col.data(), cfg->q64 + g.V, sizeof(double2) * g.V, cudaMemcpyDeviceToHost));
  double norm2 = 0.0;
  for (const double2& c : col) norm2 += c.x * c.x + c.y * c.y;
  const double b = -col[0].x, a = 1.0 + norm2;
  if (!(b > 0.0) || !(a > 2.0 * b)) return fail(cfg, HQMC_EUNSUPPORTED, "tau-line coefficients a=%g b=%g", a, b);
  const double q = a / b, rho = 0.5 * (q - std::sqrt(q * q - 4.0)), pref = std::sqrt(rho / b);
  int W = 0;
  while (pref * std::pow(rho, W + 1) >= kLineTruncation && W < 4096) ++W;
  cfg->pc_a = a;
  cfg->pc_b = b;
  cfg->lc = LineCoef{rho, std::pow(rho, W + 1), rho / b, W};
  cfg->ll64 = line_launch(g, line_chunk_candidates(g, 8, W, cfg->num_sms, cfg->smem_per_sm).front());
  cfg->ll32 = line_launch(g, line_chunk_candidates(g, 4, W, cfg->num_sms, cfg->smem_per_sm).front());
  if (line_smem_bytes(8, W, cfg->ll64.chunk) > kMaxLineSmem || line_update_smem_bytes(8, W) > kMaxLineSmem)
    return fail(cfg, HQMC_EUNSUPPORTED, "tau-line preconditioner width W=%d too large", W);
  CK(prepare_line_precond<double>(W, cfg->ll64.chunk));
  CK(prepare_line_precond<float>(W, cfg->ll32.chunk));
  CK(prepare_line_update<double>(W));
  CK(prepare_line_update<float>(W));
  CK(cudaDeviceSynchronize());
  return HQMC_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times every admissible launch shape of the fused M^dagger M for
// this lattice (generic or register-blocked kernel, strip height nby, cluster
// size along tau) and keeps the fastest per precision.  Runs once per config
// on zero-valued operands (the kernels' cost does not depend on the values).

template <class R>
int time_shape(hqmc_config* cfg, const SliceLaunch& sh, float* us) {
  MdagmArgs<R> a = mdagm_args<R, MODE_APPLY>(cfg);
  if (sizeof(R) == 8) {
    a.U = (const C2<R>*)cfg->U64;
    a.x = (const C2<R>*)cfg->p64[0];
    a.y = (C2<R>*)cfg->q64;
  } else {
    a.U = (const C2<R>*)cfg->U32;
    a.x = (const C2<R>*)cfg->p32[0];
    a.y = (C2<R>*)cfg->q32;
  }
  auto go = [&]() { return launch_shape<R, MODE_APPLY>(sh, a, 0); };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t err = go();
  const int reps = 5;
  if (err == cudaSuccess) err = cudaEventRecord(e0, 0);
  for (int k = 0; k < reps && err == cudaSuccess; ++k) err = go();
  if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    cudaGetLastError();
    *us = -1.f;
    return HQMC_OK;
  }
  cfg->launches += reps + 1;
  *us = 1e3f * ms / reps;
  return HQMC_OK;
}

// Preconditioned CG: times the vector update fused with the preconditioner
// against the plain update followed by a preconditioner application, on zero
// vectors with a CG state set to "running", and keeps the faster form.
template <class R>
int tune_pc_update(hqmc_config* cfg) {
  CgState h{};
  h.done = CG_RUNNING;
  h.k = h.k2 = 1;
  h.maxit = 1 << 30;
  h.rr[0] = h.rr[1] = 1.0;
  CK(cudaMemcpy(cfg->st, &h, sizeof(CgState), cudaMemcpyHostToDevice));
  std::vector<double> ones((size_t)cfg->sl.grid + 8, 1.0);
  CK(cudaMemcpy(cfg->part_mdagm, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice));
  const bool dbl = sizeof(R) == 8;
  C2<R>* r = dbl ? (C2<R>*)cfg->r64 : (C2<R>*)cfg->r32;
  C2<R>* rb = dbl ? (C2<R>*)cfg->r64b : (C2<R>*)cfg->r32b;
  C2<R>* q = dbl ? (C2<R>*)cfg->q64 : (C2<R>*)cfg->q32;
  C2<R>* z = dbl ? (C2<R>*)cfg->z64 : (C2<R>*)cfg->z32;
  C2<R>* x = dbl ? (C2<R>*)cfg->vscratch : (C2<R>*)cfg->xh32;
  C2<R>* pb[2] = {dbl ? (C2<R>*)cfg->p64[0] : (C2<R>*)cfg->p32[0], dbl ? (C2<R>*)cfg->p64[1] : (C2<R>*)cfg->p32[1]};
  for (C2<R>* v : {r, rb, q, z, x, pb[0], pb[1]}) CK(cudaMemset(v, 0, sizeof(C2<R>) * cfg->n));
  const LineLaunch& ll = dbl ? cfg->ll64 : cfg->ll32;
  const LineLaunch& llu = dbl ? cfg->llu64 : cfg->llu32;
  const int npq = fused_shape<R>(cfg).grid;
  auto fused = [&]() {
    LineUpdArgs<R> u{x, r, rb, pb[0], pb[1], q, z, cfg->part_mdagm, npq, cfg->part_ew, cfg->part_rz, cfg->st};
    return launch_line_update<R>(cfg->g, cfg->lc, llu, u, 0);
  };
  auto separate = [&]() {
    cudaError_t e = launch_cg_update<R>(cfg->n, cfg->ew_grid, x, dbl ? 1 : 0, r, pb, q, cfg->part_mdagm, npq,
                                        cfg->part_ew, cfg->st, 0);
    if (e == cudaSuccess) e = launch_line_precond<R>(cfg->g, cfg->lc, ll, r, z, cfg->part_rz, cfg->st, 0);
    return e;
  };
  float us[2] = {0.f, 0.f};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t err = cudaSuccess;
  for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
    // every launch advances st->k by one; the state stays "running"
    err = v ? separate() : fused();
    const int reps = 5;
    if (err == cudaSuccess) err = cudaEventRecord(e0, 0);
    for (int k = 0; k < reps && err == cudaSuccess; ++k) err = v ? separate() : fused();
    if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    us[v] = 1e3f * ms / reps;
    cfg->launches += (reps + 1) * (v ? 2 : 1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(err);
  (dbl ? cfg->fuse_pc64 : cfg->fuse_pc32) = us[0] <= us[1] ? 1 : 0;
  CK(cudaMemset(cfg->st, 0, sizeof(CgState)));
  return HQMC_OK;
}

// Tile height of the separate FP32 preconditioner: times the candidate heights
// (line_chunk_candidates: the first few, and the fixed default) on zero operands
// and keeps the fastest.  The state stays "done = running"; no partials are read.
int tune_line_chunk(hqmc_config* cfg) {
  std::vector<int> cand = line_chunk_candidates(cfg->g, 4, cfg->lc.W, cfg->num_sms, cfg->smem_per_sm);
  if (cand.size() > 4) cand.erase(cand.begin() + 3, cand.end() - 1);
  CK(cudaMemset(cfg->st, 0, sizeof(CgState)));
  CK(cudaMemset(cfg->r32, 0, sizeof(float2) * cfg->n));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int chosen = cfg->ll32.chunk;
  cudaError_t err = cudaSuccess;
  for (int tc : cand) {
    const LineLaunch ll = line_launch(cfg->g, tc);
    err = prepare_line_precond<float>(cfg->lc.W, tc);
    if (err != cudaSuccess) break;
    auto go = [&]() {
      return launch_line_precond<float>(cfg->g, cfg->lc, ll, cfg->r32, cfg->z32, cfg->part_rz, cfg->st, 0);
    };
    err = go();
    const int reps = 5;
    if (err == cudaSuccess) err = cudaEventRecord(e0, 0);
    for (int k = 0; k < reps && err == cudaSuccess; ++k) err = go();
    if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err != cudaSuccess) break;
    cfg->launches += reps + 1;
    if (ms < best) {
      best = ms;
      chosen = tc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(err);
  cfg->ll32 = line_launch(cfg->g, chosen);
  return HQMC_OK;
}

int autotune(hqmc_config* cfg) {
  const int N = cfg->p.Ntau;
  CK(cudaMemset(cfg->th0, 0, 2 * cfg->n * sizeof(double)));
  CK(cudaMemset(cfg->p64[0], 0, cfg->n * sizeof(double2)));
  CK(cudaMemset(cfg->p32[0], 0, cfg->n * sizeof(float2)));
  LK(1, launch_links(cfg->g, cfg->th0, cfg->t1, cfg->t2, cfg->U64, cfg->U32, cfg->th32, 0));
  const int clusters[4] = {1, 2, 4, 8};
  for (int prec = 0; prec < 2; ++prec) {
    const bool dbl = prec == 0;
    std::vector<SliceLaunch> cand;
    const SliceLaunch gen = dbl ? cfg->sl : cfg->sl32;
    const SliceLaunch blk = dbl ? cfg->slb64 : cfg->slb32;
    for (int c : clusters) {
      if (c > N) continue;
      SliceLaunch g = gen;
      g.nby = 0;
      g.cluster = c;
      g.grid = (N + c - 1) / c * c;
      if (cfg->p.variant != 2) cand.push_back(g);
      if (blk.nby > 0) {
        SliceLaunch b = blk;
        b.cluster = c;
        b.grid = g.grid;
        cand.push_back(b);
      }
    }
    if (!dbl && cfg->slw32.walk) {
      // tau-walking kernel, every strip height that fits: one to a few CTAs per
      // SM, never more CTAs than slices
      for (const SliceLaunch& h : cfg->slw32h) {
        if (!h.walk) continue;
        const int bps = mdagm_walk_blocks_per_sm(h);
        for (int m = 1; m <= bps && m <= 4; ++m) {
          SliceLaunch w = h;
          w.grid = std::min(N, m * cfg->num_sms);
          cand.push_back(w);
          if (w.grid == N) break;
        }
      }
    }
    if (!dbl && cfg->p.variant == 3) {  // the tau-walking kernel only
      std::vector<SliceLaunch> keep;
      for (const SliceLaunch& c : cand)
        if (c.walk) keep.push_back(c);
      cand.swap(keep);
    }
    float best = 1e30f;
    SliceLaunch chosen = dbl ? cfg->fused64 : cfg->fused32;
    for (const SliceLaunch& c : cand) {
      const int rb = dbl ? 8 : 4;
      const int nclus = c.walk ? 1
                        : c.nby > 0 ? mdagm_block_max_active_clusters(c, rb)
                                    : (dbl ? mdagm_max_active_clusters(c) : 1);
      if (c.cluster > 1 && nclus <= 0) continue;
      float us = -1.f;
      RET(dbl ? time_shape<double>(cfg, c, &us) : time_shape<float>(cfg, c, &us));
      if (us > 0.f && us < best) {
        best = us;
        chosen = c;
      }
    }
    if (dbl) {
      cfg->fused64 = chosen;
      cfg->tuned_us64 = best;
    } else {
      cfg->fused32 = chosen;
      cfg->tuned_us32 = best;
    }
  }
  RET(tune_pc_update<double>(cfg));
  RET(tune_line_chunk(cfg));
  RET(tune_pc_update<float>(cfg));
  CK(cudaDeviceSynchronize());
  return HQMC_OK;
}

}  // namespace

extern "C" {

const char* hqmc_strerror(int status) {
  switch (status) {
    case HQMC_OK: return "success";
    case HQMC_EINVAL: return "invalid argument";
    case HQMC_ENOTCONV: return "CG did not converge within maxit";
    case HQMC_EBREAKDOWN: return "CG breakdown (<d, O d> <= 0)";
    case HQMC_ENONFINITE: return "non-finite value in a reduction";
    case HQMC_ETIMEOUT: return "bounded device wait timed out";
    case HQMC_ECUDA: return "CUDA runtime error";
    case HQMC_ENOMEM: return "device allocation failed";
    case HQMC_EUNSUPPORTED: return "unsupported configuration or device";
    case HQMC_EIO: return "checkpoint file error";
    default: return "unknown status";
  }
}

const char* hqmc_last_error(const hqmc_config* cfg) { return cfg ? cfg->err : "no config"; }

long long hqmc_num_sites(const hqmc_config* cfg) { return cfg ? cfg->n : 0; }

long long hqmc_launch_count(const hqmc_config* cfg) { return cfg ? cfg->launches : 0; }

int hqmc_get_launch_shape(const hqmc_config* cfg, int precision, int* variant, int* cluster, int* threads,
                          float* tuned_us) {
  if (!cfg || (precision != HQMC_FP64 && precision != HQMC_FP32)) return HQMC_EINVAL;
  const SliceLaunch& sh = precision == HQMC_FP64 ? cfg->fused64 : cfg->fused32;
  if (variant) *variant = sh.walk ? 100 + sh.nby : sh.nby > 0 ? sh.nby : -sh.mb;
  if (cluster) *cluster = sh.walk ? 1 : sh.cluster;
  if (threads) *threads = sh.threads;
  if (tuned_us) *tuned_us = precision == HQMC_FP64 ? cfg->tuned_us64 : cfg->tuned_us32;
  return HQMC_OK;
}

int hqmc_make_config(const hqmc_params* p, hqmc_config** out) {
  if (!p || !out) return HQMC_EINVAL;
  *out = nullptr;
  if (p->L < 4 || (p->L & 1) || p->L > kMaxL) return HQMC_EINVAL;
  if (p->Ntau < 2) return HQMC_EINVAL;
  if (!(p->dtau > 0) || !std::isfinite(p->dtau) || !std::isfinite(p->t) || !(p->J > 0) ||
      !std::isfinite(p->J) || !std::isfinite(p->K))
    return HQMC_EINVAL;
  if (p->action != HQMC_ACTION_COMPACT && p->action != HQMC_ACTION_NONCOMPACT) return HQMC_EINVAL;
  if (p->variant < 0 || p->variant > 3) return HQMC_EINVAL;
  const long long n = (long long)p->L * p->L * p->Ntau;
  if (n > (1LL << 31) - 1) return HQMC_EINVAL;

  hqmc_config* cfg = new (std::nothrow) hqmc_config();
  if (!cfg) return HQMC_ENOMEM;
  cfg->p = *p;
  int rc = HQMC_OK;
  do {
    cudaError_t e = cudaGetDevice(&cfg->device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, cfg->device);
    if (e != cudaSuccess) {
      rc = fail(cfg, HQMC_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
      break;
    }
    if (prop.major != 10) {
      rc = fail(cfg, HQMC_EUNSUPPORTED, "built for sm_103a; device is sm_%d%d", prop.major, prop.minor);
      break;
    }
    const int L = p->L, V = L * L;
    cfg->g = Geo{L, V, L / 2, p->Ntau};
    cfg->n = n;
    cfg->a = p->dtau * p->t;
    cfg->t1 = std::tanh(cfg->a);
    cfg->t2 = std::tanh(cfg->a / 2);
    cfg->cB = std::cosh(cfg->a) * std::pow(std::cosh(cfg->a / 2), 6);
    cfg->bp.cK = 1.0 / (p->J * p->dtau);
    cfg->bp.Kdtau = p->K * p->dtau;
    cfg->bp.noncompact = p->action == HQMC_ACTION_NONCOMPACT;
    cfg->reliable = p->reliable_interval > 0 ? p->reliable_interval : kDefaultReliable;

    // slice kernels: enough threads for one pass over a family's V/2 bonds; the
    // fused kernel holds mb bonds of every family per thread in registers when
    // a block shape with enough registers exists (mb = 0 otherwise)
    const int bonds = V / 2;
    auto shape = [&](int real_bytes, int* mb_out) {
      for (int mb = 1; mb <= 3; ++mb) {  // mb = 4 would spill registers
        const int th = ((bonds + mb - 1) / mb + 31) / 32 * 32;
        if (th <= sweep_thread_cap(real_bytes, mb)) {
          *mb_out = mb;
          return th < 64 ? 64 : th;
        }
      }
      *mb_out = 0;
      const int rounds = (bonds + 1023) / 1024;
      return ((bonds + rounds - 1) / rounds + 31) / 32 * 32;
    };
    int mb64 = 0, mb32 = 0;
    const int th64 = shape(8, &mb64), th32 = shape(4, &mb32);
    int threads = th64;
    cfg->sl.mb = mb64;
    cfg->sl.g = cfg->g;
    cfg->sl.threads = threads;
    cfg->sl.cluster = p->Ntau < 8 ? p->Ntau : 8;
    cfg->sl1 = cfg->sl;
    cfg->sl1.cluster = 1;
    cfg->sl1.grid = p->Ntau;
    cfg->sl1.mb = 0;
    {
      const int rounds = (bonds + 1023) / 1024;
      cfg->sl1.threads = std::max(64, ((bonds + rounds - 1) / rounds + 31) / 32 * 32);
    }
    // shrink the cluster until the device can co-schedule it
    for (;;) {
      cfg->sl.grid = ((p->Ntau + cfg->sl.cluster - 1) / cfg->sl.cluster) * cfg->sl.cluster;
      if (prepare_mdagm<double, MODE_CGDIR>(cfg->sl) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(cfg, HQMC_EUNSUPPORTED, "cannot configure the M^dagger M kernel for L=%d", L);
        break;
      }
      if (cfg->sl.cluster == 1 || mdagm_max_active_clusters(cfg->sl) > 0) break;
      cfg->sl.cluster--;
    }
    cfg->sl32 = cfg->sl;
    cfg->sl32.mb = mb32;
    cfg->sl32.threads = th32;
    // register-blocked variant: strips of nby 2x2 blocks, (L/2)^2/nby threads
    auto pick_block = [&](int real_bytes, SliceLaunch* out) {
      *out = cfg->sl;
      out->nby = 0;
      const int Lh = L / 2;
      for (int nby = 1; nby <= 3; ++nby) {
        if (Lh % nby) continue;
        const int th = Lh * Lh / nby;
        const int cap = block_thread_cap(real_bytes, nby);
        if (cap <= 0 || th > cap) continue;
        SliceLaunch c = cfg->sl;
        c.nby = nby;
        c.threads = th;
        cudaError_t pe = real_bytes == 8 ? prepare_mdagm_block<double, MODE_CGDIR>(c) : prepare_mdagm_block<float, MODE_CGDIR>(c);
        if (pe == cudaSuccess)
          pe = real_bytes == 8 ? prepare_mdagm_block<double, MODE_APPLY>(c) : prepare_mdagm_block<float, MODE_APPLY>(c);
        if (pe != cudaSuccess || mdagm_block_max_active_clusters(c, real_bytes) <= 0) {
          cudaGetLastError();
          continue;
        }
        *out = c;
        return;
      }
    };
    pick_block(8, &cfg->slb64);
    pick_block(4, &cfg->slb32);
    cfg->num_sms = prop.multiProcessorCount;
    cfg->smem_per_sm = prop.sharedMemPerMultiprocessor;
    // tau-walking FP32 kernel: by default the smallest strip height whose block
    // fits; every height that fits is kept for the autotuner (a taller strip has
    // fewer threads per CTA, and on some lattices two CTAs then share an SM)
    cfg->slw32 = cfg->sl32;
    cfg->slw32.walk = 0;
    {
      const int Lh = L / 2;
      for (int nby = 1; nby <= 3; ++nby) {
        if (Lh % nby) continue;
        const int th = Lh * Lh / nby;
        if (th > walk_thread_cap(nby) || walk_smem_bytes(cfg->g, MODE_CGDIR) > prop.sharedMemPerBlockOptin) continue;
        SliceLaunch c = cfg->sl32;
        c.nby = nby;
        c.threads = th;
        c.cluster = 1;
        c.walk = 1;
        c.grid = std::min(p->Ntau, cfg->num_sms);
        if (prepare_mdagm_walk<MODE_CGDIR>(c) != cudaSuccess || prepare_mdagm_walk<MODE_APPLY>(c) != cudaSuccess ||
            mdagm_walk_blocks_per_sm(c) < 1) {
          cudaGetLastError();
          continue;
        }
        cfg->slw32h[nby - 1] = c;
        if (!cfg->slw32.walk) cfg->slw32 = c;
      }
    }
    // variant 1 keeps the generic kernel, 2 demands the register-blocked one
    if (p->variant == 1) {
      cfg->slb64.nby = 0;
      cfg->slb32.nby = 0;
      cfg->slw32.walk = 0;
    } else if (p->variant == 2) {
      cfg->slw32.walk = 0;
      if (cfg->slb64.nby == 0 || cfg->slb32.nby == 0) {
        rc = fail(cfg, HQMC_EUNSUPPORTED, "no register-blocked shape fits L=%d", L);
        break;
      }
    } else if (p->variant == 3 && !cfg->slw32.walk) {
      rc = fail(cfg, HQMC_EUNSUPPORTED, "no tau-walking shape fits L=%d", L);
      break;
    }
    // default shapes: FP32 the tau-walking kernel, else the register-blocked one,
    // where they fit (the autotuner may override)
    cfg->fused64 = cfg->slb64.nby > 0 ? cfg->slb64 : cfg->sl;
    cfg->fused32 = cfg->slw32.walk ? cfg->slw32 : cfg->slb32.nby > 0 ? cfg->slb32 : cfg->sl32;
    if (rc != HQMC_OK) break;
    if (prepare_mdagm<double, MODE_APPLY>(cfg->sl) != cudaSuccess ||
        prepare_mdagm<double, MODE_RESID>(cfg->sl) != cudaSuccess ||
        prepare_mdagm<float, MODE_APPLY>(cfg->sl32) != cudaSuccess ||
        prepare_mdagm<float, MODE_CGDIR>(cfg->sl32) != cudaSuccess || prepare_apply_M<double>(cfg->sl1) != cudaSuccess ||
        prepare_apply_M<float>(cfg->sl1) != cudaSuccess || prepare_force(cfg->sl1) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(cfg, HQMC_EUNSUPPORTED, "cannot configure slice kernels for L=%d", L);
      break;
    }
    {
      long long b = (n + 255) / 256;
      cfg->ew_grid = (int)(b < 1024 ? b : 1024);
      cfg->act_grid = (int)(b < 512 ? b : 512);
    }
    // workspace
    if ((rc = dalloc(cfg, &cfg->U64, 2 * n))) break;
    if ((rc = dalloc(cfg, &cfg->U32, 2 * n))) break;
    if ((rc = dalloc(cfg, &cfg->th32, n))) break;
    if ((rc = dalloc(cfg, &cfg->r64, n))) break;
    if ((rc = dalloc(cfg, &cfg->p64[0], n))) break;
    if ((rc = dalloc(cfg, &cfg->p64[1], n))) break;
    if ((rc = dalloc(cfg, &cfg->q64, n))) break;
    if ((rc = dalloc(cfg, &cfg->r32, n))) break;
    if ((rc = dalloc(cfg, &cfg->p32[0], n))) break;
    if ((rc = dalloc(cfg, &cfg->p32[1], n))) break;
    if ((rc = dalloc(cfg, &cfg->q32, n))) break;
    if ((rc = dalloc(cfg, &cfg->xh32, n))) break;
    if ((rc = dalloc(cfg, &cfg->eta, n))) break;
    if ((rc = dalloc(cfg, &cfg->Xw, n))) break;
    if ((rc = dalloc(cfg, &cfg->Rw, n))) break;
    if ((rc = dalloc(cfg, &cfg->vscratch, n))) break;
    if ((rc = dalloc(cfg, &cfg->dSf, 2 * n))) break;
    if ((rc = dalloc(cfg, &cfg->F, 2 * n))) break;
    if ((rc = dalloc(cfg, &cfg->th0, 2 * n))) break;
    if ((rc = dalloc(cfg, &cfg->pm, 2 * n))) break;
    // partials of the fused kernel: room for any cluster size (grid <= Ntau + 7)
    if ((rc = dalloc(cfg, &cfg->part_mdagm, 2 * ((size_t)p->Ntau + 8)))) break;
    if ((rc = dalloc(cfg, &cfg->part_resid, 2 * ((size_t)p->Ntau + 8)))) break;
    // preconditioner tiles: the FP32 height is set with the coefficients; partials
    // have room for the smallest height any config picks (16 slices)
    cfg->ll64 = line_update_launch(cfg->g, 8);
    cfg->ll32 = line_update_launch(cfg->g, 4);
    cfg->llu64 = line_update_launch(cfg->g, 8);
    cfg->llu32 = line_update_launch(cfg->g, 4);
    const LineLaunch l16 = line_launch(cfg->g, 16);
    cfg->n_part_ew = std::max(cfg->ew_grid, std::max(cfg->llu64.gx * cfg->llu64.gy, cfg->llu32.gx * cfg->llu32.gy));
    if ((rc = dalloc(cfg, &cfg->part_ew, (size_t)cfg->n_part_ew))) break;
    if ((rc = dalloc(cfg, &cfg->part_act, 4 * (size_t)cfg->act_grid))) break;
    if ((rc = dalloc(cfg, &cfg->z64, n))) break;
    if ((rc = dalloc(cfg, &cfg->z32, n))) break;
    if ((rc = dalloc(cfg, &cfg->r64b, n))) break;
    if ((rc = dalloc(cfg, &cfg->r32b, n))) break;
    if ((rc = dalloc(cfg, &cfg->part_rz,
                     (size_t)std::max(l16.gx * l16.gy, cfg->llu32.gx * cfg->llu32.gy)))) break;
    if ((rc = dalloc(cfg, &cfg->terms, 8))) break;
    if ((rc = dalloc(cfg, &cfg->report, 2))) break;
    if ((rc = dalloc(cfg, &cfg->st, 1))) break;
    if ((rc = dalloc(cfg, &cfg->dev_err, 1))) break;
    if (cudaMallocHost(&cfg->st_h, sizeof(CgState)) != cudaSuccess ||
        cudaMallocHost(&cfg->dev_err_h, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&cfg->terms_h, 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&cfg->report_h, 2 * sizeof(double)) != cudaSuccess) {
      rc = fail(cfg, HQMC_ENOMEM, "pinned host allocation failed");
      break;
    }
    if (cudaStreamCreateWithFlags(&cfg->cap, cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(cfg, HQMC_ECUDA, "stream creation failed");
      break;
    }
    cudaMemset(cfg->st, 0, sizeof(CgState));
    cudaMemset(cfg->report, 0, 2 * sizeof(double));
    cudaMemset(cfg->dev_err, 0, sizeof(int));
    *cfg->dev_err_h = 0;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      rc = fail(cfg, HQMC_ECUDA, "workspace initialisation failed: %s", cudaGetErrorString(e));
      break;
    }
    if ((rc = line_coefficients(cfg)) != HQMC_OK) break;
    cfg->fuse_pc64 = cfg->fuse_pc32 = n <= kFuseMaxSites ? 1 : 0;
    if (p->autotune && (rc = autotune(cfg)) != HQMC_OK) break;
  } while (0);
  if (rc != HQMC_OK) {
    release(cfg);
    delete cfg;
    return rc;
  }
  *out = cfg;
  return HQMC_OK;
}

int hqmc_free_config(hqmc_config* cfg) {
  if (!cfg) return HQMC_OK;
  cudaDeviceSynchronize();
  release(cfg);
  delete cfg;
  return HQMC_OK;
}

int hqmc_apply_M(hqmc_config* cfg, const double* theta, const void* x, void* y, int dagger, int precision,
                 void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(x) || !aligned16(y)) return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  if (precision != HQMC_FP64 && precision != HQMC_FP32) return fail(cfg, HQMC_EINVAL, "bad precision");
  const size_t vb = cfg->n * (precision == HQMC_FP64 ? sizeof(double2) : sizeof(float2));
  if (overlap(x, vb, y, vb)) return fail(cfg, HQMC_EINVAL, "x and y overlap");
  RET(check_device(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == HQMC_FP64) {
    RET(links(cfg, theta, true, false, s));
    LK(1, launch_apply_M<double>(cfg->sl1, cfg->cB, cfg->U64, (const double2*)x, (double2*)y, dagger ? 1 : 0, s));
  } else {
    RET(links(cfg, theta, false, false, s, true));
    LK(1, launch_apply_M<float>(cfg->sl1, (float)cfg->cB, cfg->U32, (const float2*)x, (float2*)y, dagger ? 1 : 0, s));
  }
  return HQMC_OK;
}

int hqmc_apply_MdagM(hqmc_config* cfg, const double* theta, const void* x, void* y, int precision, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(x) || !aligned16(y)) return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  if (precision != HQMC_FP64 && precision != HQMC_FP32) return fail(cfg, HQMC_EINVAL, "bad precision");
  const size_t vb = cfg->n * (precision == HQMC_FP64 ? sizeof(double2) : sizeof(float2));
  if (overlap(x, vb, y, vb)) return fail(cfg, HQMC_EINVAL, "x and y overlap");
  RET(check_device(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  int slot;
  if (precision == HQMC_FP64) {
    RET(links(cfg, theta, true, false, s));
    MdagmArgs<double> a = mdagm_args<double, MODE_APPLY>(cfg);
    a.U = cfg->U64;
    a.x = (const double2*)x;
    a.y = (double2*)y;
    RET(timer_begin(cfg, HQMC_TIMER_MDAGM, s, &slot));
    LK(1, (launch_fused<double, MODE_APPLY>(cfg, a, s)));
    RET(timer_end(cfg, HQMC_TIMER_MDAGM, s, slot));
  } else {
    RET(links(cfg, theta, false, true, s));
    MdagmArgs<float> a = mdagm_args<float, MODE_APPLY>(cfg);
    a.U = cfg->U32;
    a.x = (const float2*)x;
    a.y = (float2*)y;
    RET(timer_begin(cfg, HQMC_TIMER_MDAGM32, s, &slot));
    LK(1, (launch_fused<float, MODE_APPLY>(cfg, a, s)));
    RET(timer_end(cfg, HQMC_TIMER_MDAGM32, s, slot));
  }
  return HQMC_OK;
}

int hqmc_apply_precond(hqmc_config* cfg, const void* r, void* z, int precision, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(r) || !aligned16(z)) return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  if (precision != HQMC_FP64 && precision != HQMC_FP32) return fail(cfg, HQMC_EINVAL, "bad precision");
  const size_t vb = cfg->n * (precision == HQMC_FP64 ? sizeof(double2) : sizeof(float2));
  if (overlap(r, vb, z, vb)) return fail(cfg, HQMC_EINVAL, "r and z overlap");
  RET(check_device(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == HQMC_FP64)
    RET(precondition<double>(cfg, (const double2*)r, (double2*)z, nullptr, s));
  else
    RET(precondition<float>(cfg, (const float2*)r, (float2*)z, nullptr, s));
  return HQMC_OK;
}

int hqmc_get_precond(const hqmc_config* cfg, double* a, double* b, double* rho, int* W) {
  if (!cfg) return HQMC_EINVAL;
  if (a) *a = cfg->pc_a;
  if (b) *b = cfg->pc_b;
  if (rho) *rho = cfg->lc.rho;
  if (W) *W = cfg->lc.W;
  return HQMC_OK;
}

int hqmc_get_precond_shape(const hqmc_config* cfg, int precision, int* tile_slices, int* fused) {
  if (!cfg || (precision != HQMC_FP64 && precision != HQMC_FP32)) return HQMC_EINVAL;
  const bool dbl = precision == HQMC_FP64;
  if (tile_slices) *tile_slices = dbl ? cfg->ll64.chunk : cfg->ll32.chunk;
  if (fused) *fused = (dbl ? cfg->fuse_pc64 : cfg->fuse_pc32) && cfg->p.variant != 1 ? 1 : 0;
  return HQMC_OK;
}

int hqmc_set_precond_fused(hqmc_config* cfg, int precision, int fused) {
  if (!cfg || (precision != HQMC_FP64 && precision != HQMC_FP32) || (fused != 0 && fused != 1)) return HQMC_EINVAL;
  if (fused && cfg->p.variant == 1) return fail(cfg, HQMC_EUNSUPPORTED, "variant 1 keeps the separate update");
  (precision == HQMC_FP64 ? cfg->fuse_pc64 : cfg->fuse_pc32) = fused;
  CK(cudaDeviceSynchronize());  // no cached loop graph may still be running
  for (auto& g : cfg->graphs) cudaGraphExecDestroy(g.exec);  // loop bodies change shape
  cfg->graphs.clear();
  return HQMC_OK;
}

int hqmc_cg_solve(hqmc_config* cfg, const double* theta, const void* phi, void* x, double tol, int maxit, int solver,
                  hqmc_solve_info* info, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(phi) || !aligned16(x)) return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  if (!(tol > 0) || maxit < 0) return fail(cfg, HQMC_EINVAL, "tol must be > 0 and maxit >= 0");
  if (overlap(phi, cfg->n * 16, x, cfg->n * 16)) return fail(cfg, HQMC_EINVAL, "phi and x overlap");
  RET(check_solver(cfg, solver));
  RET(check_device(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  RET(links(cfg, theta, true, solver_fp32(solver), s, false, solver_base(solver) == HQMC_SOLVER_LEARNED));
  return solve(cfg, (const double2*)phi, (double2*)x, tol, maxit, solver, info, s);
}

}  // extern "C"

namespace {

// Stochastic estimation (Methods, "Stochastic estimation of fermionic observables").
// project: every solve after the first starts from the Galerkin projection of its
// solution onto the earlier solutions X_0..X_{k-1} (all on the same field):
// x0 = sum_i c_i X_i with G c = (<X_i, R_k>)_i, G_ij = <X_i, O X_j> = <X_i, R_j>.
// The low modes of O, which dominate every solution and set the iteration count,
// are then mostly present in x0.  Needs the solutions stored (Gxi).
int estimate_impl(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter, int nrv, double tol,
                  int maxit, int solver, void* Gxi, void* xi, double* g_host, hqmc_solve_info* infos, bool project,
                  cudaStream_t s) {
  NvtxRange nv("hqmc estimate");
  RET(links(cfg, theta, true, solver_fp32(solver), s, false, solver_base(solver) == HQMC_SOLVER_LEARNED));
  const size_t vb = (size_t)cfg->n * sizeof(double2);
  double sum_re = 0.0, sum_im = 0.0;
  int status = HQMC_OK;
  double2* prev = nullptr;
  // projection workspace: the many-dot partials and results in the scratch vector
  const int grid = cfg->act_grid;
  double* dscratch = reinterpret_cast<double*>(cfg->vscratch);
  const bool room = 2 * (size_t)grid * nrv + 2 * (size_t)nrv <= 2 * (size_t)cfg->n;
  std::vector<double> G(project ? 2 * (size_t)nrv * nrv : 0, 0.0);
  std::vector<double> col, A;
  for (int k = 0; k < nrv; ++k) {
    double2* v = xi ? (double2*)xi + (size_t)k * cfg->n : cfg->Rw;           // xi_k
    double2* X = Gxi ? (double2*)Gxi + (size_t)k * cfg->n : cfg->Xw;          // M^{-1} xi_k
    LK(1, launch_draw_vector(cfg->n, seed, 3u, counter + (uint64_t)k, v, s));
    LK(1, launch_apply_M<double>(cfg->sl1, cfg->cB, cfg->U64, v, cfg->eta, 1, s));  // R = M^dagger xi
    bool guessed = false;
    if (project && k > 0 && room) {
      const double2* X0 = (const double2*)Gxi;
      LK(2, launch_cdot_many(cfg->n, X0, cfg->n, k, cfg->eta, grid, dscratch, dscratch + 2 * (size_t)grid * k, s));
      col.assign(2 * (size_t)k, 0.0);
      CK(cudaMemcpyAsync(col.data(), dscratch + 2 * (size_t)grid * k, 2 * (size_t)k * sizeof(double),
                         cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      A.assign(2 * (size_t)k * k, 0.0);
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
          A[2 * (i * k + j)] = G[2 * (i * nrv + j)];
          A[2 * (i * k + j) + 1] = G[2 * (i * nrv + j) + 1];
        }
      std::vector<double> c = col;
      if (hermitian_solve(k, A, c)) {
        CK(cudaMemsetAsync(X, 0, vb, s));
        for (int i = 0; i < k; ++i)
          LK(1, launch_caxpy(cfg->n, c[2 * i], c[2 * i + 1], X0 + (size_t)i * cfg->n, X, s));
        guessed = true;
      }
      for (int i = 0; i < k; ++i) {  // G_ik = <X_i, R_k>, G_ki = conj(G_ik)
        G[2 * (i * nrv + k)] = col[2 * i];
        G[2 * (i * nrv + k) + 1] = col[2 * i + 1];
        G[2 * (k * nrv + i)] = col[2 * i];
        G[2 * (k * nrv + i) + 1] = -col[2 * i + 1];
      }
    }
    if (!guessed) {
      if (k == 0)
        CK(cudaMemsetAsync(X, 0, vb, s));
      else if (prev != X)
        CK(cudaMemcpyAsync(X, prev, vb, cudaMemcpyDeviceToDevice, s));  // start from the previous solution
    }
    hqmc_solve_info si{};
    const int rc = solve(cfg, cfg->eta, X, tol, maxit, solver, &si, s);
    if (rc != HQMC_OK && rc != HQMC_ENOTCONV) return rc;
    status = merge_status(status, rc);
    if (infos) infos[k] = si;
    LK(2, launch_cdot(cfg->n, v, X, cfg->act_grid, cfg->part_act, cfg->terms + 4, s));
    if (project) LK(2, launch_cdot(cfg->n, X, cfg->eta, cfg->act_grid, cfg->part_act, cfg->terms + 6, s));
    CK(cudaMemcpyAsync(cfg->terms_h + 4, cfg->terms + 4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    sum_re += cfg->terms_h[4];
    sum_im += cfg->terms_h[5];
    if (project) {
      G[2 * (k * nrv + k)] = cfg->terms_h[6];  // <X_k, R_k> (real up to the solve's tolerance)
      G[2 * (k * nrv + k) + 1] = 0.0;
    }
    prev = X;
  }
  if (g_host) {
    const double norm = 1.0 / ((double)nrv * (double)cfg->n);
    g_host[0] = sum_re * norm;
    g_host[1] = sum_im * norm;
  }
  return status;
}

// ---------------------------------------------------------------------------
// Systems solved together on one field (the N_rv right-hand sides of the
// stochastic estimation, Methods "Stochastic estimation of fermionic
// observables"): mixed-precision CG of Eq. (pCG) on every system at once, with
// per iteration one tau-walking M^dagger M launch, one update launch and (PMIXED)
// one preconditioner launch for all of them, and per loop body the FP64
// reliable updates of all of them in one launch.  Every system keeps its own
// scalars, state and convergence test; the systems share theta and its tables.

// The tau-walking shape of a multi-system launch (walk = 0: none).
SliceLaunch multi_walk_shape(const hqmc_config* cfg) {
  return cfg->fused32.walk ? cfg->fused32 : cfg->slw32;
}

// Slice ranges per system of a launch over nsys systems (multi_shape.h), unless
// hqmc_set_multi_ranges fixed them.
int multi_granges(const hqmc_config* cfg, int nsys) {
  const SliceLaunch w = multi_walk_shape(cfg);
  const int N = cfg->p.Ntau;
  if (cfg->multi_ranges > 0) return std::min(cfg->multi_ranges, N);
  const long long R = (long long)std::max(1, cfg->num_sms) * std::max(1, mdagm_walk_multi_blocks_per_sm(w));
  return multi_ranges_model(N, nsys, R);
}

// Shared memory of the systems' FP64 residual (the batched generic kernel: links
// from the FP64 table, clusters of consecutive slices).
size_t multi_res_smem(const hqmc_config* cfg) { return (size_t)3 * cfg->g.V * sizeof(double2); }

template <class T>
int mdalloc(hqmc_config* cfg, T** ptr, size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(cfg, HQMC_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  }
  cfg->mw.allocs.push_back(p);
  *ptr = (T*)p;
  return HQMC_OK;
}

// Allocates the workspace of `cap` systems and the descriptor tables that do not
// depend on the operands of a call.
int multi_setup(hqmc_config* cfg, int cap) {
  MultiWs& m = cfg->mw;
  const size_t n = (size_t)cfg->n;
  const int N = cfg->p.Ntau;
  const LineLaunch& ll = cfg->ll32;
  m.cap = cap;
  // update: about two resident waves of 256-thread blocks over all systems, so each
  // block streams enough of its vector to hide the latency of its head (state and
  // partial sums); at most the one-system grid
  {
    const long long resident = (long long)cfg->num_sms * std::max(1, cg_update_multi_blocks_per_sm());
    m.ublocks = (int)std::max(8LL, std::min((long long)cfg->ew_grid, 2 * resident / cap));
  }
  m.pstride = std::max(N, std::max(m.ublocks, ll.gx * ll.gy));
  m.nlt = ll.gx * ll.gy;
  // FP64 residual: the cluster size of the one-system residual where the batched
  // generic kernel can co-schedule it (a cluster of C slices does 2C + 1 sweeps)
  {
    const SliceLaunch& rs = (cfg->fused64.nby == 0 && cfg->fused64.mb == cfg->sl.mb) ? cfg->fused64 : cfg->sl;
    m.rC = std::max(1, std::min(rs.cluster, N));
    if (m.rC > 1 && mdagm_batch_max_active_clusters(m.rC, cfg->sl.threads, multi_res_smem(cfg)) <= 0) m.rC = 1;
    m.rnt = (N + m.rC - 1) / m.rC;
    m.rslots = m.rnt * m.rC;
    m.rstride = 2 * m.rslots;
  }
  const size_t vc = (size_t)cap * n;
  RET(mdalloc(cfg, &m.r, vc));
  RET(mdalloc(cfg, &m.p0, vc));
  RET(mdalloc(cfg, &m.p1, vc));
  RET(mdalloc(cfg, &m.q, vc));
  RET(mdalloc(cfg, &m.z, vc));
  RET(mdalloc(cfg, &m.xh, vc));
  RET(mdalloc(cfg, &m.eta, vc));
  RET(mdalloc(cfg, &m.xw, vc));
  RET(mdalloc(cfg, &m.xiw, vc));
  RET(mdalloc(cfg, &m.part_w, (size_t)cap * m.pstride));
  RET(mdalloc(cfg, &m.part_ew, (size_t)cap * m.pstride));
  RET(mdalloc(cfg, &m.part_rz, (size_t)cap * m.pstride));
  RET(mdalloc(cfg, &m.part_res, (size_t)cap * m.rstride));
  RET(mdalloc(cfg, &m.report, 2 * (size_t)cap));
  RET(mdalloc(cfg, &m.st, (size_t)cap));
  RET(mdalloc(cfg, &m.d_states, (size_t)cap));
  RET(mdalloc(cfg, &m.d_line, (size_t)cap));
  RET(mdalloc(cfg, &m.d_ltiles, (size_t)cap * m.nlt));
  RET(mdalloc(cfg, &m.d_res, 2 * (size_t)cap));
  RET(mdalloc(cfg, &m.d_fin, (size_t)cap));
  RET(mdalloc(cfg, &m.d_rtiles, (size_t)cap * m.rnt));
  CK(cudaMallocHost((void**)&m.st_h, (size_t)cap * sizeof(CgState)));
  CK(cudaMallocHost((void**)&m.report_h, 2 * (size_t)cap * sizeof(double)));
  m.stage_bytes = (size_t)cap * (2 * sizeof(MdagmArgs<double>) + sizeof(FinArgs));
  CK(cudaMallocHost(&m.h_stage, m.stage_bytes));
  CK(cudaMemset(m.st, 0, (size_t)cap * sizeof(CgState)));
  CK(cudaMemset(m.part_w, 0, (size_t)cap * m.pstride * sizeof(double)));
  CK(cudaMemset(m.part_ew, 0, (size_t)cap * m.pstride * sizeof(double)));
  CK(cudaMemset(m.part_rz, 0, (size_t)cap * m.pstride * sizeof(double)));
  // fixed tables, system-major (the first nsys systems' entries are a prefix)
  std::vector<CgState*> states(cap);
  std::vector<int2> rtiles;
  std::vector<LineBatchDesc<float>> line(cap);
  std::vector<int4> ltiles;
  for (int k = 0; k < cap; ++k) {
    states[k] = m.st + k;
    for (int t = 0; t < N; t += m.rC) rtiles.push_back(make_int2(k, t));
    line[k] = LineBatchDesc<float>{cfg->g, cfg->lc, m.r + k * n, m.z + k * n, m.part_rz + (size_t)k * m.pstride,
                                   m.st + k, ll.gx, ll.chunk};
    for (int by = 0; by < ll.gy; ++by)
      for (int bx = 0; bx < ll.gx; ++bx) ltiles.push_back(make_int4(k, bx, by, 0));
  }
  CK(cudaMemcpy(m.d_states, states.data(), cap * sizeof(CgState*), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m.d_line, line.data(), cap * sizeof(LineBatchDesc<float>), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m.d_ltiles, ltiles.data(), ltiles.size() * sizeof(int4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m.d_rtiles, rtiles.data(), rtiles.size() * sizeof(int2), cudaMemcpyHostToDevice));
  if (prepare_mdagm_walk_multi(multi_walk_shape(cfg)) != cudaSuccess ||
      prepare_line_precond_batch32(cfg->lc.W, ll.chunk) != cudaSuccess) {
    cudaGetLastError();
    return fail(cfg, HQMC_EUNSUPPORTED, "cannot configure the multi-system kernels for L=%d", cfg->p.L);
  }
  return HQMC_OK;
}

// One loop body over nsys systems: `reliable` mixed iterations, then the FP64
// reliable update of every active system and (PMIXED) its preconditioned residual.
int multi_body(hqmc_config* cfg, int nsys, bool pc, const SliceLaunch& wl, double2* x, cudaStream_t s, int* nk) {
  MultiWs& m = cfg->mw;
  MdagmArgs<float> a = mdagm_args<float, MODE_CGDIR>(cfg);
  a.U = cfg->U32;
  a.y = m.q;
  a.r = pc ? m.z : m.r;
  a.pbuf[0] = m.p0;
  a.pbuf[1] = m.p1;
  a.part_in = m.part_ew;
  a.n_part_in = m.ublocks;
  if (pc) {
    a.part_rz = m.part_rz;
    a.n_part_rz = m.nlt;
  }
  a.part_out = m.part_w;
  a.st = m.st;
  const MultiStride ms{nsys, cfg->n, m.pstride};
  const UpdArgs<float> upd{cfg->n, m.xh, 0, m.r, m.p0, m.p1, m.q, m.part_w, wl.grid, m.part_ew, m.st};
  const int iters = cfg->reliable;
  int slot;
  for (int c = 0; c < iters; ++c) {
    RET(timer_begin(cfg, HQMC_TIMER_MDAGM32, s, &slot));
    CK(launch_mdagm_walk_multi(wl, a, ms, s));
    RET(timer_end(cfg, HQMC_TIMER_MDAGM32, s, slot));
    RET(timer_begin(cfg, HQMC_TIMER_CG_UPDATE, s, &slot));
    CK(launch_cg_update_multi(upd, cfg->n, m.pstride, nsys, m.ublocks, s));
    RET(timer_end(cfg, HQMC_TIMER_CG_UPDATE, s, slot));
    if (pc) {
      RET(timer_begin(cfg, HQMC_TIMER_PRECOND, s, &slot));
      CK(launch_line_precond_batch(m.d_line, m.d_ltiles, nsys * m.nlt, cfg->lc.W, cfg->ll32.chunk, s));
      RET(timer_end(cfg, HQMC_TIMER_PRECOND, s, slot));
    }
  }
  CK(launch_accumulate_correction_multi(cfg->n, nsys, x, m.xh, m.st, GATE_ACTIVE, s));
  CK((launch_mdagm_batch<double, MODE_RESID>(m.d_res + m.cap, m.d_rtiles, nsys * m.rnt, m.rC, cfg->sl.threads,
                                             multi_res_smem(cfg), s)));
  CK(launch_resid_finalize_batch(m.d_fin, nsys, FIN_RELIABLE, 0.0, 0, GATE_ACTIVE, s));
  if (pc) CK(launch_line_precond_batch(m.d_line, m.d_ltiles, nsys * m.nlt, cfg->lc.W, cfg->ll32.chunk, s));
  *nk = (pc ? 3 : 2) * iters + 3 + (pc ? 1 : 0);
  return HQMC_OK;
}

// The WHILE-node graph of multi_body for (nsys, solver, ranges, x), built once.
int multi_graph(hqmc_config* cfg, int nsys, bool pc, const SliceLaunch& wl, double2* x, MultiWs::Graph** out) {
  MultiWs& m = cfg->mw;
  for (auto& g : m.graphs)
    if (g.nsys == nsys && g.pc == (int)pc && g.granges == wl.grid && g.x == x) {
      *out = &g;
      return HQMC_OK;
    }
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(cfg, HQMC_ECUDA, "conditional graph node: %s", cudaGetErrorString(e));
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(cfg->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cfg->capturing = 1;
  int nk = 0;
  int rc = multi_body(cfg, nsys, pc, wl, x, cfg->cap, &nk);
  if (rc == HQMC_OK) {
    cudaError_t le = launch_loop_condition_batch(m.d_states, nsys, handle, cfg->cap);
    if (le != cudaSuccess) rc = fail(cfg, HQMC_ECUDA, "loop condition launch: %s", cudaGetErrorString(le));
  }
  cfg->capturing = 0;
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cfg->cap, &captured);
  if (rc == HQMC_OK && e != cudaSuccess) rc = fail(cfg, HQMC_ECUDA, "end capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  if (rc == HQMC_OK) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) rc = fail(cfg, HQMC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  cudaGraphDestroy(graph);
  if (rc != HQMC_OK) {
    cudaGetLastError();
    return rc;
  }
  if (m.graphs.size() >= 4) {
    cudaGraphExecDestroy(m.graphs.front().exec);
    m.graphs.erase(m.graphs.begin());
  }
  m.graphs.push_back(MultiWs::Graph{nsys, (int)pc, wl.grid, x, nk + 1, exec});
  *out = &m.graphs.back();
  return HQMC_OK;
}

// Solves (M^dagger M) x_k = phi_k, k < nsys <= cap, on the field whose tables are
// built (FP64 links and theta as float).  x holds the guesses on entry.  A system
// the joint loop leaves unconverged (breakdown, stagnation or a non-finite value
// of its FP32 recurrence) is finished alone by solve() from its current iterate,
// with that solver's restarts and FP64 fallback.
int solve_multi(hqmc_config* cfg, int nsys, const double2* phi, double2* x, double tol, int maxit, int solver,
                hqmc_solve_info* infos, cudaStream_t s) {
  NvtxRange nv("hqmc multi-system cg solve");
  MultiWs& m = cfg->mw;
  const bool pc = solver_pc(solver);
  const size_t n = (size_t)cfg->n;
  SliceLaunch wl = multi_walk_shape(cfg);
  wl.grid = multi_granges(cfg, nsys);
  // per-call descriptors: FP64 residuals (start, reliable update) and their bookkeeping
  std::vector<MdagmArgs<double>> res(2 * (size_t)nsys);
  std::vector<FinArgs> fin(nsys);
  for (int k = 0; k < nsys; ++k) {
    MdagmArgs<double> r = mdagm_args<double, MODE_RESID>(cfg);
    r.U = cfg->U64;
    r.x = x + k * n;
    r.b = phi + k * n;
    r.r_out = m.r + k * n;
    r.r_out_fp32 = 1;
    r.part_out = m.part_res + (size_t)k * m.rstride;
    r.st = m.st + k;
    r.teff = cfg->sl.threads;
    r.gate = GATE_ALWAYS;
    res[k] = r;
    r.gate = GATE_ACTIVE;
    res[nsys + k] = r;
    fin[k] = FinArgs{m.part_res + (size_t)k * m.rstride, m.rslots, m.part_ew + (size_t)k * m.pstride,
                     m.ublocks, m.st + k, m.report + 2 * k};
  }
  // staged through pinned memory (the previous call synchronised, so its copies are done)
  char* hs = (char*)m.h_stage;
  std::memcpy(hs, res.data(), 2 * (size_t)nsys * sizeof(MdagmArgs<double>));
  char* hf = hs + 2 * (size_t)m.cap * sizeof(MdagmArgs<double>);
  std::memcpy(hf, fin.data(), nsys * sizeof(FinArgs));
  CK(cudaMemcpyAsync(m.d_res, hs, nsys * sizeof(MdagmArgs<double>), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m.d_res + m.cap, hs + nsys * sizeof(MdagmArgs<double>), nsys * sizeof(MdagmArgs<double>),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m.d_fin, hf, nsys * sizeof(FinArgs), cudaMemcpyHostToDevice, s));
  // start: r_k = phi_k - O x_k in FP64 (stored as float), states, corrections zero, z_k
  LK(1, (launch_mdagm_batch<double, MODE_RESID>(m.d_res, m.d_rtiles, nsys * m.rnt, m.rC, cfg->sl.threads,
                                                multi_res_smem(cfg), s)));
  LK(1, launch_resid_finalize_batch(m.d_fin, nsys, FIN_START, tol, maxit, GATE_ALWAYS, s));
  CK(cudaMemsetAsync(m.xh, 0, (size_t)nsys * n * sizeof(float2), s));
  if (pc) LK(1, launch_line_precond_batch(m.d_line, m.d_ltiles, nsys * m.nlt, cfg->lc.W, cfg->ll32.chunk, s));
  auto read_states = [&]() -> int {
    CK(cudaMemcpyAsync(m.st_h, m.st, nsys * sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(m.report_h, m.report, 2 * (size_t)nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return HQMC_OK;
  };
  if (!cfg->timing) {  // the device-side loop
    MultiWs::Graph* gr = nullptr;
    RET(multi_graph(cfg, nsys, pc, wl, x, &gr));
    CK(cudaGraphLaunch(gr->exec, s));
    RET(read_states());
    cfg->launches += (long long)m.st_h[0].loops * gr->body_kernels;
  } else {  // event timing around every launch: bodies enqueued from the host
    const long long cap_bodies = 2LL * maxit / std::max(1, cfg->reliable) + 64;
    for (long long b = 0;; ++b) {
      RET(read_states());
      bool run = false;
      for (int k = 0; k < nsys; ++k) run = run || m.st_h[k].done == CG_RUNNING || m.st_h[k].done == CG_REC_CONVERGED;
      if (!run || b >= cap_bodies) break;
      int nk = 0;
      RET(multi_body(cfg, nsys, pc, wl, x, s, &nk));
      cfg->launches += nk;
    }
  }
  int worst = HQMC_OK;
  for (int k = 0; k < nsys; ++k) {
    const CgState st = m.st_h[k];
    hqmc_solve_info inf{};
    inf.iterations = st.k;
    inf.reliable_updates = st.n_rel;
    int status = HQMC_OK;
    if (st.bb == 0.0) {  // phi_k = 0: the solution is zero whatever the guess
      CK(cudaMemsetAsync(x + k * n, 0, n * sizeof(double2), s));
    } else if (st.done == CG_CONVERGED) {
      inf.true_residual = std::sqrt(m.report_h[2 * k] / st.bb);
      const double rr_rec = (pc && st.k > st.seg_start) ? st.rr_rec : st.rr[st.k & 1];
      inf.recursive_residual = std::sqrt(rr_rec / st.bb);
    } else {
      // fold in the correction the joint loop left, then finish this system alone
      LK(1, launch_accumulate_correction(cfg->n, x + k * n, m.xh + k * n, nullptr, GATE_ALWAYS, s));
      hqmc_solve_info si{};
      status = solve(cfg, phi + k * n, x + k * n, tol, std::max(0, maxit - st.k), solver, &si, s);
      if (status != HQMC_OK && status != HQMC_ENOTCONV && status != HQMC_EBREAKDOWN && status != HQMC_ENONFINITE &&
          status != HQMC_ETIMEOUT)
        return status;
      inf = si;
      inf.iterations += st.k;
      inf.reliable_updates += st.n_rel;
      inf.restarts += 1;
    }
    inf.status = status;
    if (status == HQMC_OK && !(inf.true_residual <= tol)) status = inf.status = HQMC_ENOTCONV;
    if (infos) infos[k] = inf;
    worst = merge_status(worst, status);
  }
  return worst;
}

int check_multi(hqmc_config* cfg, int nsys, int solver, double tol, int maxit) {
  if (cfg->mw.cap < 1) return fail(cfg, HQMC_EINVAL, "no multi-system workspace: call hqmc_set_multi_rhs first");
  if (solver != HQMC_SOLVER_MIXED && solver != HQMC_SOLVER_PMIXED)
    return fail(cfg, HQMC_EUNSUPPORTED, "systems solved together take HQMC_SOLVER_MIXED or HQMC_SOLVER_PMIXED");
  if (!(tol > 0) || maxit < 0) return fail(cfg, HQMC_EINVAL, "tol must be > 0 and maxit >= 0");
  if (nsys < 1) return fail(cfg, HQMC_EINVAL, "at least one system is needed");
  return HQMC_OK;
}

// The estimate of hqmc_estimate with its right-hand sides solved in groups of up
// to cap systems (solve_multi), each from X = 0.  The draws, R_k and the traces
// are those of hqmc_estimate.
int estimate_multi(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter, int nrv, double tol,
                   int maxit, int solver, void* Gxi, void* xi, double* g_host, hqmc_solve_info* infos,
                   cudaStream_t s) {
  NvtxRange nv("hqmc estimate (systems together)");
  MultiWs& m = cfg->mw;
  const size_t n = (size_t)cfg->n;
  RET(links(cfg, theta, true, true, s, false, true));
  double sum_re = 0.0, sum_im = 0.0;
  int status = HQMC_OK;
  for (int g0 = 0; g0 < nrv; g0 += m.cap) {
    const int ns = std::min(m.cap, nrv - g0);
    double2* X = Gxi ? (double2*)Gxi + (size_t)g0 * n : m.xw;
    for (int k = 0; k < ns; ++k) {
      double2* v = xi ? (double2*)xi + (size_t)(g0 + k) * n : m.xiw + k * n;
      LK(1, launch_draw_vector(cfg->n, seed, 3u, counter + (uint64_t)(g0 + k), v, s));
      LK(1, launch_apply_M<double>(cfg->sl1, cfg->cB, cfg->U64, v, m.eta + k * n, 1, s));  // R = M^dagger xi
    }
    CK(cudaMemsetAsync(X, 0, (size_t)ns * n * sizeof(double2), s));
    const int rc = solve_multi(cfg, ns, m.eta, X, tol, maxit, solver, infos ? infos + g0 : nullptr, s);
    if (rc != HQMC_OK && rc != HQMC_ENOTCONV && rc != HQMC_EBREAKDOWN && rc != HQMC_ENONFINITE) return rc;
    status = merge_status(status, rc);
    for (int k = 0; k < ns; ++k) {
      const double2* v = xi ? (double2*)xi + (size_t)(g0 + k) * n : m.xiw + k * n;
      LK(2, launch_cdot(cfg->n, v, X + k * n, cfg->act_grid, cfg->part_act, cfg->terms + 4, s));
      CK(cudaMemcpyAsync(cfg->terms_h + 4, cfg->terms + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      sum_re += cfg->terms_h[4];
      sum_im += cfg->terms_h[5];
    }
  }
  if (g_host) {
    const double norm = 1.0 / ((double)nrv * (double)cfg->n);
    g_host[0] = sum_re * norm;
    g_host[1] = sum_im * norm;
  }
  return status;
}

int check_estimate(hqmc_config* cfg, const double* theta, int nrv, double tol, int maxit, int solver, void* Gxi,
                   void* xi) {
  if (!aligned16(theta) || (Gxi && !aligned16(Gxi)) || (xi && !aligned16(xi)))
    return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  if (nrv < 1) return fail(cfg, HQMC_EINVAL, "nrv must be >= 1");
  if (!(tol > 0) || maxit < 0) return fail(cfg, HQMC_EINVAL, "tol must be > 0 and maxit >= 0");
  const size_t vb = (size_t)cfg->n * sizeof(double2);
  if (Gxi && xi && overlap(Gxi, vb * nrv, xi, vb * nrv)) return fail(cfg, HQMC_EINVAL, "Gxi and xi overlap");
  RET(check_solver(cfg, solver));
  return check_device(cfg);
}

}  // namespace

extern "C" {

int hqmc_estimate(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter, int nrv, double tol,
                  int maxit, int solver, void* Gxi, void* xi, double* g_host, hqmc_solve_info* infos, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  RET(check_estimate(cfg, theta, nrv, tol, maxit, solver, Gxi, xi));
  return estimate_impl(cfg, theta, seed, counter, nrv, tol, maxit, solver, Gxi, xi, g_host, infos, false,
                       (cudaStream_t)stream);
}

int hqmc_estimate_projected(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter, int nrv,
                            double tol, int maxit, int solver, void* Gxi, void* xi, double* g_host,
                            hqmc_solve_info* infos, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!Gxi) return fail(cfg, HQMC_EINVAL, "the projected estimate needs the solution array Gxi");
  RET(check_estimate(cfg, theta, nrv, tol, maxit, solver, Gxi, xi));
  return estimate_impl(cfg, theta, seed, counter, nrv, tol, maxit, solver, Gxi, xi, g_host, infos, true,
                       (cudaStream_t)stream);
}

int hqmc_set_multi_rhs(hqmc_config* cfg, int nmax) {
  if (!cfg) return HQMC_EINVAL;
  if (nmax < 0 || nmax > kMaxMultiRhs) return fail(cfg, HQMC_EINVAL, "nmax must be in [0, %d]", kMaxMultiRhs);
  RET(check_device(cfg));
  if (nmax > 0 && nmax <= cfg->mw.cap) return HQMC_OK;
  if (nmax > 0 && !multi_walk_shape(cfg).walk)
    return fail(cfg, HQMC_EUNSUPPORTED, "no tau-walking shape for L=%d (or variant %d)", cfg->p.L, cfg->p.variant);
  CK(cudaDeviceSynchronize());  // no graph over the old workspace may still run
  multi_release(cfg->mw);
  if (nmax == 0) return HQMC_OK;
  const int rc = multi_setup(cfg, nmax);
  if (rc != HQMC_OK) multi_release(cfg->mw);
  return rc;
}

int hqmc_set_multi_ranges(hqmc_config* cfg, int ranges) {
  if (!cfg) return HQMC_EINVAL;
  if (ranges < 0 || ranges > cfg->p.Ntau) return fail(cfg, HQMC_EINVAL, "ranges must be in [0, Ntau]");
  cfg->multi_ranges = ranges;
  return HQMC_OK;
}

int hqmc_multi_launch_shape(const hqmc_config* cfg, int nrhs, int* ranges, int* threads, int* nby) {
  if (!cfg || nrhs < 1) return HQMC_EINVAL;
  const SliceLaunch w = multi_walk_shape(cfg);
  if (!w.walk) return HQMC_EUNSUPPORTED;
  if (ranges) *ranges = multi_granges(cfg, nrhs);
  if (threads) *threads = w.threads;
  if (nby) *nby = w.nby;
  return HQMC_OK;
}

int hqmc_cg_solve_multi(hqmc_config* cfg, const double* theta, int nrhs, const void* phi, void* x, double tol,
                        int maxit, int solver, hqmc_solve_info* infos, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(phi) || !aligned16(x)) return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  RET(check_multi(cfg, nrhs, solver, tol, maxit));
  if (nrhs > cfg->mw.cap)
    return fail(cfg, HQMC_EINVAL, "%d systems exceed the %d of hqmc_set_multi_rhs", nrhs, cfg->mw.cap);
  const size_t vb = (size_t)cfg->n * sizeof(double2) * (size_t)nrhs;
  if (overlap(phi, vb, x, vb)) return fail(cfg, HQMC_EINVAL, "phi and x overlap");
  RET(check_device(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  RET(links(cfg, theta, true, true, s, false, true));
  return solve_multi(cfg, nrhs, (const double2*)phi, (double2*)x, tol, maxit, solver, infos, s);
}

int hqmc_estimate_multi(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter, int nrv, double tol,
                        int maxit, int solver, void* Gxi, void* xi, double* g_host, hqmc_solve_info* infos,
                        void* stream) {
  if (!cfg) return HQMC_EINVAL;
  RET(check_estimate(cfg, theta, nrv, tol, maxit, solver, Gxi, xi));
  RET(check_multi(cfg, nrv, solver, tol, maxit));
  return estimate_multi(cfg, theta, seed, counter, nrv, tol, maxit, solver, Gxi, xi, g_host, infos,
                        (cudaStream_t)stream);
}

int hqmc_force(hqmc_config* cfg, const double* theta, const void* X, double* F, double* dSf, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(X) || !aligned16(F) || (dSf && !aligned16(dSf)))
    return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  const size_t fb = cfg->n * 16;
  if (overlap(F, fb, theta, fb) || (dSf && (overlap(dSf, fb, theta, fb) || overlap(dSf, fb, F, fb))))
    return fail(cfg, HQMC_EINVAL, "output overlaps an input");
  RET(check_device(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  RET(links(cfg, theta, true, false, s));
  return force(cfg, theta, (const double2*)X, F, dSf ? dSf : cfg->dSf, s);
}

int hqmc_action_terms(hqmc_config* cfg, const double* theta, const double* p, const void* phi, const void* X,
                      double* out_host, void* stream) {
  if (!cfg || !out_host) return HQMC_EINVAL;
  if (!aligned16(theta) || (p && !aligned16(p)) || (phi && !aligned16(phi)) || (X && !aligned16(X)))
    return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  RET(check_device(cfg));
  cudaStream_t s = (cudaStream_t)stream;
  const bool ab = phi && X;
  LK(2, launch_action_terms(cfg->g, cfg->bp, theta, p, ab ? (const double2*)phi : nullptr,
                         ab ? (const double2*)X : nullptr, cfg->act_grid, cfg->part_act, cfg->terms, s));
  CK(cudaMemcpyAsync(cfg->terms_h, cfg->terms, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < 3; ++i) out_host[i] = cfg->terms_h[i];
  return HQMC_OK;
}

int hqmc_draw(hqmc_config* cfg, uint64_t seed, uint64_t traj_counter, double* p, void* R, double* u_host,
              void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if ((p && !aligned16(p)) || (R && !aligned16(R))) return fail(cfg, HQMC_EINVAL, "misaligned pointer");
  RET(check_device(cfg));
  if (p || R) LK(1, launch_draw(cfg->n, seed, traj_counter, p, (double2*)R, (cudaStream_t)stream));
  if (u_host) philox_uniform_host(seed, traj_counter, u_host);
  return HQMC_OK;
}

int hqmc_leapfrog(hqmc_config* cfg, double* theta, double* p, const void* phi, void* X, int nsteps, double dt,
                  double tol, int maxit, int solver, hqmc_traj_info* info, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(p) || !aligned16(phi) || !aligned16(X))
    return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  if (nsteps < 0 || !std::isfinite(dt) || !(tol > 0) || maxit < 0) return fail(cfg, HQMC_EINVAL, "bad step parameters");
  RET(check_solver(cfg, solver));
  RET(check_device(cfg));
  hqmc_traj_info ti{};
  const int rc = leapfrog(cfg, theta, p, (const double2*)phi, (double2*)X, nsteps, dt, tol, maxit, solver, &ti,
                          (cudaStream_t)stream);
  if (rc == HQMC_OK || rc == HQMC_ENOTCONV) CK(cudaStreamSynchronize((cudaStream_t)stream));
  ti.status = rc;
  if (info) *info = ti;
  return rc;
}

int hqmc_trajectory(hqmc_config* cfg, double* theta, uint64_t seed, uint64_t traj_counter, const double* p_in,
                    const void* R_in, const double* u_in, int nsteps, double dt, double tol, int maxit, int solver,
                    hqmc_traj_info* info, void* stream) {
  if (!cfg) return HQMC_EINVAL;
  if (!aligned16(theta) || (p_in && !aligned16(p_in)) || (R_in && !aligned16(R_in)))
    return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  if (nsteps < 0 || !std::isfinite(dt) || !(tol > 0) || maxit < 0) return fail(cfg, HQMC_EINVAL, "bad step parameters");
  RET(check_solver(cfg, solver));
  RET(check_device(cfg));
  NvtxRange nv("hqmc trajectory");
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = cfg->n;
  hqmc_traj_info ti{};
  // (i) momenta and pseudofermion source
  if (p_in)
    CK(cudaMemcpyAsync(cfg->pm, p_in, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    LK(1, launch_draw(n, seed, traj_counter, cfg->pm, nullptr, s));
  if (R_in)
    CK(cudaMemcpyAsync(cfg->Rw, R_in, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  else
    LK(1, launch_draw(n, seed, traj_counter, nullptr, cfg->Rw, s));
  if (u_in)
    ti.u = *u_in;
  else
    philox_uniform_host(seed, traj_counter, &ti.u);
  RET(links(cfg, theta, true, false, s));
  LK(1, launch_apply_M<double>(cfg->sl1, cfg->cB, cfg->U64, cfg->Rw, cfg->eta, 1, s));  // eta = M^dagger R
  // H0 = S_B + sum p^2 + R^dagger R
  LK(2, launch_action_terms(cfg->g, cfg->bp, theta, cfg->pm, cfg->Rw, cfg->Rw, cfg->act_grid, cfg->part_act,
                         cfg->terms, s));
  CK(cudaMemcpyAsync(cfg->th0, theta, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(cfg->Xw, 0, n * sizeof(double2), s));
  // (ii) leapfrog
  int rc = leapfrog(cfg, theta, cfg->pm, cfg->eta, cfg->Xw, nsteps, dt, tol, maxit, solver, &ti, s);
  if (rc != HQMC_OK && rc != HQMC_ENOTCONV) {
    CK(cudaMemcpyAsync(theta, cfg->th0, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    ti.status = rc;
    if (info) *info = ti;
    return rc;
  }
  // H1 = S_B + sum p^2 + eta^dagger X
  LK(2, launch_action_terms(cfg->g, cfg->bp, theta, cfg->pm, cfg->eta, cfg->Xw, cfg->act_grid, cfg->part_act,
                         cfg->terms + 3, s));
  CK(cudaMemcpyAsync(cfg->terms_h, cfg->terms, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double* t = cfg->terms_h;
  ti.H0 = t[0] + t[1] + t[2];
  ti.H1 = t[3] + t[4] + t[5];
  ti.dH = ti.H1 - ti.H0;
  if (!std::isfinite(ti.dH)) rc = HQMC_ENONFINITE;
  // (iii) Metropolis: accept iff u < exp(H0 - H1)
  ti.accepted = (rc == HQMC_OK || rc == HQMC_ENOTCONV) && std::isfinite(ti.dH) && ti.u < std::exp(-ti.dH);
  if (!ti.accepted) {
    CK(cudaMemcpyAsync(theta, cfg->th0, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  ti.status = rc;
  if (info) *info = ti;
  return rc;
}

int hqmc_probe_fp64_rate(hqmc_config* cfg, double* tflops_out) {
  if (!cfg || !tflops_out) return HQMC_EINVAL;
  RET(check_device(cfg));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device));
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    CK(cudaEventRecord(a, 0));
    LK(1, launch_fp64_probe(blocks, threads, iters, cfg->report, 0));
    CK(cudaEventRecord(b, 0));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (rep > 0 && ms < best) best = ms;  // the first launch is a warm-up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const double flops = 16.0 * iters * (double)blocks * threads;
  *tflops_out = flops / (best * 1e-3) / 1e12;
  return HQMC_OK;
}

int hqmc_set_timing(hqmc_config* cfg, int enable) {
  if (!cfg) return HQMC_EINVAL;
  CK(cudaDeviceSynchronize());
  cfg->timing = enable ? 1 : 0;
  for (auto& tc : cfg->timers) tc.used = 0;
  return HQMC_OK;
}

int hqmc_get_timing(hqmc_config* cfg, int timer, long long* launches, double* total_ms) {
  if (!cfg || timer < 0 || timer >= HQMC_TIMER_COUNT) return HQMC_EINVAL;
  CK(cudaDeviceSynchronize());
  const TimerClass& tc = cfg->timers[timer];
  double sum = 0.0;
  for (size_t i = 0; i < tc.used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, tc.pairs[i].first, tc.pairs[i].second));
    sum += ms;
  }
  if (launches) *launches = (long long)tc.used;
  if (total_ms) *total_ms = sum;
  return HQMC_OK;
}

int hqmc_get_timing_samples(hqmc_config* cfg, int timer, float* us, int max_n, int* n_out) {
  if (!cfg || timer < 0 || timer >= HQMC_TIMER_COUNT || max_n < 0 || (max_n > 0 && !us)) return HQMC_EINVAL;
  CK(cudaDeviceSynchronize());
  const TimerClass& tc = cfg->timers[timer];
  const int n = (int)std::min(tc.used, (size_t)max_n);
  for (int i = 0; i < n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, tc.pairs[i].first, tc.pairs[i].second));
    us[i] = 1e3f * ms;
  }
  if (n_out) *n_out = (int)tc.used;
  return HQMC_OK;
}

}  // extern "C"

// ===========================================================================
// Batches of independent chains (lattices of different L in one launch per CG
// iteration).  Each chain keeps its own config (workspace, link tables, CG
// state); the CG loop runs the generic fused kernel over a tile table that
// covers every chain's slices, and a batched update over every chain's vector
// blocks, under one WHILE node that continues while any chain is running.

struct hqmc_batch {
  std::vector<hqmc_config*> cfgs;
  int C = 1;           // cluster size (slices per tile), shared by all chains
  int tile_order = 0;  // order of the tile table (batch_tiles)
  float tuned_us = 0.f;  // autotuner: time of one batched fused launch (0: not tuned)
  int threads = 64;    // block size of the batched fused kernel
  size_t smem = 0;     // its dynamic shared memory (largest chain)
  int ntiles = 0;
  int tiles_cap = 0;   // capacity of d_tiles (one tile per slice)
  int total_ublocks = 0;
  MdagmArgs<double>* d_cgdir = nullptr;
  MdagmArgs<double>* d_resid_start = nullptr;
  MdagmArgs<double>* d_resid_loop = nullptr;
  UpdArgs<double>* d_upd = nullptr;
  FinArgs* d_fin = nullptr;
  int2* d_tiles = nullptr;
  int2* d_ublocks = nullptr;
  int* d_unblocks = nullptr;
  CgState** d_states = nullptr;
  int solver = HQMC_SOLVER_CG64;  // CG64 or PCG64 (tau-line preconditioner)
  LineBatchDesc<double>* d_line = nullptr;  // per-chain preconditioner descriptors
  int4* d_ltiles = nullptr;                 // (chain, bx, by) tiles of the batched preconditioner
  int nltiles = 0;
  int maxW = 0;
  int maxtc = 0;  // tallest preconditioner tile of the chains (shared memory of the batched launch)
  void* h_stage = nullptr;  // pinned staging of the descriptor arrays
  size_t stage_bytes = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int body_kernels = 0;
  long long launches = 0;
  // one graph per trajectory: per-chain descriptors, block tables, device info
  MdagmArgs<double>* d_resid_report = nullptr;  // residual of unconverged chains after a loop (FIN_REPORT)
  ChainDesc* d_chain = nullptr;
  ChainDesc* h_chain = nullptr;        // pinned staging
  uint64_t* d_counter = nullptr;       // trajectory counter (device; read by the draws and the Metropolis uniform)
  unsigned long long* d_bodies = nullptr;  // loop bodies run by the last trajectory graph
  hqmc_traj_info* d_info = nullptr;
  struct TrajMirror {
    uint64_t counter;
    unsigned long long bodies;
  }* h_mirror = nullptr;               // pinned: counter to upload, bodies read back
  hqmc_traj_info* h_info = nullptr;    // pinned mirror of d_info
  int4 *d_site_tab = nullptr, *d_act_tab = nullptr, *d_ff_tab = nullptr;
  int n_site_tab = 0, n_act_tab = 0, n_ff_tab = 0;
  int2* d_stiles = nullptr;            // (chain, slice) of the slice kernels (M^dagger R, force)
  int n_stiles = 0;
  int slice_threads = 64;
  size_t smem_apply = 0, smem_force = 0;
  cudaStream_t cap2 = nullptr;         // captures the loop bodies while a trajectory is being captured
  cudaGraphExec_t traj_exec = nullptr;
  int traj_nsteps = -1, traj_maxit = -1, traj_solver = -1;
  double traj_tol = -1.0;
  long long traj_static_kernels = 0;   // kernels of a trajectory graph outside its loop bodies
  char err[512] = {0};
};

namespace {

int bfail(hqmc_batch* b, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->err, sizeof(b->err), fmt, ap);
  va_end(ap);
  return code;
}

#define BCK(call)                                                                                       \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess)                                                                              \
      return bfail(b, HQMC_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define BRET(call, c)                                          \
  do {                                                         \
    int rc_ = (call);                                          \
    if (rc_ != HQMC_OK) {                                      \
      snprintf(b->err, sizeof(b->err), "%s", (c)->err);        \
      return rc_;                                              \
    }                                                          \
  } while (0)

void batch_release(hqmc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->traj_exec) cudaGraphExecDestroy(b->traj_exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  cudaFree(b->d_resid_report);
  cudaFree(b->d_chain);
  cudaFree(b->d_counter);
  cudaFree(b->d_bodies);
  cudaFree(b->d_info);
  cudaFree(b->d_site_tab);
  cudaFree(b->d_act_tab);
  cudaFree(b->d_ff_tab);
  cudaFree(b->d_stiles);
  if (b->h_chain) cudaFreeHost(b->h_chain);
  if (b->h_mirror) cudaFreeHost(b->h_mirror);
  if (b->h_info) cudaFreeHost(b->h_info);
  cudaFree(b->d_cgdir);
  cudaFree(b->d_resid_start);
  cudaFree(b->d_resid_loop);
  cudaFree(b->d_upd);
  cudaFree(b->d_fin);
  cudaFree(b->d_tiles);
  cudaFree(b->d_ublocks);
  cudaFree(b->d_unblocks);
  cudaFree(b->d_states);
  cudaFree(b->d_line);
  cudaFree(b->d_ltiles);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  for (hqmc_config* c : b->cfgs) hqmc_free_config(c);
  b->cfgs.clear();
}

// Cluster tiles (chain, first slice) of the batched fused kernel for cluster
// size C, in one of three orders: 0 chain by chain as given, 1 the chains with
// the most sites per slice first, 2 round robin over the chains.  The order
// changes only which CTAs the hardware dispatches first, never a result.
std::vector<int2> batch_tiles(const std::vector<hqmc_config*>& cfgs, int C, int order) {
  const int nc = (int)cfgs.size();
  std::vector<int> ch(nc);
  for (int c = 0; c < nc; ++c) ch[c] = c;
  if (order == 1)
    std::stable_sort(ch.begin(), ch.end(), [&](int a, int b) { return cfgs[a]->g.V > cfgs[b]->g.V; });
  std::vector<int2> tiles;
  if (order == 2) {
    for (int t0 = 0;; t0 += C) {
      bool any = false;
      for (int c : ch)
        if (t0 < cfgs[c]->p.Ntau) {
          tiles.push_back(make_int2(c, t0));
          any = true;
        }
      if (!any) break;
    }
  } else {
    for (int c : ch)
      for (int t0 = 0; t0 < cfgs[c]->p.Ntau; t0 += C) tiles.push_back(make_int2(c, t0));
  }
  return tiles;
}

// Cluster size and tile order of the batched fused kernel; every chain's
// partial-sum slots follow the cluster size.
int batch_set_tiles(hqmc_batch* b, int C, int order) {
  b->C = C;
  b->tile_order = order;
  for (hqmc_config* cfg : b->cfgs) {
    cfg->sl.cluster = C;
    cfg->sl.grid = (cfg->p.Ntau + C - 1) / C * C;
    cfg->fused64.cluster = C;
    cfg->fused64.grid = cfg->sl.grid;
  }
  const std::vector<int2> tiles = batch_tiles(b->cfgs, C, order);
  if ((int)tiles.size() > b->tiles_cap) return bfail(b, HQMC_EINVAL, "tile table overflow");
  b->ntiles = (int)tiles.size();
  BCK(cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice));
  return HQMC_OK;
}

// Autotuner of the batch: times the batched fused launch (an FP64 residual
// r = phi - O x of every chain, zero operands, links of theta = 0) at every
// cluster size 1, 2, 4, 8 the device can co-schedule and every tile order, and
// keeps the fastest.  Results do not depend on the choice: the neighbour's z_{tau-1}
// is the same arithmetic as the recomputed halo, and the reduction slots are
// per slice.
int batch_autotune(hqmc_batch* b) {
  const int nc = (int)b->cfgs.size();
  int minN = 1 << 30;
  std::vector<MdagmArgs<double>> descs(nc);
  for (int c = 0; c < nc; ++c) {
    hqmc_config* cfg = b->cfgs[c];
    minN = std::min(minN, cfg->p.Ntau);
    BCK(cudaMemset(cfg->th0, 0, 2 * cfg->n * sizeof(double)));
    BCK(cudaMemset(cfg->p64[0], 0, cfg->n * sizeof(double2)));
    BCK(cudaMemset(cfg->p64[1], 0, cfg->n * sizeof(double2)));
    BCK(launch_links(cfg->g, cfg->th0, cfg->t1, cfg->t2, cfg->U64, cfg->U32, cfg->th32, 0));
    MdagmArgs<double> r = mdagm_args<double, MODE_RESID>(cfg);
    r.U = cfg->U64;
    r.x = cfg->p64[0];
    r.b = cfg->p64[1];
    r.r_out = cfg->r64;
    r.r_out_fp32 = 0;
    r.part_out = cfg->part_resid;
    r.st = cfg->st;
    r.teff = cfg->sl.threads;
    r.gate = GATE_ALWAYS;
    descs[c] = r;
  }
  BCK(cudaMemcpy(b->d_resid_start, descs.data(), nc * sizeof(MdagmArgs<double>), cudaMemcpyHostToDevice));
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  const int reps = 5;
  float best = 1e30f;
  int bestC = b->C, bestOrder = b->tile_order;
  int rc = HQMC_OK;
  for (int C : {1, 2, 4, 8}) {
    if (C > minN || (C > 1 && mdagm_batch_max_active_clusters(C, b->threads, b->smem) <= 0)) continue;
    for (int order = 0; order < 3 && rc == HQMC_OK; ++order) {
      if ((rc = batch_set_tiles(b, C, order)) != HQMC_OK) break;
      auto go = [&]() {
        return launch_mdagm_batch<double, MODE_RESID>(b->d_resid_start, b->d_tiles, b->ntiles, b->C, b->threads,
                                                      b->smem, 0);
      };
      cudaError_t err = go();
      if (err == cudaSuccess) err = cudaEventRecord(e0, 0);
      for (int k = 0; k < reps && err == cudaSuccess; ++k) err = go();
      if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err != cudaSuccess) {  // a shape the device refuses is skipped
        cudaGetLastError();
        continue;
      }
      b->launches += reps + 1;
      const float us = 1e3f * ms / reps;
      if (us < best) {
        best = us;
        bestC = C;
        bestOrder = order;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HQMC_OK) return rc;
  if (best >= 1e30f) return bfail(b, HQMC_EUNSUPPORTED, "no batched launch shape ran");
  b->tuned_us = best;
  return batch_set_tiles(b, bestC, bestOrder);
}

// Per-chain descriptors of the batched CG kernels for operands (phi, x).
int batch_descriptors(hqmc_batch* b, const double2* const* phi, double2* const* x, cudaStream_t s) {
  const int nc = (int)b->cfgs.size();
  char* st = (char*)b->h_stage;
  auto* cgdir = (MdagmArgs<double>*)st;
  auto* rs = cgdir + nc;
  auto* rl = rs + nc;
  auto* up = (UpdArgs<double>*)(rl + nc);
  auto* fin = (FinArgs*)(up + nc);
  auto* ld = (LineBatchDesc<double>*)(fin + nc);
  auto* rep = (MdagmArgs<double>*)(ld + nc);
  const bool pc = b->solver == HQMC_SOLVER_PCG64;
  for (int c = 0; c < nc; ++c) {
    hqmc_config* cfg = b->cfgs[c];
    const int nslots = (cfg->p.Ntau + b->C - 1) / b->C * b->C;
    MdagmArgs<double> a = mdagm_args<double, MODE_CGDIR>(cfg);
    a.U = cfg->U64;
    a.y = cfg->q64;
    a.r = pc ? cfg->z64 : cfg->r64;
    if (pc) {
      a.part_rz = cfg->part_rz;
      a.n_part_rz = cfg->ll64.gx * cfg->ll64.gy;
    }
    ld[c] = LineBatchDesc<double>{cfg->g,        cfg->lc,  cfg->r64,         cfg->z64,
                                  cfg->part_rz, cfg->st, cfg->ll64.gx, cfg->ll64.chunk};
    a.pbuf[0] = cfg->p64[0];
    a.pbuf[1] = cfg->p64[1];
    a.part_in = cfg->part_ew;
    a.n_part_in = cfg->ew_grid;
    a.part_out = cfg->part_mdagm;
    a.st = cfg->st;
    a.teff = cfg->fused64.threads;  // this chain's own block size: identical reduction order
    cgdir[c] = a;
    MdagmArgs<double> r = mdagm_args<double, MODE_RESID>(cfg);
    r.U = cfg->U64;
    r.x = x[c];
    r.b = phi[c];
    r.r_out = cfg->r64;
    r.r_out_fp32 = 0;
    r.part_out = cfg->part_resid;
    r.st = cfg->st;
    r.teff = cfg->sl.threads;
    r.gate = GATE_ALWAYS;
    rs[c] = r;
    r.gate = GATE_REC;
    rl[c] = r;
    r.gate = GATE_UNCONVERGED;  // after a loop: the true residual of chains that did not converge
    r.r_out = cfg->vscratch;
    rep[c] = r;
    up[c] = UpdArgs<double>{cfg->n, x[c], 1, cfg->r64, cfg->p64[0], cfg->p64[1], cfg->q64, cfg->part_mdagm,
                            nslots, cfg->part_ew, cfg->st};
    fin[c] = FinArgs{cfg->part_resid, nslots, cfg->part_ew, cfg->ew_grid, cfg->st, cfg->report};
  }
  BCK(cudaMemcpyAsync(b->d_cgdir, cgdir, nc * sizeof(MdagmArgs<double>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_resid_start, rs, nc * sizeof(MdagmArgs<double>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_resid_loop, rl, nc * sizeof(MdagmArgs<double>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_upd, up, nc * sizeof(UpdArgs<double>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_fin, fin, nc * sizeof(FinArgs), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_line, ld, nc * sizeof(LineBatchDesc<double>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_resid_report, rep, nc * sizeof(MdagmArgs<double>), cudaMemcpyHostToDevice, s));
  return HQMC_OK;
}

int batch_body(hqmc_batch* b, cudaStream_t s) {
  const int nc = (int)b->cfgs.size();
  const bool pc = b->solver == HQMC_SOLVER_PCG64;
  for (int it = 0; it < kBodyIters64; ++it) {
    BCK((launch_mdagm_batch<double, MODE_CGDIR>(b->d_cgdir, b->d_tiles, b->ntiles, b->C, b->threads, b->smem, s)));
    BCK(launch_cg_update_batch(b->d_upd, b->d_ublocks, b->d_unblocks, b->total_ublocks, s));
    if (pc) BCK(launch_line_precond_batch(b->d_line, b->d_ltiles, b->nltiles, b->maxW, b->maxtc, s));
  }
  BCK((launch_mdagm_batch<double, MODE_RESID>(b->d_resid_loop, b->d_tiles, b->ntiles, b->C, b->threads, b->smem, s)));
  BCK(launch_resid_finalize_batch(b->d_fin, nc, FIN_RESTART, 0.0, 0, GATE_REC, s));
  if (pc) BCK(launch_line_precond_batch(b->d_line, b->d_ltiles, b->nltiles, b->maxW, b->maxtc, s));
  return HQMC_OK;
}

int batch_graph(hqmc_batch* b) {
  if (b->exec) return HQMC_OK;
  cudaGraph_t graph = nullptr;
  BCK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return bfail(b, HQMC_ECUDA, "conditional graph node: %s", cudaGetErrorString(e));
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  BCK(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = batch_body(b, b->cap);
  if (rc == HQMC_OK) {
    cudaError_t le = launch_loop_condition_batch(b->d_states, (int)b->cfgs.size(), handle, b->cap);
    if (le != cudaSuccess) rc = bfail(b, HQMC_ECUDA, "loop condition: %s", cudaGetErrorString(le));
  }
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(b->cap, &captured);
  if (rc == HQMC_OK && e != cudaSuccess) rc = bfail(b, HQMC_ECUDA, "end capture: %s", cudaGetErrorString(e));
  if (rc == HQMC_OK) {
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (e != cudaSuccess) rc = bfail(b, HQMC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  cudaGraphDestroy(graph);
  if (rc != HQMC_OK) cudaGetLastError();
  const bool pc = b->solver == HQMC_SOLVER_PCG64;
  b->body_kernels = (pc ? 3 : 2) * kBodyIters64 + 3 + (pc ? 1 : 0);
  return rc;
}

// CG on every chain (links already built); infos[c] filled; returns the worst status.
int batch_solve(hqmc_batch* b, const double2* const* phi, double2* const* x, double tol, int maxit,
                hqmc_solve_info* infos, cudaStream_t s) {
  const int nc = (int)b->cfgs.size();
  int rc = batch_descriptors(b, phi, x, s);
  if (rc != HQMC_OK) return rc;
  BCK((launch_mdagm_batch<double, MODE_RESID>(b->d_resid_start, b->d_tiles, b->ntiles, b->C, b->threads, b->smem, s)));
  BCK(launch_resid_finalize_batch(b->d_fin, nc, FIN_START, tol, maxit, GATE_ALWAYS, s));
  b->launches += 2;
  if (b->solver == HQMC_SOLVER_PCG64) {
    BCK(launch_line_precond_batch(b->d_line, b->d_ltiles, b->nltiles, b->maxW, b->maxtc, s));
    b->launches += 1;
  }
  if ((rc = batch_graph(b)) != HQMC_OK) return rc;
  BCK(cudaGraphLaunch(b->exec, s));
  int worst = HQMC_OK;
  int max_loops = 0;
  for (int c = 0; c < nc; ++c) {
    hqmc_config* cfg = b->cfgs[c];
    BRET(read_state(cfg, s), cfg);
    max_loops = std::max(max_loops, cfg->st_h->loops);
  }
  b->launches += (long long)max_loops * (b->body_kernels + 1);
  for (int c = 0; c < nc; ++c) {
    hqmc_config* cfg = b->cfgs[c];
    const CgState st = *cfg->st_h;
    int status = HQMC_OK;
    if (st.bb == 0.0) {
      BCK(cudaMemsetAsync(x[c], 0, sizeof(double2) * cfg->n, s));
      cfg->report_h[0] = 0.0;
    } else if (st.done != CG_CONVERGED) {
      status = solve_status(st.done, false);  // the batched kernels have no device-side waits
      BRET(residual(cfg, phi[c], x[c], cfg->vscratch, false, FIN_REPORT, tol, maxit, GATE_ALWAYS, s), cfg);
      BRET(read_state(cfg, s), cfg);
    }
    hqmc_solve_info inf{};
    inf.status = status;
    inf.iterations = st.k;
    inf.true_residual = st.bb > 0 ? std::sqrt(cfg->report_h[0] / st.bb) : 0.0;
    const double rr_rec = (b->solver == HQMC_SOLVER_PCG64 && st.k > st.seg_start) ? st.rr_rec : st.rr[st.k & 1];
    inf.recursive_residual = st.bb > 0 ? std::sqrt(rr_rec / st.bb) : 0.0;
    if (status == HQMC_OK && !(inf.true_residual <= tol)) status = inf.status = HQMC_ENOTCONV;
    if (infos) infos[c] = inf;
    worst = merge_status(worst, status);
  }
  return worst;
}

// One batched solve of (M^dagger M) X_c = eta_c for every chain, enqueued while a
// trajectory graph is being captured on s: the start residual, a conditional WHILE
// node (added to the capture's graph) whose body is the batched CG loop body,
// captured on a second stream, then the true residual of the chains that did not
// converge and the per-chain bookkeeping of the trajectory info.
int traj_solve(hqmc_batch* b, double tol, int maxit, long long* nk, cudaStream_t s) {
  const int nc = (int)b->cfgs.size();
  const bool pc = b->solver == HQMC_SOLVER_PCG64;
  BCK((launch_mdagm_batch<double, MODE_RESID>(b->d_resid_start, b->d_tiles, b->ntiles, b->C, b->threads, b->smem, s)));
  BCK(launch_resid_finalize_batch(b->d_fin, nc, FIN_START, tol, maxit, GATE_ALWAYS, s));
  *nk += 2;
  if (pc) {
    BCK(launch_line_precond_batch(b->d_line, b->d_ltiles, b->nltiles, b->maxW, b->maxtc, s));
    *nk += 1;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  BCK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return bfail(b, HQMC_ECUDA, "trajectory capture is not active");
  cudaGraphConditionalHandle h;
  BCK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  BCK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  BCK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  BCK(cudaStreamBeginCaptureToGraph(b->cap2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed));
  int rc = batch_body(b, b->cap2);
  if (rc == HQMC_OK) {
    const cudaError_t le = launch_loop_condition_batch(b->d_states, nc, h, b->cap2, b->d_bodies);
    if (le != cudaSuccess) rc = bfail(b, HQMC_ECUDA, "loop condition: %s", cudaGetErrorString(le));
  }
  cudaGraph_t body = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap2, &body);
  if (rc != HQMC_OK) return rc;
  BCK(e);
  BCK((launch_mdagm_batch<double, MODE_RESID>(b->d_resid_report, b->d_tiles, b->ntiles, b->C, b->threads, b->smem, s)));
  BCK(launch_resid_finalize_batch(b->d_fin, nc, FIN_REPORT, tol, maxit, GATE_UNCONVERGED, s));
  BCK(launch_batch_solve_close(b->d_chain, nc, s));
  *nk += 3;
  return HQMC_OK;
}

// The whole trajectory of every chain as one graph (rebuilt when nsteps, tol, maxit
// or the solver change): draws, links, phi = M^dagger R, H0, the leapfrog with its
// N_lf + 1 batched solves and forces, H1, the Metropolis test and the restore of
// rejected fields.  Every kernel reads the per-chain descriptors and the trajectory
// counter from device memory, which the host rewrites before each launch.
int traj_graph(hqmc_batch* b, int nsteps, double tol, int maxit) {
  if (b->traj_exec && b->traj_nsteps == nsteps && b->traj_tol == tol && b->traj_maxit == maxit &&
      b->traj_solver == b->solver)
    return HQMC_OK;
  if (b->traj_exec) {
    BCK(cudaDeviceSynchronize());
    cudaGraphExecDestroy(b->traj_exec);
    b->traj_exec = nullptr;
  }
  const int nc = (int)b->cfgs.size();
  cudaStream_t s = b->cap;
  long long nk = 0;
  BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  auto ew = [&](int op) -> int {
    BCK(launch_batch_elementwise(b->d_chain, b->d_site_tab, b->n_site_tab, op, b->d_counter, s));
    nk += 1;
    return HQMC_OK;
  };
  auto force = [&]() -> int {
    BCK(launch_batch_force(b->d_chain, b->d_stiles, b->n_stiles, b->slice_threads, b->smem_force, s));
    BCK(launch_batch_force_finish(b->d_chain, b->d_ff_tab, b->n_ff_tab, s));
    nk += 2;
    return HQMC_OK;
  };
  auto body = [&]() -> int {
    BCK(launch_batch_info_init(b->d_chain, nc, b->d_counter, s));
    nk += 1;
    RET(ew(BT_DRAW));
    RET(ew(BT_LINKS));
    BCK(launch_batch_apply_Mdag(b->d_chain, b->d_stiles, b->n_stiles, b->slice_threads, b->smem_apply, s));
    BCK(launch_batch_action(b->d_chain, b->d_act_tab, b->n_act_tab, nc, 0, s));  // H0
    nk += 3;
    RET(ew(BT_SAVE));
    RET(ew(BT_ZERO_X));
    RET(traj_solve(b, tol, maxit, &nk, s));
    RET(force());
    for (int step = 0; step < nsteps; ++step) {
      RET(ew(BT_KICK_DRIFT));
      RET(ew(BT_LINKS));
      RET(traj_solve(b, tol, maxit, &nk, s));
      RET(force());
      RET(ew(BT_KICK));
    }
    BCK(launch_batch_action(b->d_chain, b->d_act_tab, b->n_act_tab, nc, 1, s));  // H1
    BCK(launch_batch_metropolis(b->d_chain, nc, s));
    nk += 3;
    return ew(BT_RESTORE);
  };
  int rc = body();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (rc == HQMC_OK && e != cudaSuccess) rc = bfail(b, HQMC_ECUDA, "trajectory capture: %s", cudaGetErrorString(e));
  if (rc == HQMC_OK) {
    e = cudaGraphInstantiate(&b->traj_exec, graph, 0);
    if (e != cudaSuccess) {
      b->traj_exec = nullptr;
      rc = bfail(b, HQMC_ECUDA, "trajectory graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  if (graph) cudaGraphDestroy(graph);
  if (rc != HQMC_OK) {
    cudaGetLastError();
    return rc;
  }
  b->traj_nsteps = nsteps;
  b->traj_tol = tol;
  b->traj_maxit = maxit;
  b->traj_solver = b->solver;
  b->traj_static_kernels = nk;
  return HQMC_OK;
}

}  // namespace

extern "C" {

int hqmc_make_batch(const hqmc_params* params, int nchains, hqmc_batch** out) {
  if (!params || !out || nchains < 1) return HQMC_EINVAL;
  *out = nullptr;
  hqmc_batch* b = new (std::nothrow) hqmc_batch();
  if (!b) return HQMC_ENOMEM;
  int rc = HQMC_OK;
  do {
    int maxV = 0, minC = 8, maxThreads = 64;
    bool tune = false;
    for (int c = 0; c < nchains; ++c) {
      hqmc_params p = params[c];
      tune = tune || p.autotune;
      p.variant = 1;  // the batched kernel is the generic one; chains stay bit-identical to it
      p.autotune = 0;
      hqmc_config* cfg = nullptr;
      if ((rc = hqmc_make_config(&p, &cfg)) != HQMC_OK) {
        bfail(b, rc, "chain %d: %s", c, hqmc_strerror(rc));
        break;
      }
      b->cfgs.push_back(cfg);
      maxV = std::max(maxV, cfg->g.V);
      minC = std::min(minC, cfg->sl.cluster);
      maxThreads = std::max(maxThreads, std::max(cfg->sl.threads, cfg->fused64.threads));
    }
    if (rc != HQMC_OK) break;
    b->C = minC;
    b->threads = maxThreads;
    b->smem = (size_t)3 * maxV * sizeof(double2);
    std::vector<int2> ublocks;
    std::vector<int> unblocks;
    for (int c = 0; c < nchains; ++c) {
      hqmc_config* cfg = b->cfgs[c];
      b->tiles_cap += cfg->p.Ntau;  // cluster size 1: one tile per slice
      for (int j = 0; j < cfg->ew_grid; ++j) ublocks.push_back(make_int2(c, j));
      unblocks.push_back(cfg->ew_grid);
    }
    b->total_ublocks = (int)ublocks.size();
    // tiles of the batched preconditioner: every chain's own (bx, by) grid
    std::vector<int4> ltiles;
    for (int c = 0; c < nchains; ++c) {
      const LineLaunch& ll = b->cfgs[c]->ll64;
      b->maxW = std::max(b->maxW, b->cfgs[c]->lc.W);
      b->maxtc = std::max(b->maxtc, ll.chunk);
      for (int by = 0; by < ll.gy; ++by)
        for (int bx = 0; bx < ll.gx; ++bx) ltiles.push_back(make_int4(c, bx, by, 0));
    }
    b->nltiles = (int)ltiles.size();
    if (prepare_line_precond_batch(b->maxW, b->maxtc) != cudaSuccess) {
      cudaGetLastError();
      rc = bfail(b, HQMC_EUNSUPPORTED, "batched preconditioner does not fit");
      break;
    }
    std::vector<CgState*> states;
    for (hqmc_config* cfg : b->cfgs) states.push_back(cfg->st);
    auto dal = [&](void** p, size_t bytes) {
      if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return true;
    };
    if (!dal((void**)&b->d_cgdir, nchains * sizeof(MdagmArgs<double>)) ||
        !dal((void**)&b->d_resid_start, nchains * sizeof(MdagmArgs<double>)) ||
        !dal((void**)&b->d_resid_loop, nchains * sizeof(MdagmArgs<double>)) ||
        !dal((void**)&b->d_upd, nchains * sizeof(UpdArgs<double>)) ||
        !dal((void**)&b->d_fin, nchains * sizeof(FinArgs)) || !dal((void**)&b->d_tiles, b->tiles_cap * sizeof(int2)) ||
        !dal((void**)&b->d_ublocks, ublocks.size() * sizeof(int2)) ||
        !dal((void**)&b->d_unblocks, unblocks.size() * sizeof(int)) ||
        !dal((void**)&b->d_states, states.size() * sizeof(CgState*)) ||
        !dal((void**)&b->d_line, nchains * sizeof(LineBatchDesc<double>)) ||
        !dal((void**)&b->d_ltiles, ltiles.size() * sizeof(int4))) {
      rc = bfail(b, HQMC_ENOMEM, "batch tables");
      break;
    }
    b->stage_bytes = nchains * (4 * sizeof(MdagmArgs<double>) + sizeof(UpdArgs<double>) + sizeof(FinArgs) +
                                sizeof(LineBatchDesc<double>));
    if (cudaMallocHost(&b->h_stage, b->stage_bytes) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      rc = bfail(b, HQMC_ENOMEM, "batch staging");
      break;
    }
    // trajectory graphs: block tables of the batched kernels over every chain
    std::vector<int4> site_tab, act_tab, ff_tab;
    std::vector<int2> stiles;
    auto ew = [](long long count) { return (int)std::max(1LL, std::min(4096LL, (count + 255) / 256)); };
    int maxSliceThreads = 64;
    for (int c = 0; c < nchains; ++c) {
      hqmc_config* cfg = b->cfgs[c];
      const int nsb = ew(2 * cfg->n);  // the longest loop of the element-wise ops (2 per site)
      for (int j = 0; j < nsb; ++j) site_tab.push_back(make_int4(c, j, nsb, 0));
      for (int j = 0; j < cfg->act_grid; ++j) act_tab.push_back(make_int4(c, j, cfg->act_grid, 0));
      const long long nff = (long long)cfg->g.V * ((cfg->p.Ntau + 31) / 32);
      const int nfb = ew(nff);
      for (int j = 0; j < nfb; ++j) ff_tab.push_back(make_int4(c, j, nfb, 0));
      for (int t = 0; t < cfg->p.Ntau; ++t) stiles.push_back(make_int2(c, t));
      maxSliceThreads = std::max(maxSliceThreads, cfg->sl1.threads);
      b->smem_apply = std::max(b->smem_apply, (size_t)cfg->g.V * sizeof(double2));
      b->smem_force = std::max(b->smem_force, 2 * (size_t)cfg->g.V * sizeof(double2));
    }
    b->slice_threads = maxSliceThreads;
    b->n_site_tab = (int)site_tab.size();
    b->n_act_tab = (int)act_tab.size();
    b->n_ff_tab = (int)ff_tab.size();
    b->n_stiles = (int)stiles.size();
    if (!dal((void**)&b->d_resid_report, nchains * sizeof(MdagmArgs<double>)) ||
        !dal((void**)&b->d_chain, nchains * sizeof(ChainDesc)) || !dal((void**)&b->d_counter, sizeof(uint64_t)) ||
        !dal((void**)&b->d_bodies, sizeof(unsigned long long)) ||
        !dal((void**)&b->d_info, nchains * sizeof(hqmc_traj_info)) ||
        !dal((void**)&b->d_site_tab, site_tab.size() * sizeof(int4)) ||
        !dal((void**)&b->d_act_tab, act_tab.size() * sizeof(int4)) ||
        !dal((void**)&b->d_ff_tab, ff_tab.size() * sizeof(int4)) ||
        !dal((void**)&b->d_stiles, stiles.size() * sizeof(int2)) ||
        cudaMallocHost(&b->h_chain, nchains * sizeof(ChainDesc)) != cudaSuccess ||
        cudaMallocHost(&b->h_mirror, sizeof(*b->h_mirror)) != cudaSuccess ||
        cudaMallocHost(&b->h_info, nchains * sizeof(hqmc_traj_info)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      rc = bfail(b, HQMC_ENOMEM, "batch trajectory tables");
      break;
    }
    if (cudaMemcpy(b->d_site_tab, site_tab.data(), site_tab.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_act_tab, act_tab.data(), act_tab.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_ff_tab, ff_tab.data(), ff_tab.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_stiles, stiles.data(), stiles.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = bfail(b, HQMC_ECUDA, "batch trajectory table upload");
      break;
    }
    if (cudaMemcpy(b->d_ublocks, ublocks.data(), ublocks.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_unblocks, unblocks.data(), unblocks.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_states, states.data(), states.size() * sizeof(CgState*), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_ltiles, ltiles.data(), ltiles.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = bfail(b, HQMC_ECUDA, "batch table upload");
      break;
    }
    // each chain keeps the batch's cluster size C in its own partial-sum slots
    if ((rc = batch_set_tiles(b, b->C, 0)) != HQMC_OK) break;
    if (tune && (rc = batch_autotune(b)) != HQMC_OK) break;
  } while (0);
  if (rc != HQMC_OK) {
    const int keep = rc;
    batch_release(b);
    delete b;
    return keep;
  }
  *out = b;
  return HQMC_OK;
}

int hqmc_free_batch(hqmc_batch* b) {
  if (!b) return HQMC_OK;
  cudaDeviceSynchronize();
  batch_release(b);
  delete b;
  return HQMC_OK;
}

const char* hqmc_batch_last_error(const hqmc_batch* b) { return b ? b->err : "no batch"; }

int hqmc_batch_set_solver(hqmc_batch* b, int solver) {
  if (!b) return HQMC_EINVAL;
  if (solver != HQMC_SOLVER_CG64 && solver != HQMC_SOLVER_PCG64)
    return bfail(b, HQMC_EINVAL, "batched solver must be HQMC_SOLVER_CG64 or HQMC_SOLVER_PCG64");
  if (solver != b->solver && (b->exec || b->traj_exec)) {  // the loop body changes: capture again on next use
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->traj_exec) cudaGraphExecDestroy(b->traj_exec);
    b->exec = nullptr;
    b->traj_exec = nullptr;
  }
  b->solver = solver;
  return HQMC_OK;
}

int hqmc_batch_launch_shape(const hqmc_batch* b, int* cluster, int* order, int* threads, float* tuned_us) {
  if (!b) return HQMC_EINVAL;
  if (cluster) *cluster = b->C;
  if (order) *order = b->tile_order;
  if (threads) *threads = b->threads;
  if (tuned_us) *tuned_us = b->tuned_us;
  return HQMC_OK;
}

long long hqmc_batch_launch_count(const hqmc_batch* b) {
  if (!b) return 0;
  long long n = b->launches;
  for (const hqmc_config* c : b->cfgs) n += c->launches;
  return n;
}

int hqmc_batch_cg_solve(hqmc_batch* b, const double* const* theta, const void* const* phi, void* const* x, double tol,
                        int maxit, hqmc_solve_info* infos, void* stream) {
  if (!b || !theta || !phi || !x) return HQMC_EINVAL;
  if (!(tol > 0) || maxit < 0) return bfail(b, HQMC_EINVAL, "tol must be > 0 and maxit >= 0");
  const int nc = (int)b->cfgs.size();
  for (int c = 0; c < nc; ++c)
    if (!aligned16(theta[c]) || !aligned16(phi[c]) || !aligned16(x[c]))
      return bfail(b, HQMC_EINVAL, "chain %d: NULL or misaligned pointer", c);
  cudaStream_t s = (cudaStream_t)stream;
  for (int c = 0; c < nc; ++c) BRET(links(b->cfgs[c], theta[c], true, false, s), b->cfgs[c]);
  return batch_solve(b, (const double2* const*)phi, (double2* const*)x, tol, maxit, infos, s);
}

int hqmc_batch_trajectory(hqmc_batch* b, double* const* theta, const uint64_t* seeds, uint64_t traj_counter,
                          int nsteps, const double* dt, double tol, int maxit, hqmc_traj_info* infos, void* stream) {
  if (!b || !theta || !seeds || !dt) return HQMC_EINVAL;
  if (nsteps < 0 || !(tol > 0) || maxit < 0) return bfail(b, HQMC_EINVAL, "bad step parameters");
  const int nc = (int)b->cfgs.size();
  for (int c = 0; c < nc; ++c)
    if (!aligned16(theta[c]) || !std::isfinite(dt[c])) return bfail(b, HQMC_EINVAL, "chain %d: bad theta or dt", c);
  cudaStream_t s = (cudaStream_t)stream;
  // per-chain descriptors of this trajectory (field pointer, seed and dt may change between calls)
  std::vector<const double2*> eta(nc);
  std::vector<double2*> X(nc);
  for (int c = 0; c < nc; ++c) {
    hqmc_config* cfg = b->cfgs[c];
    ChainDesc& d = b->h_chain[c];
    d = ChainDesc{};
    d.g = cfg->g;
    d.bp = cfg->bp;
    d.cB = cfg->cB;
    d.t1 = cfg->t1;
    d.t2 = cfg->t2;
    d.inv1 = 1.0 / (1.0 - cfg->t1 * cfg->t1);  // as the single-chain force launch forms them
    d.inv2 = 1.0 / (1.0 - cfg->t2 * cfg->t2);
    d.n = cfg->n;
    d.theta = theta[c];
    d.th0 = cfg->th0;
    d.p = cfg->pm;
    d.R = cfg->Rw;
    d.eta = cfg->eta;
    d.X = cfg->Xw;
    d.F = cfg->F;
    d.dSf = cfg->dSf;
    d.U64 = cfg->U64;
    d.part_act = cfg->part_act;
    d.act_grid = cfg->act_grid;
    d.terms = cfg->terms;
    d.st = cfg->st;
    d.report = cfg->report;
    d.seed = seeds[c];
    d.dt = dt[c];
    d.info = b->d_info + c;
    eta[c] = cfg->eta;
    X[c] = cfg->Xw;
  }
  int rc = batch_descriptors(b, eta.data(), X.data(), s);
  if (rc != HQMC_OK) return rc;
  BCK(cudaMemcpyAsync(b->d_chain, b->h_chain, nc * sizeof(ChainDesc), cudaMemcpyHostToDevice, s));
  b->h_mirror->counter = traj_counter;
  BCK(cudaMemcpyAsync(b->d_counter, &b->h_mirror->counter, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  BCK(cudaMemsetAsync(b->d_bodies, 0, sizeof(unsigned long long), s));
  if ((rc = traj_graph(b, nsteps, tol, maxit)) != HQMC_OK) return rc;
  NvtxRange nv("hqmc batched trajectory");
  BCK(cudaGraphLaunch(b->traj_exec, s));
  BCK(cudaMemcpyAsync(b->h_info, b->d_info, nc * sizeof(hqmc_traj_info), cudaMemcpyDeviceToHost, s));
  BCK(cudaMemcpyAsync(&b->h_mirror->bodies, b->d_bodies, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  const bool pc = b->solver == HQMC_SOLVER_PCG64;
  const long long body = (pc ? 3 : 2) * kBodyIters64 + 3 + (pc ? 1 : 0) + 1;  // with the loop condition
  b->launches += b->traj_static_kernels + (long long)b->h_mirror->bodies * body;
  int worst = HQMC_OK;
  for (int c = 0; c < nc; ++c) {
    if (infos) infos[c] = b->h_info[c];
    worst = merge_status(worst, b->h_info[c].status);
  }
  return worst;
}

}  // extern "C"

// ===========================================================================
// Learned preconditioner API.

namespace {

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int net_upload(hqmc_net* net, const float* host) {
  std::vector<__nv_bfloat16> hb(net->total);
  for (int e = 0; e < net->total; ++e) hb[e] = __float2bfloat16(host[e]);
  if (cudaMemcpy(net->w, host, net->total * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(net->wb, hb.data(), net->total * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->m, 0, net->total * sizeof(float)) != cudaSuccess ||
      cudaMemset(net->v, 0, net->total * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return HQMC_ECUDA;
  }
  net->hw.resize(net->total);
  for (int e = 0; e < net->total; ++e) net->hw[e] = __bfloat162float(hb[e]);
  net->hw_valid = 1;
  net->steps = 0;
  net->version++;
  return HQMC_OK;
}

}  // namespace

extern "C" {

int hqmc_net_create(uint64_t seed, hqmc_net** out) {
  if (!out) return HQMC_EINVAL;
  *out = nullptr;
  hqmc_net* net = new (std::nothrow) hqmc_net();
  if (!net) return HQMC_ENOMEM;
  cudaGetDevice(&net->device);
  for (int l = 0; l < kNetLayers; ++l) net->off[l + 1] = net->off[l] + 7 * net->cin[l] * net->cout[l];
  net->total = net->off[kNetLayers];
  const size_t n = net->total;
  if (cudaMalloc((void**)&net->w, n * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&net->m, n * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&net->v, n * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&net->wb, n * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&net->wt, n * sizeof(__nv_bfloat16)) != cudaSuccess) {
    cudaGetLastError();
    hqmc_net_free(net);
    return HQMC_ENOMEM;
  }
  // start from the identity map r -> r (channel 0 carried by the centre taps)
  // plus a small random perturbation of every weight
  std::vector<float> w(n);
  uint64_t st = seed ^ 0x5DEECE66Dull;
  for (size_t e = 0; e < n; ++e) w[e] = (float)(((splitmix64(st) >> 11) * (1.0 / 9007199254740992.0)) - 0.5) * 0.02f;
  for (int l = 0; l < kNetLayers; ++l) {
    float* wl = w.data() + net->off[l];
    const int ci = net->cin[l], co = net->cout[l];
    for (int c = 0; c < co && c < ci; ++c) wl[(0 * co + c) * ci + c] += 1.0f;  // centre tap, c -> c
  }
  const int rc = net_upload(net, w.data());
  if (rc != HQMC_OK) {
    hqmc_net_free(net);
    return rc;
  }
  *out = net;
  return HQMC_OK;
}

int hqmc_net_free(hqmc_net* net) {
  if (!net) return HQMC_OK;
  cudaDeviceSynchronize();
  cudaFree(net->w);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->wb);
  cudaFree(net->wt);
  delete net;
  return HQMC_OK;
}

int hqmc_net_num_weights(const hqmc_net* net) { return net ? net->total : 0; }

int hqmc_net_get_weights(const hqmc_net* net, float* host, int n) {
  if (!net || !host || n != net->total) return HQMC_EINVAL;
  if (cudaMemcpy(host, net->w, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return HQMC_ECUDA;
  return HQMC_OK;
}

int hqmc_net_set_weights(hqmc_net* net, const float* host, int n) {
  if (!net || !host || n != net->total) return HQMC_EINVAL;
  return net_upload(net, host);
}

int hqmc_net_apply(hqmc_config* cfg, hqmc_net* net, const double* theta, const void* r, void* z, void* stream) {
  if (!cfg || !net) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(r) || !aligned16(z)) return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  RET(check_device(cfg));
  if (!net_ready(cfg))
    return fail(cfg, HQMC_EINVAL, "no net workspace on this config: attach a net with hqmc_set_preconditioner first");
  cudaStream_t s = (cudaStream_t)stream;
  RET(theta_float(cfg, theta, s));
  return net_forward(cfg, net, (const double2*)r, (double2*)z, s);
}

int hqmc_net_train_step(hqmc_config* cfg, hqmc_net* net, const double* theta, const void* phi, const void* x,
                        double lr, double* loss_host, void* stream) {
  if (!cfg || !net || !(lr >= 0)) return HQMC_EINVAL;
  if (!aligned16(theta) || !aligned16(phi) || !aligned16(x)) return fail(cfg, HQMC_EINVAL, "NULL or misaligned pointer");
  RET(check_device(cfg));
  if (!net_ready(cfg))
    return fail(cfg, HQMC_EINVAL, "no net workspace on this config: attach a net with hqmc_set_preconditioner first");
  cudaStream_t s = (cudaStream_t)stream;
  RET(theta_float(cfg, theta, s));
  RET(net_forward(cfg, net, (const double2*)phi, nullptr, s, false));  // activations h0..h4
  net->hw_valid = 0;  // this step's Adam update changes the device weights
  net->version++;
  // ||x||^2 on the device, then the loss and its gradient with respect to h4
  LK(2, launch_action_terms(cfg->g, cfg->bp, theta, nullptr, (const double2*)x, (const double2*)x, cfg->act_grid,
                            cfg->part_act, cfg->terms, s));
  double* loss_part = cfg->net_part + (size_t)kNetChunks * 7 * kNetCh * kNetCh;
  const int lblocks = 512;
  LK(1, launch_net_loss(cfg->net_h[kNetLayers], (const double2*)x, cfg->terms + 2, cfg->net_d[0], loss_part, lblocks,
                        cfg->n, s));
  // backward: layer l uses d_{l+1} and h_l; the adjoint weights are taken before the update
  net->steps++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)net->steps), c2 = 1.f - std::pow(b2, (float)net->steps);
  int din = 0;
  for (int l = kNetLayers - 1; l >= 0; --l) {
    const int ci = net->cin[l], co = net->cout[l];
    const int nw = 7 * ci * co;
    LK(1, launch_net_wgrad(cfg->g, cfg->th32, ci, co, cfg->net_d[din], cfg->net_h[l], cfg->net_part, kNetChunks, s));
    if (l > 0) {
      void* wt = (char*)net->wt + 2 * (size_t)net->off[l];
      LK(1, launch_net_adjoint_weights((char*)net->wb + 2 * (size_t)net->off[l], wt, ci, co, s));
      LK(1, launch_net_layer(cfg->g, cfg->th32, wt, co, ci, cfg->net_d[din], cfg->net_d[din ^ 1], s));
    }
    LK(1, launch_net_adam(net->w + net->off[l], net->m + net->off[l], net->v + net->off[l], cfg->net_part, kNetChunks,
                          nw, (char*)net->wb + 2 * (size_t)net->off[l], (float)lr, b1, b2, c1, c2, 1e-8f, 1.f, s));
    din ^= 1;
  }
  if (loss_host) {
    std::vector<double> lp(lblocks);
    CK(cudaMemcpyAsync(cfg->vscratch, loss_part, lblocks * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(lp.data(), loss_part, lblocks * sizeof(double), cudaMemcpyDeviceToHost));
    double sum = 0.0;
    for (double v : lp) sum += v;
    *loss_host = sum;
  }
  return HQMC_OK;
}

int hqmc_set_guess_history(hqmc_config* cfg, int k) {
  if (!cfg || k < 0 || k > 8) return HQMC_EINVAL;
  if (k > cfg->guess_cap) {
    RET(check_device(cfg));
    // the guess's many-dot partials and results live in the config's scratch vector
    if (2 * (size_t)cfg->act_grid * k + 2 * (size_t)k > 2 * (size_t)cfg->n)
      return fail(cfg, HQMC_EUNSUPPORTED, "lattice too small for a guess history of %d", k);
    double2 *h = nullptr, *q = nullptr;
    RET(dalloc(cfg, &h, (size_t)k * cfg->n));
    RET(dalloc(cfg, &q, (size_t)k * cfg->n));
    cfg->hist = h;
    cfg->qbasis = q;
    cfg->guess_cap = k;
  }
  cfg->guess_k = k;
  cfg->hist_n = cfg->hist_next = 0;
  return HQMC_OK;
}

int hqmc_set_net_interval(hqmc_config* cfg, int k) {
  if (!cfg || k < 1) return HQMC_EINVAL;
  if (k == cfg->net_interval) return HQMC_OK;
  cfg->net_interval = k;
  CK(cudaDeviceSynchronize());  // no cached loop graph may still be running
  for (auto& g : cfg->graphs) cudaGraphExecDestroy(g.exec);
  cfg->graphs.clear();
  return HQMC_OK;
}

int hqmc_set_net_tensor_cores(hqmc_config* cfg, int on) {
  if (!cfg || (on != 0 && on != 1)) return HQMC_EINVAL;
  if (on == cfg->net_tc) return HQMC_OK;
  cfg->net_tc = on;
  CK(cudaDeviceSynchronize());  // no cached loop graph may still be running
  for (auto& g : cfg->graphs) cudaGraphExecDestroy(g.exec);
  cfg->graphs.clear();
  return HQMC_OK;
}

int hqmc_set_preconditioner(hqmc_config* cfg, hqmc_net* net) {
  if (!cfg) return HQMC_EINVAL;
  if (net) {
    RET(check_device(cfg));
    if (net->device != cfg->device)
      return fail(cfg, HQMC_EINVAL, "net belongs to device %d, config to device %d", net->device, cfg->device);
    RET(net_workspace(cfg));
  }
  cfg->net = net;
  return HQMC_OK;
}

}  // extern "C"
