// C ABI of the Basic-Scheme solver (declared in include/fftHomog.h).
//
// Host orchestration only: argument checks, device memory, the Gamma^p table
// build, and the iteration loop.  The iteration body (row pass + line passes,
// see kernels.cuh) is captured once per (precision, load count, chunk) into a
// CUDA graph of `chunk` iterations; the host replays it and reads one flag per
// replay.  Loads that have converged make their blocks return at entry, so the
// per-load iteration counts are exact.

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.hpp"
#include "kernels.cuh"
#include "cluster.cuh"
#include "warprow.cuh"
#include "linewarp.cuh"
#include "colpass2.cuh"
#include "rowpass2.cuh"
#include "krylov.cuh"
#include "planewarp.cuh"

namespace fh {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace fh

using fh::Control;
using fh::DevPlan;
using fh::GridInfo;
using fh::LoadState;

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      fh::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
      return FH_ERR_CUDA;                                                            \
    }                                                                                \
  } while (0)

namespace {

// NVTX range over a host call (header-only NVTX 3: inert unless a profiler
// attaches), so that a timeline shows the table build, the phases of a solve
// and the batched queue launches by name
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kThreads = 256;
constexpr int kMeanBlocks = 512;   // blocks per load of the mean-stress reduction
constexpr int kHistCap = 65536;
constexpr size_t kMaxSmem = 227 * 1024;
constexpr int kMaxPhases = 16;

int mandel_nv(int d) { return d == 2 ? 3 : 6; }

struct Axis {
  int L = 1;
  DevPlan plan{};        // radix schedule of the cluster kernel (and the default)
  DevPlan planp[2]{};    // radix schedule of the passes per bulk precision (autotuned)
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
};

struct GraphEntry {
  int prec, nload, chunk, method;
  cudaGraphExec_t exec;
};

}  // namespace

struct fh_solver {
  fh::Pattern P;
  fh_generator gen{};
  cudaStream_t user = nullptr;
  cudaStream_t work = nullptr;
  int nload_max = 0;
  GridInfo g{};
  Axis ax[3];
  // device memory
  double* E64 = nullptr;
  float* E32 = nullptr;
  void* S = nullptr;
  uint8_t* phase = nullptr;
  double* Cp64 = nullptr;
  double* dC64 = nullptr;
  float* dC32 = nullptr;
  float* Cp32 = nullptr;
  int form = 0;  // iteration form of the solve in progress (0 or 1)
  bool dc_decoupled = false;  // 3-D phase matrices and C0 with zero normal-shear blocks, diagonal shear block
  bool polish = false;        // the FP64 phase of a mixed solve is in progress
  // autotuned (path, cluster size) per bulk precision [fp64, fp32]; path 0 = not tuned yet
  int tuned_path[2] = {0, 0};
  int tuned_cs[2] = {0, 0};
  float tuned_us[2][FH_TUNE_CANDIDATES] = {};  // per-iteration time of each autotuner candidate (-1: not eligible)
  int tuned_cand[2] = {0, 0};                   // the candidate chosen
  double* G64 = nullptr;
  float* G32 = nullptr;
  Control* ctl = nullptr;
  LoadState* st = nullptr;
  double* partials = nullptr;
  double* partials2 = nullptr;
  double* hist = nullptr;
  double* mstress = nullptr;
  int* err = nullptr;
  double* scratch64 = nullptr;  // nv*m doubles, for strain copies
  int* h_flag = nullptr;        // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_user = nullptr;
  // host state
  int nphase = 0;
  double Cp[kMaxPhases * 36] = {};
  double C0[36] = {};
  bool have_phases = false, have_table = false;
  int E_prec = -1;  // precision of the strain currently held in E
  int last_nload = 0;
  double last_eps0[FH_MAX_LOADS * 6] = {};
  double last_ms[FH_MAX_LOADS * 6] = {};
  bool have_solution = false;
  int last_iters[FH_MAX_LOADS] = {};
  // launch shapes per precision (0: fp64, 1: fp32)
  int rpb[2] = {1, 1};
  int row_warp[2] = {0, 0};  // > 0: warp-per-row pass with L = 32 * row_warp
  int plane[2] = {0, 0};     // 3-D FP32: > 0 = the fused plane pass applies (axis-1 P, axis-2 P packed as 10 P1 + P2)
  bool plane_on = false;     // path 3 of the solve in progress: take the fused plane pass where it applies
  bool col2s = true;         // rows and columns of 32, 64 or 128 points: the two-step passes (else the earlier forms)
  int row2[2] = {0, 0};      // 3-D fields with rows of 32, 64 or 128 points: the two-step row pass applies (L), else 0
  int row2_bpl[2] = {1, 1};  // its blocks per load
  bool skip_mean = false;   // the phase in progress is followed by another (mixed mode): its mean stress is not used
  int warp_res[2] = {0, 0};  // resident blocks per SM of that pass
  int sms = 0;               // multiprocessors of the device
  int row_bpl[2] = {1, 1};
  size_t row_smem[2] = {0, 0};
  int lineW[2][3] = {};
  int ntiles[2][3] = {};
  size_t line_smem[2][3] = {};
  std::vector<GraphEntry> graphs;
  bool cl_gsmem[2][2] = {{true, true}, {true, true}};  // [fp64/fp32][cluster 8/16]: table slice in smem
  LoadState* h_states = nullptr;                       // pinned copies read back after a phase
  double* h_ms = nullptr;
  fh::ClusterTask* qtasks = nullptr;                    // cluster-kernel task list of a single solve
  unsigned int* qnext = nullptr;
  fh::ClusterTask* h_tasks = nullptr;                   // pinned staging of that list
  // BiCGStab (fh_solve_opts.method = 1): fields r, rhat, p, v, s, t per bulk
  // precision (allocated on first use), scalars, block sums, and a copy of
  // the control block with a zero macroscopic strain for operator applications
  int method = 0;
  // point-by-point stiffness (fh_set_stiffness_field with more than 16 distinct
  // matrices): C(x), C(x) - C0 (FP64, FP32) and C(x) in FP32, upper triangle
  // [tri][m]; such solves take the block row pass on the whole-GPU passes
  bool field = false;
  double* Cf64 = nullptr;
  double* dCf64 = nullptr;
  float* dCf32 = nullptr;
  float* Cf32 = nullptr;
  double field_lam[2] = {0, 0}, field_mu[2] = {0, 0};  // ranges over the points (reference-medium rule)
  // shapes of the block row pass per precision (the warp and plane passes
  // replace it where they apply, the point-by-point stiffness needs it)
  int rpb_gen[2] = {1, 1};
  int row_bpl_gen[2] = {1, 1};
  size_t row_smem_gen[2] = {0, 0};
  // the shapes and radix schedules choose_shapes and make_plan gave, per bulk
  // precision: the autotuner's candidates start from these
  struct PassShapes {
    int rpb_gen, row_bpl_gen;
    size_t row_smem_gen;
    int lineW[3], ntiles[3];
    size_t line_smem[3];
    fh::DevPlan plans[3];
  } shape_def[2];
  void* kbuf[2] = {nullptr, nullptr};
  fh::KrylovScal* ksc = nullptr;
  double* kpart = nullptr;
  Control* ctl0 = nullptr;
};

namespace {

size_t csize(int prec) { return prec == FH_PREC_FP64 ? sizeof(double2) : sizeof(float2); }

size_t plane_smem_of(int P1, int P2) {
  const int N1 = 32 * P1, L = 32 * P2, H = L / 2 + 1;
  return (size_t)(3 * N1 * H + N1 + L + fh::kPlaneWarps * fh::plane_ws(L)) * sizeof(float2);
}

void choose_shapes(fh_solver* s, int prec) {
  const GridInfo& g = s->g;
  const int sms = 152;
  const int nl = s->nload_max;
  const int Lp = prec == FH_PREC_FP64 ? fh::padded_len<3>(g.L) : fh::padded_len<4>(g.L);
  auto row_smem = [&](int rpb) { return (size_t)2 * ((rpb * g.nv + 1) / 2) * Lp * csize(prec); };
  // rows per block: grow while the grid keeps >= 2 blocks per SM and a block's
  // shared memory stays small enough for several resident blocks
  const size_t row_smem_cap = 96 * 1024;
  int rpb = 1;
  while (rpb * 2 <= g.nrows && (g.nrows * nl) / (rpb * 2) >= 2 * sms && row_smem(rpb * 2) <= row_smem_cap) rpb *= 2;
  s->rpb[prec] = rpb;
  s->row_bpl[prec] = (int)((g.nrows + rpb - 1) / rpb);
  s->row_smem[prec] = row_smem(rpb);
  s->rpb_gen[prec] = rpb;
  s->row_bpl_gen[prec] = s->row_bpl[prec];
  s->row_smem_gen[prec] = s->row_smem[prec];
  // FP32 3-D grids whose contiguous axis is 32, 64, 128 or 256 points long
  // take the warp-per-row pass (FP64 keeps the block pass: its radix-8
  // stages need fewer operations on the narrow FP64 pipe)
  s->row_warp[prec] = 0;
  if (prec == FH_PREC_FP32 && g.nv == 6 && g.L % 32 == 0) {
    const int P = g.L / 32;
    if (P == 1 || P == 2 || P == 4 || P == 8) {
      const int nw = fh::kWarpRowThreads / 32;
      s->row_warp[prec] = P;
      s->row_bpl[prec] = (int)((g.nrows + nw - 1) / nw);
      s->row_smem[prec] = fh::warprow_smem<float>(g.L);
    }
  }
  // FP64 3-D fields whose contiguous axis is 32, 64 or 128 points long: the
  // two-step row pass (128^3 x 6 loads: 5.4 ms against 7.5 ms for the block
  // row pass; in FP32 the warp row pass is faster, 0.288 against 0.354 ms)
  s->row2[prec] = 0;
  if (prec == FH_PREC_FP64 && g.nv == 6 && (g.L == 32 || g.L == 64 || g.L == 128)) {
    const int rb = g.L == 32 ? fh::Row2<4, 8>::RB : fh::Row2<8, 8>::RB;
    s->row2[prec] = g.L;
    s->row2_bpl[prec] = (int)((g.nrows + rb - 1) / rb);
  }
  // FP32 3-D grids whose axis-1 and axis-2 lengths are 32, 64 or 128 points
  // (and whose plane fits in a CTA's shared memory): the fused plane pass
  s->plane[prec] = 0;
  if (prec == FH_PREC_FP32 && g.nv == 6 && g.nd == 3 && s->row_warp[prec] > 0) {
    const int P1 = g.dims[1] % 32 == 0 ? g.dims[1] / 32 : 0, P2 = s->row_warp[prec];
    if ((P1 == 1 || P1 == 2 || P1 == 4) && (P2 == 1 || P2 == 2 || P2 == 4) && plane_smem_of(P1, P2) + 4096 <= kMaxSmem)
      s->plane[prec] = 10 * P1 + P2;
  }
  for (int a = 0; a + 1 < g.nd; ++a) {
    const int N = g.dims[a];
    long long others = 1;
    for (int k = 0; k + 1 < g.nd; ++k)
      if (k != a) others *= g.dims[k];
    int W = 16;
    auto smem = [&](int w) { return (size_t)2 * g.nv * w * (N + 1) * csize(prec); };
    auto blocks = [&](int w) { return (long long)nl * others * ((g.H + w - 1) / w); };
    const int wmin = prec == FH_PREC_FP64 ? 2 : 4;
    // FP64 allows a wider tile (four 128-point columns: 99 KB, two blocks per
    // SM), measured faster than two (5.07 against 5.38 ms for the axis-0 pass
    // at 128^3 x 6 loads)
    const size_t line_cap = (prec == FH_PREC_FP64 ? 112 : 96) * 1024;
    while (W > wmin && (smem(W) > line_cap || blocks(W) < 2 * sms)) W /= 2;
    while (W > 1 && smem(W) > kMaxSmem) W /= 2;
    s->lineW[prec][a] = W;
    s->ntiles[prec][a] = (g.H + W - 1) / W;
    s->line_smem[prec][a] = smem(W);
  }
}

void save_default_shapes(fh_solver* s) {
  for (int prec = 0; prec < 2; ++prec) {
    fh_solver::PassShapes& d = s->shape_def[prec];
    d.rpb_gen = s->rpb_gen[prec];
    d.row_bpl_gen = s->row_bpl_gen[prec];
    d.row_smem_gen = s->row_smem_gen[prec];
    for (int a = 0; a < 3; ++a) {
      d.lineW[a] = s->lineW[prec][a];
      d.ntiles[a] = s->ntiles[prec][a];
      d.line_smem[a] = s->line_smem[prec][a];
      d.plans[a] = s->ax[a].planp[prec];
    }
  }
}

void clear_graphs(fh_solver* s) {
  for (auto& e : s->graphs) cudaGraphExecDestroy(e.exec);
  s->graphs.clear();
}

template <typename T>
const typename fh::cplx_t<T>::type* twp(const Axis& a);
template <>
const double2* twp<double>(const Axis& a) { return a.tw64; }
template <>
const float2* twp<float>(const Axis& a) { return a.tw32; }

template <typename T>
T* Eptr(fh_solver* s);
template <>
double* Eptr<double>(fh_solver* s) { return s->E64; }
template <>
float* Eptr<float>(fh_solver* s) { return s->E32; }

// stiffness table of the pointwise stage: C - C0 for Eq. (pde_coefficients),
// C itself for the variational form
template <typename T>
const T* dCptr(fh_solver* s);
template <>
const double* dCptr<double>(fh_solver* s) { return s->form == 1 ? s->Cp64 : s->dC64; }
template <>
const float* dCptr<float>(fh_solver* s) { return s->form == 1 ? s->Cp32 : s->dC32; }

template <typename T>
const T* Gptr(fh_solver* s);
template <>
const double* Gptr<double>(fh_solver* s) { return s->G64; }
template <>
const float* Gptr<float>(fh_solver* s) { return s->G32; }

template <typename T, int NV>
void launch_line_nv(fh_solver* s, int prec, int a, int mode, unsigned blocks, int n_outer, int n_inner) {
  using C = typename fh::cplx_t<T>::type;
  C* S = reinterpret_cast<C*>(s->S);
  const size_t sm = s->line_smem[prec][a];
  const int W = s->lineW[prec][a], nt = s->ntiles[prec][a];
  if (mode == 0)
    fh::line_pass<T, NV, 0><<<blocks, kThreads, sm, s->work>>>(s->g, s->ax[a].planp[prec], twp<T>(s->ax[a]), S, Gptr<T>(s), s->st, a, W, nt, n_outer, n_inner);
  else if (mode == 1)
    fh::line_pass<T, NV, 1><<<blocks, kThreads, sm, s->work>>>(s->g, s->ax[a].planp[prec], twp<T>(s->ax[a]), S, Gptr<T>(s), s->st, a, W, nt, n_outer, n_inner);
  else
    fh::line_pass<T, NV, 2><<<blocks, kThreads, sm, s->work>>>(s->g, s->ax[a].planp[prec], twp<T>(s->ax[a]), S, Gptr<T>(s), s->st, a, W, nt, n_outer, n_inner);
}

template <typename T>
void launch_line(fh_solver* s, int prec, int a, int mode, unsigned blocks, int n_outer, int n_inner) {
  if (s->g.nv == 3) launch_line_nv<T, 3>(s, prec, a, mode, blocks, n_outer, n_inner);
  else launch_line_nv<T, 6>(s, prec, a, mode, blocks, n_outer, n_inner);
}

// Warp-per-column line pass (FP32, 3-D fields) for an axis of 32, 64, 128 or
// 256 points: P = N / 32, else 0.
int col_warp_p(const fh_solver* s, int prec, int a) {
  if (prec != FH_PREC_FP32 || s->g.nv != 6) return 0;
  const int N = s->g.dims[a];
  return (N == 32 || N == 64 || N == 128 || N == 256) ? N / 32 : 0;
}

template <int P, int MODE>
void launch_col_pass(fh_solver* s, int a, int nload) {
  const GridInfo& g = s->g;
  long long stride = g.H;
  for (int k = a + 1; k + 1 < g.nd; ++k) stride *= g.dims[k];
  const long long ncols = g.nhalf / g.dims[a];
  const long long tiles = (ncols + fh::kColTile - 1) / fh::kColTile;
  fh::line_pass_warp6<P, MODE><<<(unsigned)(tiles * nload), fh::kColThreads, fh::colpass_smem<P>(), s->work>>>(
      g, s->ax[a].tw32, reinterpret_cast<float2*>(s->S), s->G32, s->st, stride, ncols, nload);
}

template <int P>
void launch_col_pass_mode(fh_solver* s, int a, int mode, int nload) {
  if (mode == 0) launch_col_pass<P, 0>(s, a, nload);
  else if (mode == 1) launch_col_pass<P, 1>(s, a, nload);
  else launch_col_pass<P, 2>(s, a, nload);
}

// The two-step column pass (colpass2.cuh) applies to the axes of 32, 64 or
// 128 points of 3-D fields (either precision): returns N there, else 0.
int col2_len(const fh_solver* s, int prec, int a) {
  (void)prec;
  if (!s->col2s || s->g.nv != 6) return 0;
  const int N = s->g.dims[a];
  return (N == 32 || N == 64 || N == 128) ? N : 0;
}

// columns per block and resident blocks per SM of the two-step column pass:
// 8 in FP32, 4 in FP64 (whose tile of 8 would leave one block per SM)
template <typename T>
constexpr int col2_ct() { return sizeof(T) == 4 ? fh::kColTile : 4; }
template <typename T, int MODE>
constexpr int col2_mb() { return sizeof(T) == 4 ? fh::col2_minb<MODE>() : 3; }

template <typename T, int R1, int R2, int MODE>
void launch_col2(fh_solver* s, int a, int nload) {
  using C = typename fh::cplx_t<T>::type;
  constexpr int CT = col2_ct<T>();
  const GridInfo& g = s->g;
  long long stride = g.H;
  for (int k = a + 1; k + 1 < g.nd; ++k) stride *= g.dims[k];
  const long long ncols = g.nhalf / g.dims[a];
  const long long tiles = (ncols + CT - 1) / CT;
  fh::line_pass_2s<R1, R2, MODE, CT, col2_mb<T, MODE>(), T>
      <<<(unsigned)(tiles * nload), fh::Col2<R1, R2, CT, T>::THREADS, fh::col2_smem<R1, R2, CT, T>(), s->work>>>(
          g, twp<T>(s->ax[a]), reinterpret_cast<C*>(s->S), Gptr<T>(s), s->st, stride, ncols, nload);
}

template <typename T, int R1, int R2>
void launch_col2_mode(fh_solver* s, int a, int mode, int nload) {
  if (mode == 0) launch_col2<T, R1, R2, 0>(s, a, nload);
  else if (mode == 1) launch_col2<T, R1, R2, 1>(s, a, nload);
  else launch_col2<T, R1, R2, 2>(s, a, nload);
}

// line pass along axis a in the given mode (0 forward, 1 inverse, 2 forward +
// Green + inverse), by the warp-per-column kernel where it applies
template <typename T>
void launch_axis(fh_solver* s, int prec, int a, int mode, int nload) {
  const GridInfo& g = s->g;
  switch (col2_len(s, prec, a)) {
    case 32: launch_col2_mode<T, 4, 8>(s, a, mode, nload); return;
    case 64: launch_col2_mode<T, 8, 8>(s, a, mode, nload); return;
    case 128: launch_col2_mode<T, 8, 16>(s, a, mode, nload); return;
    default: break;
  }
  if constexpr (sizeof(T) == 4) {
    switch (col_warp_p(s, prec, a)) {
      case 1: launch_col_pass_mode<1>(s, a, mode, nload); return;
      case 2: launch_col_pass_mode<2>(s, a, mode, nload); return;
      case 4: launch_col_pass_mode<4>(s, a, mode, nload); return;
      case 8: launch_col_pass_mode<8>(s, a, mode, nload); return;
      default: break;
    }
  }
  long long n_outer = 1, n_inner = 1;
  for (int k = 0; k < a; ++k) n_outer *= g.dims[k];
  for (int k = a + 1; k + 1 < g.nd; ++k) n_inner *= g.dims[k];
  const long long blocks = (long long)nload * n_outer * n_inner * s->ntiles[prec][a];
  launch_line<T>(s, prec, a, mode, (unsigned)blocks, (int)n_outer, (int)n_inner);
}

// the fused plane pass applies: FP32, an eligible 3-D grid, asked for (path 3)
bool use_plane(const fh_solver* s, int prec) {
  return prec == FH_PREC_FP32 && s->plane[prec] > 0 && s->plane_on && !s->field;
}

// Enqueue the line passes of one iteration (everything between two row passes).
template <typename T>
void enqueue_line_passes(fh_solver* s, int prec, int nload, bool plane_ok = true) {
  const GridInfo& g = s->g;
  using C = typename fh::cplx_t<T>::type;
  C* S = reinterpret_cast<C*>(s->S);
  if (g.nd == 1) {
    const long long total = (long long)nload * g.nhalf;
    const int blocks = (int)std::min<long long>((total + kThreads - 1) / kThreads, 4096);
    fh::green_1d<T><<<blocks, kThreads, 0, s->work>>>(g, S, Gptr<T>(s), s->st, nload);
    return;
  }
  auto launch = [&](int a, int mode) { launch_axis<T>(s, prec, a, mode, nload); };
  if (plane_ok && use_plane(s, prec)) {   // the plane pass transforms axes 1 and 2
    launch(0, 2);
    return;
  }
  // forward along axes nd-2 .. 1, then axis 0 with the Green step, then inverse 1 .. nd-2
  for (int a = g.nd - 2; a >= 1; --a) launch(a, 0);
  launch(0, 2);
  for (int a = 1; a <= g.nd - 2; ++a) launch(a, 1);
}

// the point-by-point stiffness of the constitutive stage (null: phase table)
template <typename T>
const T* field_ptr(const fh_solver* s, int form);
template <>
const double* field_ptr<double>(const fh_solver* s, int form) { return !s->field ? nullptr : form == 1 ? s->Cf64 : s->dCf64; }
template <>
const float* field_ptr<float>(const fh_solver* s, int form) { return !s->field ? nullptr : form == 1 ? s->Cf32 : s->dCf32; }

template <typename T, int NV, bool FIRST>
void enqueue_row_pass_nv(fh_solver* s, int prec, int nload) {
  const GridInfo& g = s->g;
  using C = typename fh::cplx_t<T>::type;
  const int last = g.nd - 1;
  const int bpl = s->row_bpl_gen[prec];
  fh::row_pass<T, NV, FIRST><<<nload * bpl, kThreads, s->row_smem_gen[prec], s->work>>>(
      g, s->ax[last].planp[prec], twp<T>(s->ax[last]), Eptr<T>(s), reinterpret_cast<C*>(s->S), s->phase, dCptr<T>(s), s->ctl,
      s->st, s->partials, s->hist, s->rpb_gen[prec], bpl, nullptr, nullptr, field_ptr<T>(s, s->form));
}

template <typename T, int P, bool FIRST>
void enqueue_row_pass_warp(fh_solver* s, int prec, int nload) {
  using C = typename fh::cplx_t<T>::type;
  // at most one wave of resident blocks, split evenly over the loads
  // (row_bpl, one row per warp, is the bound the partial-sum buffer is sized for)
  const int resident = std::max(1, s->warp_res[prec]) * std::max(1, s->sms);
  const int bpl = std::max(1, std::min(s->row_bpl[prec], resident / nload));
  fh::row_pass_warp6<T, P, FIRST><<<nload * bpl, fh::kWarpRowThreads, s->row_smem[prec], s->work>>>(
      s->g, twp<T>(s->ax[s->g.nd - 1]), Eptr<T>(s), reinterpret_cast<C*>(s->S), s->phase, dCptr<T>(s), s->ctl, s->st,
      s->partials, s->hist, bpl);
}

// the fused plane pass (planewarp.cuh): one cluster of two CTAs per plane x0
// and load
template <int P1, int P2, bool FIRST>
void launch_plane(fh_solver* s, int nload) {
  const GridInfo& g = s->g;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * g.dims[0] * nload));
  cfg.blockDim = dim3(fh::kPlaneThreads);
  cfg.dynamicSmemBytes = fh::plane_smem<P1, P2>();
  cfg.stream = s->work;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, fh::plane_pass_warp6<P1, P2, FIRST>, g, (const float2*)s->ax[1].tw32,
                     (const float2*)s->ax[2].tw32, s->E32, reinterpret_cast<float2*>(s->S), (const uint8_t*)s->phase,
                     (const float*)dCptr<float>(s), s->ctl, s->st, s->partials, s->hist);
}

template <bool FIRST>
void enqueue_plane(fh_solver* s, int nload) {
  switch (s->plane[FH_PREC_FP32]) {
    case 11: launch_plane<1, 1, FIRST>(s, nload); break;
    case 12: launch_plane<1, 2, FIRST>(s, nload); break;
    case 14: launch_plane<1, 4, FIRST>(s, nload); break;
    case 21: launch_plane<2, 1, FIRST>(s, nload); break;
    case 22: launch_plane<2, 2, FIRST>(s, nload); break;
    case 24: launch_plane<2, 4, FIRST>(s, nload); break;
    case 41: launch_plane<4, 1, FIRST>(s, nload); break;
    case 42: launch_plane<4, 2, FIRST>(s, nload); break;
    default: launch_plane<4, 4, FIRST>(s, nload); break;
  }
}

// the two-step row pass (rowpass2.cuh) applies: rows of 32, 64 or 128
// points of 3-D fields, phase-wise stiffness, not switched off by the
// autotuner's candidate 5
bool use_row2(const fh_solver* s, int prec) { return s->col2s && s->row2[prec] > 0 && !s->field; }

template <typename T, int R1, int R2, bool FIRST, bool KINV>
void launch_row2(fh_solver* s, int prec, int nload, T* X, const T* dC, Control* ctl, T* Wout, const T* Yaux) {
  using C = typename fh::cplx_t<T>::type;
  const GridInfo& g = s->g;
  const int bpl = s->row2_bpl[prec];
  fh::row_pass_2s<T, R1, R2, FIRST, KINV><<<(unsigned)(nload * bpl), fh::Row2<R1, R2>::THREADS,
                                             fh::row2_smem<T, R1, R2>(), s->work>>>(
      g, twp<T>(s->ax[g.nd - 1]), X, reinterpret_cast<C*>(s->S), s->phase, dC, ctl, s->st, s->partials, s->hist, bpl,
      Wout, Yaux);
}

// returns the blocks per load (the partial sums' layout)
template <typename T, bool FIRST, bool KINV>
int enqueue_row2(fh_solver* s, int prec, int nload, T* X, const T* dC, Control* ctl, T* Wout, const T* Yaux) {
  switch (s->row2[prec]) {
    case 32: launch_row2<T, 4, 8, FIRST, KINV>(s, prec, nload, X, dC, ctl, Wout, Yaux); break;
    case 64: launch_row2<T, 8, 8, FIRST, KINV>(s, prec, nload, X, dC, ctl, Wout, Yaux); break;
    default: launch_row2<T, 8, 16, FIRST, KINV>(s, prec, nload, X, dC, ctl, Wout, Yaux); break;
  }
  return s->row2_bpl[prec];
}

template <typename T, bool FIRST>
void enqueue_row_pass(fh_solver* s, int prec, int nload) {
  if (use_row2(s, prec) && !(sizeof(T) == 4 && use_plane(s, prec))) {
    enqueue_row2<T, FIRST, false>(s, prec, nload, Eptr<T>(s), dCptr<T>(s), s->ctl, nullptr, nullptr);
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (s->field) {   // point-by-point stiffness: the block row pass
      if (s->g.nv == 3) enqueue_row_pass_nv<T, 3, FIRST>(s, prec, nload);
      else enqueue_row_pass_nv<T, 6, FIRST>(s, prec, nload);
      return;
    }
    if (use_plane(s, prec)) {
      enqueue_plane<FIRST>(s, nload);
      return;
    }
    switch (s->row_warp[prec]) {
      case 1: enqueue_row_pass_warp<T, 1, FIRST>(s, prec, nload); return;
      case 2: enqueue_row_pass_warp<T, 2, FIRST>(s, prec, nload); return;
      case 4: enqueue_row_pass_warp<T, 4, FIRST>(s, prec, nload); return;
      case 8: enqueue_row_pass_warp<T, 8, FIRST>(s, prec, nload); return;
      default: break;
    }
  }
  if (s->g.nv == 3) enqueue_row_pass_nv<T, 3, FIRST>(s, prec, nload);
  else enqueue_row_pass_nv<T, 6, FIRST>(s, prec, nload);
}

template <typename T, int P>
cudaError_t set_warp_attrs(fh_solver* s, int prec, size_t rs) {
  cudaError_t e = cudaFuncSetAttribute(fh::row_pass_warp6<T, P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fh::row_pass_warp6<T, P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fh::row_pass_warp6<T, P, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s->warp_res[prec], fh::row_pass_warp6<T, P, false>,
                                                       fh::kWarpRowThreads, rs);
}

template <int P>
cudaError_t set_col_attrs() {
  const int sm = (int)fh::colpass_smem<P>();
  cudaError_t e = cudaFuncSetAttribute(fh::line_pass_warp6<P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fh::line_pass_warp6<P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fh::line_pass_warp6<P, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

template <typename T, int R1, int R2>
cudaError_t set_col2_attrs() {
  constexpr int CT = col2_ct<T>();
  const int sm = (int)fh::col2_smem<R1, R2, CT, T>();
  cudaError_t e = cudaFuncSetAttribute(fh::line_pass_2s<R1, R2, 0, CT, col2_mb<T, 0>(), T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fh::line_pass_2s<R1, R2, 1, CT, col2_mb<T, 1>(), T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fh::line_pass_2s<R1, R2, 2, CT, col2_mb<T, 2>(), T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

template <int P1, int P2>
cudaError_t set_plane_attrs() {
  const int sm = (int)fh::plane_smem<P1, P2>();
  cudaError_t e = cudaFuncSetAttribute(fh::plane_pass_warp6<P1, P2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fh::plane_pass_warp6<P1, P2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

cudaError_t set_plane_attrs_of(int code) {
  switch (code) {
    case 11: return set_plane_attrs<1, 1>();
    case 12: return set_plane_attrs<1, 2>();
    case 14: return set_plane_attrs<1, 4>();
    case 21: return set_plane_attrs<2, 1>();
    case 22: return set_plane_attrs<2, 2>();
    case 24: return set_plane_attrs<2, 4>();
    case 41: return set_plane_attrs<4, 1>();
    case 42: return set_plane_attrs<4, 2>();
    case 44: return set_plane_attrs<4, 4>();
    default: return cudaSuccess;
  }
}

template <typename T, int R1, int R2>
cudaError_t set_row2_attrs() {
  const int sm = (int)fh::row2_smem<T, R1, R2>();
  cudaError_t e = cudaFuncSetAttribute(fh::row_pass_2s<T, R1, R2, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fh::row_pass_2s<T, R1, R2, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fh::row_pass_2s<T, R1, R2, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

template <typename T, int NV>
fh_status set_smem_attrs_nv(fh_solver* s, int prec) {
  const size_t rs = s->row_smem[prec];
  if constexpr (NV == 6) {
    switch (s->row2[prec]) {
      case 32: CK((set_row2_attrs<T, 4, 8>())); break;
      case 64: CK((set_row2_attrs<T, 8, 8>())); break;
      case 128: CK((set_row2_attrs<T, 8, 16>())); break;
      default: break;
    }
  }
  if (sizeof(T) == 4 && s->plane[prec] > 0) CK(set_plane_attrs_of(s->plane[prec]));
  if (rs > kMaxSmem) {
    fh::set_error("contiguous axis too long for this precision (shared memory)");
    return FH_ERR_UNSUPPORTED;
  }
  if (s->field && s->row_smem_gen[prec] > kMaxSmem) {
    fh::set_error("contiguous axis too long for the point-by-point stiffness in this precision (shared memory)");
    return FH_ERR_UNSUPPORTED;
  }
  if (s->row_smem_gen[prec] <= kMaxSmem) {   // the block row pass (also taken by point-by-point stiffness)
    const int rg = (int)s->row_smem_gen[prec];
    CK(cudaFuncSetAttribute(fh::row_pass<T, NV, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rg));
    CK(cudaFuncSetAttribute(fh::row_pass<T, NV, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rg));
    CK(cudaFuncSetAttribute(fh::row_pass<T, NV, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rg));
  }
  if (s->row_warp[prec] != 0) {
    if constexpr (sizeof(T) == 4) {
    switch (s->row_warp[prec]) {
      case 1: CK((set_warp_attrs<T, 1>(s, prec, rs))); break;
      case 2: CK((set_warp_attrs<T, 2>(s, prec, rs))); break;
      case 4: CK((set_warp_attrs<T, 4>(s, prec, rs))); break;
      case 8: CK((set_warp_attrs<T, 8>(s, prec, rs))); break;
      default: break;
    }
    }
  }
  size_t lm = 0;
  for (int a = 0; a + 1 < s->g.nd; ++a) {
    switch (col2_len(s, prec, a)) {
      case 32: CK((set_col2_attrs<T, 4, 8>())); continue;
      case 64: CK((set_col2_attrs<T, 8, 8>())); continue;
      case 128: CK((set_col2_attrs<T, 8, 16>())); continue;
      default: break;
    }
    if constexpr (sizeof(T) == 4) {
      switch (col_warp_p(s, prec, a)) {
        case 1: CK((set_col_attrs<1>())); continue;
        case 2: CK((set_col_attrs<2>())); continue;
        case 4: CK((set_col_attrs<4>())); continue;
        case 8: CK((set_col_attrs<8>())); continue;
        default: break;
      }
    }
    lm = std::max(lm, s->line_smem[prec][a]);
  }
  if (lm > kMaxSmem) {
    fh::set_error("axis too long for this precision (shared memory)");
    return FH_ERR_UNSUPPORTED;
  }
  if (lm > 0) {
    CK(cudaFuncSetAttribute(fh::line_pass<T, NV, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lm));
    CK(cudaFuncSetAttribute(fh::line_pass<T, NV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lm));
    CK(cudaFuncSetAttribute(fh::line_pass<T, NV, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lm));
  }
  return FH_OK;
}

template <typename T>
fh_status set_smem_attrs(fh_solver* s, int prec) {
  return s->g.nv == 3 ? set_smem_attrs_nv<T, 3>(s, prec) : set_smem_attrs_nv<T, 6>(s, prec);
}

template <typename T>
fh_status get_graph(fh_solver* s, int prec, int nload, int chunk, cudaGraphExec_t* out) {
  const int variant = s->plane_on ? 2 : 0;   // graphs with and without the plane pass differ
  for (auto& e : s->graphs)
    if (e.prec == prec && e.nload == nload && e.chunk == chunk && e.method == variant) {
      *out = e.exec;
      return FH_OK;
    }
  CK(cudaStreamBeginCapture(s->work, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < chunk; ++i) {
    enqueue_line_passes<T>(s, prec, nload);
    enqueue_row_pass<T, false>(s, prec, nload);
  }
  cudaGraph_t graph;
  CK(cudaStreamEndCapture(s->work, &graph));
  cudaGraphExec_t exec;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    fh::set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return FH_ERR_CUDA;
  }
  s->graphs.push_back({prec, nload, chunk, variant, exec});
  *out = exec;
  return FH_OK;
}

int line_launches_per_iter(const GridInfo& g) { return g.nd == 1 ? 1 : 1 + 2 * (g.nd - 2); }
int line_launches_per_iter(const fh_solver* s, int prec) { return use_plane(s, prec) ? 1 : line_launches_per_iter(s->g); }

template <typename T>
fh_status run_solve(fh_solver* s, int prec, int nload, int chunk, int max_iter, long long* launches) {
  fh_status rc = set_smem_attrs<T>(s, prec);
  if (rc != FH_OK) return rc;
  cudaGraphExec_t exec;
  rc = get_graph<T>(s, prec, nload, chunk, &exec);
  if (rc != FH_OK) return rc;
  CK(cudaEventRecord(s->ev0, s->work));
  enqueue_row_pass<T, true>(s, prec, nload);
  CK(cudaGetLastError());
  long long launched = 0, extra = 0;
  bool finished = false;
  if (s->polish && prec == FH_PREC_FP64 && use_row2(s, prec) && !s->plane_on) {
    // The FP64 phase of a mixed solve usually stops after its first
    // iteration: that iteration's row pass ends after the E update and the
    // residual (the two-step row pass skips tau and the forward transform).
    // If a load goes on, a FIRST pass rebuilds the spectra from E (the same
    // values the full pass would have written) before the graph replays.
    enqueue_line_passes<T>(s, prec, nload);
    // bytes of 1: any nonzero value sets the flag
    CK(cudaMemsetAsync(&s->ctl->no_forward, 1, sizeof(int), s->work));
    enqueue_row_pass<T, false>(s, prec, nload);
    CK(cudaMemsetAsync(&s->ctl->no_forward, 0, sizeof(int), s->work));
    CK(cudaGetLastError());
    launched = 1;
    CK(cudaMemcpyAsync(s->h_flag, &s->ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, s->work));
    CK(cudaStreamSynchronize(s->work));
    finished = *s->h_flag != 0;
    if (!finished) {
      enqueue_row_pass<T, true>(s, prec, nload);
      CK(cudaGetLastError());
      extra = 1;
    }
  }
  while (!finished) {
    CK(cudaGraphLaunch(exec, s->work));
    launched += chunk;
    CK(cudaMemcpyAsync(s->h_flag, &s->ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, s->work));
    CK(cudaStreamSynchronize(s->work));
    if (*s->h_flag) break;
    if (launched > (long long)max_iter + chunk) {
      fh::set_error("iteration state did not terminate");
      return FH_ERR_INTERNAL;
    }
  }
  const int bpl = std::max(1, (int)std::min<long long>((s->g.m + kThreads - 1) / kThreads, kMeanBlocks));
  if (!s->skip_mean)
    fh::mean_stress<T><<<nload * bpl, kThreads, 0, s->work>>>(s->g, Eptr<T>(s), s->phase, s->Cp64, s->ctl, s->partials2,
                                                              s->mstress, bpl, s->field ? s->Cf64 : nullptr, s->nphase);
  CK(cudaGetLastError());
  CK(cudaEventRecord(s->ev1, s->work));
  *launches = (s->skip_mean ? 1 : 2) + extra + launched * (1 + line_launches_per_iter(s, prec));
  return FH_OK;
}

// ---------------------------------------------------------------------------
// BiCGStab on the pass path (see krylov.cuh)
// ---------------------------------------------------------------------------
constexpr int kKryBpl = 128;  // blocks per load of the vector kernels

template <typename T>
T* kry_field(fh_solver* s, int prec, int which) {
  return reinterpret_cast<T*>(s->kbuf[prec == FH_PREC_FP64 ? 0 : 1]) + (size_t)which * s->nload_max * s->g.nv * s->g.m;
}
enum { KR = 0, KRH = 1, KP = 2, KV = 3, KS = 4, KT = 5 };

template <typename T>
const T* dC_form0(const fh_solver* s);
template <>
const double* dC_form0<double>(const fh_solver* s) { return s->dC64; }
template <>
const float* dC_form0<float>(const fh_solver* s) { return s->dC32; }

// Row pass on an explicit field X with an explicit control block: FIRST (stress
// of X + ctl's eps0, forward transform) or KINV (Wout = X - inverse transform,
// block sums of Wout . Yaux and Wout . Wout).  Returns the blocks per load.
template <typename T, bool FIRST, bool KINV>
int enqueue_row_x(fh_solver* s, int prec, int nload, T* X, Control* ctl, T* Wout, const T* Yaux) {
  using C = typename fh::cplx_t<T>::type;
  const GridInfo& g = s->g;
  C* S = reinterpret_cast<C*>(s->S);
  const int last = g.nd - 1;
  if (use_row2(s, prec)) return enqueue_row2<T, FIRST, KINV>(s, prec, nload, X, dC_form0<T>(s), ctl, Wout, Yaux);
  if constexpr (sizeof(T) == 4) {
    const int P = s->field ? 0 : s->row_warp[prec];
    if (P > 0) {
      const int resident = std::max(1, s->warp_res[prec]) * std::max(1, s->sms);
      const int bpl = std::max(1, std::min(s->row_bpl[prec], resident / nload));
      const unsigned blocks = nload * bpl;
      const size_t sm = s->row_smem[prec];
      const C* tw = twp<T>(s->ax[last]);
      switch (P) {
        case 1: fh::row_pass_warp6<T, 1, FIRST, KINV><<<blocks, fh::kWarpRowThreads, sm, s->work>>>(g, tw, X, S, s->phase, dC_form0<T>(s), ctl, s->st, s->partials, s->hist, bpl, Wout, Yaux); break;
        case 2: fh::row_pass_warp6<T, 2, FIRST, KINV><<<blocks, fh::kWarpRowThreads, sm, s->work>>>(g, tw, X, S, s->phase, dC_form0<T>(s), ctl, s->st, s->partials, s->hist, bpl, Wout, Yaux); break;
        case 4: fh::row_pass_warp6<T, 4, FIRST, KINV><<<blocks, fh::kWarpRowThreads, sm, s->work>>>(g, tw, X, S, s->phase, dC_form0<T>(s), ctl, s->st, s->partials, s->hist, bpl, Wout, Yaux); break;
        default: fh::row_pass_warp6<T, 8, FIRST, KINV><<<blocks, fh::kWarpRowThreads, sm, s->work>>>(g, tw, X, S, s->phase, dC_form0<T>(s), ctl, s->st, s->partials, s->hist, bpl, Wout, Yaux); break;
      }
      return bpl;
    }
  }
  const int bpl = s->row_bpl_gen[prec];
  const int blocks = nload * bpl;
  if (g.nv == 3)
    fh::row_pass<T, 3, FIRST, KINV><<<blocks, kThreads, s->row_smem_gen[prec], s->work>>>(
        g, s->ax[last].planp[prec], twp<T>(s->ax[last]), X, S, s->phase, dC_form0<T>(s), ctl, s->st, s->partials, s->hist,
        s->rpb_gen[prec], bpl, Wout, Yaux, field_ptr<T>(s, 0));
  else
    fh::row_pass<T, 6, FIRST, KINV><<<blocks, kThreads, s->row_smem_gen[prec], s->work>>>(
        g, s->ax[last].planp[prec], twp<T>(s->ax[last]), X, S, s->phase, dC_form0<T>(s), ctl, s->st, s->partials, s->hist,
        s->rpb_gen[prec], bpl, Wout, Yaux, field_ptr<T>(s, 0));
  return bpl;
}

// W = A X = X + Gamma^p (C - C0) X (the stress with ctl's eps0: zero for the
// operator, eps0 for the start), with the block sums of W . Yaux and W . W;
// returns the blocks per load of those sums
template <typename T>
int enqueue_apply(fh_solver* s, int prec, int nload, T* X, Control* ctl, T* W, const T* Yaux) {
  enqueue_row_x<T, true, false>(s, prec, nload, X, ctl, nullptr, nullptr);
  enqueue_line_passes<T>(s, prec, nload, false);
  return enqueue_row_x<T, false, true>(s, prec, nload, X, ctl, W, Yaux);
}

// one BiCGStab iteration of every load that has not stopped
template <typename T>
void enqueue_bicgstab_iteration(fh_solver* s, int prec, int nload) {
  const long long n = (long long)s->g.nv * s->g.m;
  T* x = Eptr<T>(s);
  T *r = kry_field<T>(s, prec, KR), *rh = kry_field<T>(s, prec, KRH), *p = kry_field<T>(s, prec, KP);
  T *v = kry_field<T>(s, prec, KV), *sv = kry_field<T>(s, prec, KS), *t = kry_field<T>(s, prec, KT);
  const unsigned vb = nload * kKryBpl;
  fh::kry_update_p<T><<<vb, fh::kKryThreads, 0, s->work>>>(p, r, v, s->ksc, s->st, n, kKryBpl);
  int bpl = enqueue_apply<T>(s, prec, nload, p, s->ctl0, v, rh);                       // v = A p
  fh::kry_scalars<1><<<1, fh::kKryThreads, 0, s->work>>>(s->ksc, s->st, s->ctl, s->hist, s->partials, 2, bpl);
  fh::kry_update_s<T><<<vb, fh::kKryThreads, 0, s->work>>>(sv, r, v, s->ksc, s->st, n, kKryBpl);
  bpl = enqueue_apply<T>(s, prec, nload, sv, s->ctl0, t, nullptr);                       // t = A s
  fh::kry_scalars<2><<<1, fh::kKryThreads, 0, s->work>>>(s->ksc, s->st, s->ctl, s->hist, s->partials, 2, bpl);
  fh::kry_update_xr<T><<<vb, fh::kKryThreads, 0, s->work>>>(x, r, p, sv, t, rh, s->ksc, s->st, s->ctl, s->g.m,
                                                            s->g.nv, kKryBpl, s->kpart);
  fh::kry_scalars<3><<<1, fh::kKryThreads, 0, s->work>>>(s->ksc, s->st, s->ctl, s->hist, s->kpart, 3, kKryBpl);
}

int kry_launches_per_iter(const GridInfo& g) { return 4 + 2 * (2 + line_launches_per_iter(g)) + 3; }

template <typename T>
fh_status run_bicgstab(fh_solver* s, int prec, int nload, int chunk, int max_iter, long long* launches) {
  fh_status rc = set_smem_attrs<T>(s, prec);
  if (rc != FH_OK) return rc;
  const int slot = prec == FH_PREC_FP64 ? 0 : 1;
  const size_t nfield = (size_t)s->nload_max * s->g.nv * s->g.m;
  if (!s->kbuf[slot]) CK(cudaMalloc(&s->kbuf[slot], 6 * nfield * sizeof(T)));
  if (!s->ksc) {
    CK(cudaMalloc(&s->ksc, FH_MAX_LOADS * sizeof(fh::KrylovScal)));
    CK(cudaMalloc(&s->kpart, (size_t)FH_MAX_LOADS * kKryBpl * 3 * sizeof(double)));
    CK(cudaMalloc(&s->ctl0, sizeof(Control)));
  }
  // control block of the operator applications: the solve's, with eps0 = 0
  CK(cudaMemcpyAsync(s->ctl0, s->ctl, sizeof(Control), cudaMemcpyDeviceToDevice, s->work));
  CK(cudaMemsetAsync(s->ctl0->eps0, 0, sizeof(s->ctl0->eps0), s->work));
  cudaGraphExec_t exec = nullptr;
  for (auto& e : s->graphs)
    if (e.prec == prec && e.nload == nload && e.chunk == chunk && e.method == 1) exec = e.exec;
  if (!exec) {
    CK(cudaStreamBeginCapture(s->work, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) enqueue_bicgstab_iteration<T>(s, prec, nload);
    cudaGraph_t graph;
    CK(cudaStreamEndCapture(s->work, &graph));
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      fh::set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      return FH_ERR_CUDA;
    }
    s->graphs.push_back({prec, nload, chunk, 1, exec});
  }
  CK(cudaEventRecord(s->ev0, s->work));
  // start: r = b - A E0 (the stress of E0 + eps0 through the passes), rhat = r
  T* x = Eptr<T>(s);
  T* r = kry_field<T>(s, prec, KR);
  enqueue_apply<T>(s, prec, nload, x, s->ctl, r, nullptr);
  fh::kry_init<T><<<nload * kKryBpl, fh::kKryThreads, 0, s->work>>>(r, kry_field<T>(s, prec, KRH), x, s->st, s->ctl,
                                                                     s->g.m, s->g.nv, kKryBpl, s->kpart);
  fh::kry_scalars<0><<<1, fh::kKryThreads, 0, s->work>>>(s->ksc, s->st, s->ctl, s->hist, s->kpart, 3, kKryBpl);
  CK(cudaGetLastError());
  long long launched = 0;
  for (;;) {
    CK(cudaGraphLaunch(exec, s->work));
    launched += chunk;
    CK(cudaMemcpyAsync(s->h_flag, &s->ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, s->work));
    CK(cudaStreamSynchronize(s->work));
    if (*s->h_flag) break;
    if (launched > (long long)max_iter + chunk) {
      fh::set_error("iteration state did not terminate");
      return FH_ERR_INTERNAL;
    }
  }
  const int bpl = std::max(1, (int)std::min<long long>((s->g.m + kThreads - 1) / kThreads, kMeanBlocks));
  if (!s->skip_mean)
    fh::mean_stress<T><<<nload * bpl, kThreads, 0, s->work>>>(s->g, x, s->phase, s->Cp64, s->ctl, s->partials2,
                                                              s->mstress, bpl, s->field ? s->Cf64 : nullptr, s->nphase);
  CK(cudaGetLastError());
  CK(cudaEventRecord(s->ev1, s->work));
  *launches = (2 + line_launches_per_iter(s->g)) + 2 + (s->skip_mean ? 0 : 1) + launched * kry_launches_per_iter(s->g);
  return FH_OK;
}

// both axis plans use radices 2, 4, 8 only: the cluster kernel variant
// without the other stages (fewer registers, 16 warps per CTA)
bool pow2_plans(const fh_solver* s) {
  for (int a = 0; a < 2; ++a)
    for (int q = 0; q < s->ax[a].plan.np; ++q) {
      const int r = s->ax[a].plan.r[q];
      if (r != 2 && r != 4 && r != 8) return false;
    }
  return true;
}

// Cluster-resident path (2-axis grids): one cluster of CS CTAs per load case.
template <typename T, int NV, int CS, bool POW2>
fh_status cluster_fits_nv(fh_solver* s, bool* ok) {
  *ok = false;
  const GridInfo& g = s->g;
  if (g.nd != 2) return FH_OK;
  bool gs = true;
  fh::ClusterLayout lay = fh::cluster_layout<T>(g.dims[0], g.L, g.nv, CS, true);
  if (lay.total + 1024 > kMaxSmem) {
    gs = false;
    lay = fh::cluster_layout<T>(g.dims[0], g.L, g.nv, CS, false);
  }
  if (lay.total + 1024 > kMaxSmem) return FH_OK;
  s->cl_gsmem[sizeof(T) == 8 ? 0 : 1][CS == 16 ? 1 : 0] = gs;
  auto kern = fh::cluster_solve_2d<T, NV, CS, POW2>;
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
  if (CS > 8) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(fh::ClusterThreads<T, POW2>::value);
  cfg.dynamicSmemBytes = lay.total;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return FH_OK;
  }
  *ok = n >= 1;
  return FH_OK;
}

template <typename T, int CS>
fh_status cluster_fits(fh_solver* s, bool* ok) {
  if (pow2_plans(s))
    return s->g.nv == 3 ? cluster_fits_nv<T, 3, CS, true>(s, ok) : cluster_fits_nv<T, 6, CS, true>(s, ok);
  return s->g.nv == 3 ? cluster_fits_nv<T, 3, CS, false>(s, ok) : cluster_fits_nv<T, 6, CS, false>(s, ok);
}

// Task of the cluster kernel for load l of solver s.
template <typename T, int CS>
fh::ClusterTask cluster_task(const fh_solver* s, int l) {
  const bool gs = s->cl_gsmem[sizeof(T) == 8 ? 0 : 1][CS == 16 ? 1 : 0];
  fh::ClusterTask t{};
  t.g = s->g;
  t.plan0 = s->ax[0].plan;
  t.plan1 = s->ax[1].plan;
  t.tw0 = twp<T>(s->ax[0]);
  t.tw1 = twp<T>(s->ax[1]);
  t.E = Eptr<T>(const_cast<fh_solver*>(s));
  t.phase = s->phase;
  t.dC = dCptr<T>(const_cast<fh_solver*>(s));
  t.Gt = Gptr<T>(const_cast<fh_solver*>(s));
  t.ctl = s->ctl;
  t.st = s->st;
  t.hist = s->hist;
  t.nphase = s->nphase;
  t.g_smem = gs ? 1 : 0;
  t.load = l;
  return t;
}

// Launch configuration of the cluster kernel with `nclusters` clusters.
template <typename T, int NV, int CS, bool POW2>
cudaLaunchConfig_t cluster_config(size_t smem, int nclusters, cudaStream_t stream, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * CS);
  cfg.blockDim = dim3(fh::ClusterThreads<T, POW2>::value);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// A single solve: one cluster per load, each taking its own load's task.
template <typename T, int NV, int CS, bool POW2>
fh_status launch_cluster_nv(fh_solver* s, int nload) {
  const GridInfo& g = s->g;
  const bool gs = s->cl_gsmem[sizeof(T) == 8 ? 0 : 1][CS == 16 ? 1 : 0];
  const fh::ClusterLayout lay = fh::cluster_layout<T>(g.dims[0], g.L, g.nv, CS, gs);
  for (int l = 0; l < nload; ++l) s->h_tasks[l] = cluster_task<T, CS>(s, l);
  CK(cudaMemcpyAsync(s->qtasks, s->h_tasks, nload * sizeof(fh::ClusterTask), cudaMemcpyHostToDevice, s->work));
  CK(cudaMemsetAsync(s->qnext, 0, sizeof(unsigned int), s->work));
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<T, NV, CS, POW2>(lay.total, nload, s->work, attr);
  const fh::ClusterTask* tp = s->qtasks;
  unsigned int* np = s->qnext;
  CK(cudaLaunchKernelEx(&cfg, fh::cluster_solve_2d<T, NV, CS, POW2>, tp, nload, np));
  return FH_OK;
}

template <typename T, int CS>
fh_status launch_cluster(fh_solver* s, int nload) {
  if (pow2_plans(s))
    return s->g.nv == 3 ? launch_cluster_nv<T, 3, CS, true>(s, nload) : launch_cluster_nv<T, 6, CS, true>(s, nload);
  return s->g.nv == 3 ? launch_cluster_nv<T, 3, CS, false>(s, nload) : launch_cluster_nv<T, 6, CS, false>(s, nload);
}

// Pick path and cluster size; returns 1 (passes) or 2 (cluster) in *path.
template <typename T>
fh_status choose_path(fh_solver* s, int want_path, int want_cs, int* path, int* cs) {
  *path = 1;
  *cs = 0;
  s->plane_on = want_path == 3;
  if (s->field && want_path == 2) {
    fh::set_error("the cluster-resident path takes phase ids; a point-by-point stiffness runs on the passes");
    return FH_ERR_UNSUPPORTED;
  }
  if (want_path == 1 || want_path == 3 || s->field) return FH_OK;
  bool ok8 = false, ok16 = false;
  if (want_cs == 0 || want_cs == 16) {
    fh_status rc = cluster_fits<T, 16>(s, &ok16);
    if (rc != FH_OK) return rc;
  }
  if (want_cs == 0 || want_cs == 8) {
    fh_status rc = cluster_fits<T, 8>(s, &ok8);
    if (rc != FH_OK) return rc;
  }
  if (ok16 && (want_cs == 16 || want_cs == 0)) { *path = 2; *cs = 16; }
  else if (ok8) { *path = 2; *cs = 8; }
  if (want_path == 2 && *path != 2) {
    fh::set_error("cluster-resident path unavailable for this grid (needs 2 axes and fields that fit in a cluster)");
    return FH_ERR_UNSUPPORTED;
  }
  return FH_OK;
}

template <typename T>
fh_status run_solve_cluster(fh_solver* s, int nload, int cs, long long* launches) {
  CK(cudaEventRecord(s->ev0, s->work));
  fh_status rc = cs == 16 ? launch_cluster<T, 16>(s, nload) : launch_cluster<T, 8>(s, nload);
  if (rc != FH_OK) return rc;
  const int bpl = std::max(1, (int)std::min<long long>((s->g.m + kThreads - 1) / kThreads, kMeanBlocks));
  if (!s->skip_mean)
    fh::mean_stress<T><<<nload * bpl, kThreads, 0, s->work>>>(s->g, Eptr<T>(s), s->phase, s->Cp64, s->ctl, s->partials2,
                                                              s->mstress, bpl, s->field ? s->Cf64 : nullptr, s->nphase);
  CK(cudaGetLastError());
  CK(cudaEventRecord(s->ev1, s->work));
  *launches = s->skip_mean ? 1 : 2;
  return FH_OK;
}

void free_all(fh_solver* s) {
  for (auto& e : s->graphs) cudaGraphExecDestroy(e.exec);
  s->graphs.clear();
  void* ptrs[] = {s->E64, s->E32, s->S, s->phase, s->Cp64, s->dC64, s->dC32, s->Cp32, s->G64, s->G32, s->ctl, s->st,
                  s->partials, s->partials2, s->hist, s->mstress, s->err, s->scratch64, s->qtasks, s->qnext,
                  s->kbuf[0], s->kbuf[1], s->ksc, s->kpart, s->ctl0, s->Cf64, s->dCf64, s->dCf32, s->Cf32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& a : s->ax) {
    if (a.tw64) cudaFree(a.tw64);
    if (a.tw32) cudaFree(a.tw32);
  }
  if (s->h_flag) cudaFreeHost(s->h_flag);
  if (s->h_states) cudaFreeHost(s->h_states);
  if (s->h_ms) cudaFreeHost(s->h_ms);
  if (s->h_tasks) cudaFreeHost(s->h_tasks);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  if (s->ev_user) cudaEventDestroy(s->ev_user);
  if (s->work) cudaStreamDestroy(s->work);
}

// order the private work stream after everything already queued on the user stream
fh_status join_user(fh_solver* s) {
  CK(cudaEventRecord(s->ev_user, s->user));
  CK(cudaStreamWaitEvent(s->work, s->ev_user, 0));
  return FH_OK;
}

bool cholesky_ok(const double* A, int n) {
  double L[36] = {};
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) return false;
    L[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = v / L[j * n + j];
    }
  }
  return true;
}

// Mandel matrix -> fourth-order tensor C_ijkl (3x3x3x3 storage)
// The closed-form table kernel (green_table_iso) applies when C0 is isotropic
// (Mandel: lam0 + 2 mu0 on the normal diagonal, lam0 off it, 2 mu0 on the shear
// diagonal, zero elsewhere; compared to 1e-15 of its largest entry) and the
// symbol is a product of per-axis factors: Dirichlet, dlVP, or a box spline
// whose directions are all +-e_i.  Fills lam0, mu0 and the per-axis direction
// counts of GP.
bool closed_form_table(const fh_solver* s, const double* c0, fh::GreenParams* GP) {
  const int nv = s->g.nv, d = s->g.d;
  const double lam0 = c0[1], mu0 = 0.5 * c0[(nv - 1) * nv + nv - 1];
  double big = 0.0;
  for (int e = 0; e < nv * nv; ++e) big = std::max(big, std::fabs(c0[e]));
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      double want = 0.0;
      if (a < d && b < d) want = lam0 + (a == b ? 2.0 * mu0 : 0.0);
      else if (a == b) want = 2.0 * mu0;
      if (std::fabs(c0[a * nv + b] - want) > 1e-15 * big) return false;
    }
  if (!(mu0 > 0.0) || !(lam0 + 2.0 * mu0 > 0.0)) return false;
  for (int i = 0; i < 3; ++i) GP->xcount[i] = 0;
  if (s->gen.kind == FH_GEN_BOXSPLINE) {
    for (int q = 0; q < s->gen.n_xi; ++q) {
      int axis = -1, nonzero = 0;
      for (int i = 0; i < d; ++i) {
        const double v = s->gen.xi[3 * q + i];
        if (v != 0.0) { ++nonzero; axis = i; }
        if (v != 0.0 && std::fabs(v) != 1.0) return false;
      }
      if (nonzero != 1) return false;
      GP->xcount[axis] += 1;
    }
  }
  GP->lam0 = lam0;
  GP->mu0 = mu0;
  return true;
}

// Mirror symmetry of the table (green_table_iso): M diagonal and every Smith
// axis one of M's axes (each row of Fmap a single +-1), all d axes non-trivial.
// geo[k] receives the geometric axis of the full storage axes k = 0 .. d-2.
bool mirror_axes(const fh_solver* s, int* geo) {
  const int d = s->g.d;
  if (s->g.nd != d) return false;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && s->P.M[i][j] != 0) return false;
  for (int k = 0; k < d; ++k) {
    int axis = -1, nonzero = 0;
    for (int i = 0; i < d; ++i) {
      const long long v = s->P.Fmap[k][i];
      if (v != 0) { ++nonzero; axis = i; }
      if (v != 0 && v != 1 && v != -1) return false;
    }
    if (nonzero != 1) return false;
    if (k < d - 1) geo[k] = axis;
  }
  return true;
}

// A 6 x 6 Mandel matrix whose normal-shear blocks are zero and whose shear
// block is diagonal (isotropic, cubic or orthotropic in the grid axes)
bool decoupled6(const double* c) {
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      const bool structural_zero = ((a < 3) != (b < 3)) || (a >= 3 && b >= 3 && a != b);
      if (structural_zero && c[a * 6 + b] != 0.0) return false;
    }
  return true;
}

// Cubic symmetry of the table (green_table_iso<3>): on top of the mirror
// conditions, three storage axes of one length, |M_00| = |M_11| = |M_22|, and
// the same per-axis symbol on every axis (Dirichlet; dlVP with equal ramps; a
// box spline with the same count of each direction).  Then permuting the
// geometric axes maps the alias set and its weights onto themselves.
bool cubic_axes(const fh_solver* s, const fh::GreenParams& GP) {
  if (s->g.d != 3 || s->g.nd != 3) return false;
  if (s->g.dims[0] != s->g.dims[1] || s->g.dims[1] != s->g.dims[2]) return false;
  const long long a0 = std::llabs(s->P.M[0][0]);
  if (std::llabs(s->P.M[1][1]) != a0 || std::llabs(s->P.M[2][2]) != a0) return false;
  if (s->gen.kind == FH_GEN_DLVP)
    return s->gen.alpha[0] == s->gen.alpha[1] && s->gen.alpha[1] == s->gen.alpha[2];
  if (s->gen.kind == FH_GEN_BOXSPLINE) return GP.xcount[0] == GP.xcount[1] && GP.xcount[1] == GP.xcount[2];
  return true;
}

void mandel_to_c4(const double* Cm, int d, double* C4) {
  const int I2[3] = {0, 1, 0}, J2[3] = {0, 1, 1};
  const int I3[6] = {0, 1, 2, 1, 0, 0}, J3[6] = {0, 1, 2, 2, 2, 1};
  const int* I = d == 2 ? I2 : I3;
  const int* J = d == 2 ? J2 : J3;
  const int nv = mandel_nv(d);
  for (int q = 0; q < 81; ++q) C4[q] = 0.0;
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      const double sa = I[a] == J[a] ? 1.0 : std::sqrt(2.0);
      const double sb = I[b] == J[b] ? 1.0 : std::sqrt(2.0);
      const double v = Cm[a * nv + b] / (sa * sb);
      const int ij[2][2] = {{I[a], J[a]}, {J[a], I[a]}};
      const int kl[2][2] = {{I[b], J[b]}, {J[b], I[b]}};
      for (auto& p : ij)
        for (auto& q : kl) C4[((p[0] * 3 + p[1]) * 3 + q[0]) * 3 + q[1]] = v;
    }
}

}  // namespace

namespace {
template <typename T>
fh_status profile_passes(fh_solver* s, int prec, int nload, int reps, double* ms) {
  fh_status rc = set_smem_attrs<T>(s, prec);
  if (rc != FH_OK) return rc;
  // every load active, no stopping: tol 0 and a max_iter beyond any count
  int big = 0x7fffffff;
  double zero = 0.0;
  CK(cudaMemsetAsync(s->st, 0, FH_MAX_LOADS * sizeof(LoadState), s->work));
  CK(cudaMemcpyAsync(&s->ctl->tol, &zero, sizeof(double), cudaMemcpyHostToDevice, s->work));
  CK(cudaMemcpyAsync(&s->ctl->max_iter, &big, sizeof(int), cudaMemcpyHostToDevice, s->work));
  CK(cudaMemcpyAsync(&s->ctl->nload, &nload, sizeof(int), cudaMemcpyHostToDevice, s->work));
  const int no_stall = 0;
  CK(cudaMemcpyAsync(&s->ctl->stall_window, &no_stall, sizeof(int), cudaMemcpyHostToDevice, s->work));
  const GridInfo& g = s->g;
  using C = typename fh::cplx_t<T>::type;
  C* S = reinterpret_cast<C*>(s->S);
  for (int q = 0; q < 4; ++q) ms[q] = 0.0;
  auto timed = [&](int q, auto&& launch) -> fh_status {
    launch();
    CK(cudaGetLastError());
    CK(cudaEventRecord(s->ev0, s->work));
    for (int i = 0; i < reps; ++i) launch();
    CK(cudaEventRecord(s->ev1, s->work));
    CK(cudaEventSynchronize(s->ev1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, s->ev0, s->ev1));
    ms[q] = (double)t / reps;
    return FH_OK;
  };
  rc = timed(0, [&] { enqueue_row_pass<T, false>(s, prec, nload); });
  if (rc != FH_OK) return rc;
  auto line = [&](int a, int mode) { launch_axis<T>(s, prec, a, mode, nload); };
  if (g.nd == 1) {
    rc = timed(1, [&] {
      const long long total = (long long)nload * g.nhalf;
      const int blocks = (int)std::min<long long>((total + kThreads - 1) / kThreads, 4096);
      fh::green_1d<T><<<blocks, kThreads, 0, s->work>>>(g, S, Gptr<T>(s), s->st, nload);
    });
    if (rc != FH_OK) return rc;
  } else {
    rc = timed(1, [&] { line(0, 2); });
    if (rc != FH_OK) return rc;
    if (g.nd == 3 && !use_plane(s, prec)) {
      rc = timed(2, [&] { line(1, 0); });
      if (rc != FH_OK) return rc;
      rc = timed(3, [&] { line(1, 1); });
      if (rc != FH_OK) return rc;
    }
  }
  CK(cudaStreamSynchronize(s->work));
  return FH_OK;
}
}  // namespace

namespace {

const char* check_site_name(int site) {
  static const char* names[fh::CK_NSITES] = {
      "?", "row pass: half spectrum", "row pass: strain", "row pass: phase", "row pass: work buffer",
      "row pass: stiffness field", "partial sums", "line pass: half spectrum", "line pass: table",
      "line pass: line buffer", "warp row pass: half spectrum", "warp row pass: strain", "warp row pass: phase",
      "warp row pass: scratch", "warp column pass: half spectrum", "warp column pass: table",
      "warp column pass: tile", "two-step column pass: half spectrum", "two-step column pass: table",
      "two-step column pass: tile", "1-D Green step", "mean stress", "Krylov vectors", "cluster solve",
      "Green table", "self test"};
  return (site > 0 && site < fh::CK_NSITES) ? names[site] : "?";
}

// Checked build: after an entry point's work, the record of the first index
// found outside its array turns the call's status into FH_ERR_INTERNAL (the
// record is cleared).  Without FH_CHECKED the status passes through.
fh_status checked(fh_status rc) {
#ifdef FH_CHECKED
  CK(cudaDeviceSynchronize());
  fh::CheckRecord rec{};
  CK(cudaMemcpyFromSymbol(&rec, fh::g_check, sizeof(rec)));
  if (rec.count != 0ull) {
    const fh::CheckRecord zero{};
    CK(cudaMemcpyToSymbol(fh::g_check, &zero, sizeof(zero)));
    fh::set_error(std::string("index check failed (") + std::to_string(rec.count) + " accesses): " +
                  check_site_name(rec.site) + ", index " + std::to_string(rec.index) + " outside [0, " +
                  std::to_string(rec.extent) + ")");
    return FH_ERR_INTERNAL;
  }
#endif
  return rc;
}

#ifdef FH_CHECKED
// one index inside and one outside a declared extent of 4 (the buffer holds
// 64 entries, so even a failed check would stay inside it)
__global__ void check_selftest_kernel(int* buf) {
  for (int i = 3; i <= 5; i += 2)
    if (FH_IN(fh::CK_SELFTEST, i, 4)) buf[i] = 1;
}
#endif

}  // namespace

extern "C" {

int fh_checked_build(void) {
#ifdef FH_CHECKED
  return 1;
#else
  return 0;
#endif
}

fh_status fh_check_selftest(void) {
#ifdef FH_CHECKED
  fh_status rc = checked(FH_OK);   // start from a clear record
  if (rc != FH_OK) return rc;
  int* buf = nullptr;
  CK(cudaMalloc(&buf, 64 * sizeof(int)));
  check_selftest_kernel<<<1, 1>>>(buf);
  cudaError_t e = cudaGetLastError();
  rc = checked(FH_OK);
  cudaFree(buf);
  if (e != cudaSuccess) {
    fh::set_error(std::string("self test launch: ") + cudaGetErrorString(e));
    return FH_ERR_CUDA;
  }
  return rc;
#else
  fh::set_error("not a checked build (compile with FH_CHECKED)");
  return FH_ERR_UNSUPPORTED;
#endif
}

const char* fh_status_string(fh_status st) {
  switch (st) {
    case FH_OK: return "ok";
    case FH_NOT_CONVERGED: return "not converged (max_iter reached)";
    case FH_DIVERGED: return "diverged";
    case FH_NONFINITE: return "non-finite residual";
    case FH_ERR_ARG: return "invalid argument";
    case FH_ERR_SINGULAR_M: return "singular pattern matrix";
    case FH_ERR_OVERFLOW: return "integer overflow";
    case FH_ERR_NO_ONB: return "translates cannot be orthonormalised";
    case FH_ERR_CUDA: return "CUDA error";
    case FH_ERR_TIMEOUT: return "device wait timed out";
    case FH_ERR_INTERNAL: return "internal error";
    case FH_ERR_UNSUPPORTED: return "unsupported size";
    case FH_ERR_STATE: return "call order violated";
  }
  return "unknown status";
}

const char* fh_last_error(void) { return fh::g_err.c_str(); }

fh_status fh_pattern_create(int d, const int64_t* M, fh_pattern** out) {
  if (!M || !out) { fh::set_error("null argument"); return FH_ERR_ARG; }
  fh_pattern* p = new fh_pattern();
  fh_status rc = fh::build_pattern(d, M, &p->p);
  if (rc != FH_OK) { delete p; return rc; }
  *out = p;
  return FH_OK;
}

void fh_pattern_destroy(fh_pattern* p) { delete p; }

fh_status fh_pattern_info(const fh_pattern* p, int64_t* m, int* ndims, int* dims) {
  if (!p) { fh::set_error("null pattern"); return FH_ERR_ARG; }
  if (m) *m = p->p.D;
  if (ndims) *ndims = p->p.nd;
  if (dims)
    for (int k = 0; k < 3; ++k) dims[k] = k < p->p.nd ? p->p.dims[k] : 1;
  return FH_OK;
}

fh_status fh_pattern_numerators(const fh_pattern* p, int64_t* a) {
  if (!p || !a) { fh::set_error("null argument"); return FH_ERR_ARG; }
  const int d = p->p.d;
  for (int64_t i = 0; i < p->p.D; ++i) p->p.point_numerator(i, a + i * d);
  return FH_OK;
}

fh_status fh_pattern_points(const fh_pattern* p, double* y) {
  if (!p || !y) { fh::set_error("null argument"); return FH_ERR_ARG; }
  const int d = p->p.d;
  int64_t a[3];
  for (int64_t i = 0; i < p->p.D; ++i) {
    p->p.point_numerator(i, a);
    for (int k = 0; k < d; ++k) y[i * d + k] = (double)a[k] / (double)p->p.D;
  }
  return FH_OK;
}

fh_status fh_pattern_half_freqs(const fh_pattern* p, int64_t* h, int64_t* nh) {
  if (!p) { fh::set_error("null pattern"); return FH_ERR_ARG; }
  const int64_t n = p->p.n_half();
  if (nh) *nh = n;
  if (!h) return FH_OK;
  for (int64_t f = 0; f < n; ++f) p->p.half_freq(f, h + f * p->p.d);
  return FH_OK;
}

fh_status fh_solver_create(const fh_pattern* p, const fh_generator* gen, int nload_max, void* stream,
                           fh_solver** out) {
  if (!p || !gen || !out) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (nload_max < 1 || nload_max > FH_MAX_LOADS) { fh::set_error("nload_max out of range"); return FH_ERR_ARG; }
  if (gen->kind < FH_GEN_DIRICHLET || gen->kind > FH_GEN_BOXSPLINE) { fh::set_error("unknown generator"); return FH_ERR_ARG; }
  const int d = p->p.d;
  if (p->p.D < 2) {
    fh::set_error("single-point pattern (|det M| = 1): E = 0 and C_eff = C(0), nothing to iterate");
    return FH_ERR_UNSUPPORTED;
  }
  if (gen->kind == FH_GEN_DLVP)
    for (int i = 0; i < d; ++i)
      if (!(gen->alpha[i] >= 0.0 && gen->alpha[i] <= 0.5)) { fh::set_error("dlVP alpha outside [0, 1/2]"); return FH_ERR_ARG; }
  if (gen->kind == FH_GEN_BOXSPLINE) {
    if (gen->n_xi < 1 || gen->n_xi > FH_MAX_XI) { fh::set_error("box spline n_xi out of range"); return FH_ERR_ARG; }
    if (gen->alias_radius < 0 || gen->alias_radius > 16) { fh::set_error("alias radius out of range"); return FH_ERR_ARG; }
  }
  fh_solver* s = new fh_solver();
  s->P = p->p;
  s->gen = *gen;
  s->user = reinterpret_cast<cudaStream_t>(stream);
  s->nload_max = nload_max;
  GridInfo& g = s->g;
  g.d = d;
  g.nv = mandel_nv(d);
  g.ntri = g.nv * (g.nv + 1) / 2;
  g.nd = s->P.nd;
  for (int k = 0; k < 3; ++k) g.dims[k] = k < g.nd ? s->P.dims[k] : 1;
  g.L = g.dims[g.nd - 1];
  g.H = g.L / 2 + 1;
  g.m = s->P.D;
  g.nrows = g.m / g.L;
  g.nhalf = s->P.n_half();
  g.inv_m = 1.0 / (double)g.m;
  for (int k = 0; k < g.nd; ++k) {
    if (g.dims[k] > 4096) { delete s; fh::set_error("SNF axis longer than 4096"); return FH_ERR_UNSUPPORTED; }
    fh::FftPlan fp;
    if (!fh::make_plan(g.dims[k], &fp)) { delete s; fh::set_error("SNF axis length needs more than 24 radix stages"); return FH_ERR_UNSUPPORTED; }
    s->ax[k].L = fp.L;
    s->ax[k].plan.L = fp.L;
    s->ax[k].plan.np = fp.np;
    for (int q = 0; q < 24; ++q) s->ax[k].plan.r[q] = fp.r[q];
    s->ax[k].planp[0] = s->ax[k].planp[1] = s->ax[k].plan;
  }
  choose_shapes(s, FH_PREC_FP64);
  choose_shapes(s, FH_PREC_FP32);
  save_default_shapes(s);
  auto fail = [&](fh_status rc) { free_all(s); delete s; return rc; };
#define CKS(call)                                                             \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      fh::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));      \
      return fail(FH_ERR_CUDA);                                               \
    }                                                                         \
  } while (0)
  CKS(cudaStreamCreateWithFlags(&s->work, cudaStreamNonBlocking));
  {
    int dev = 0;
    CKS(cudaGetDevice(&dev));
    CKS(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev));
  }
  CKS(cudaEventCreate(&s->ev0));
  CKS(cudaEventCreate(&s->ev1));
  CKS(cudaEventCreateWithFlags(&s->ev_user, cudaEventDisableTiming));
  const size_t nfield = (size_t)nload_max * g.nv * g.m;
  const size_t nspec = (size_t)nload_max * g.nv * g.nhalf;
  CKS(cudaMalloc(&s->E64, nfield * sizeof(double)));
  CKS(cudaMalloc(&s->E32, nfield * sizeof(float)));
  CKS(cudaMalloc(&s->S, nspec * sizeof(double2)));
  CKS(cudaMalloc(&s->phase, (size_t)g.m));
  CKS(cudaMalloc(&s->Cp64, kMaxPhases * 36 * sizeof(double)));
  CKS(cudaMalloc(&s->dC64, kMaxPhases * 36 * sizeof(double)));
  CKS(cudaMalloc(&s->dC32, kMaxPhases * 36 * sizeof(float)));
  CKS(cudaMalloc(&s->Cp32, kMaxPhases * 36 * sizeof(float)));
  CKS(cudaMalloc(&s->G64, (size_t)g.ntri * g.nhalf * sizeof(double)));
  CKS(cudaMalloc(&s->G32, (size_t)g.ntri * g.nhalf * sizeof(float)));
  CKS(cudaMalloc(&s->ctl, sizeof(Control)));
  CKS(cudaMalloc(&s->st, FH_MAX_LOADS * sizeof(LoadState)));
  const size_t nblk = (size_t)nload_max * std::max({s->row_bpl[0], s->row_bpl[1], s->row_bpl_gen[0], s->row_bpl_gen[1],
                                                    s->row2_bpl[0], s->row2_bpl[1],
                                                    2 * g.dims[0]});
  CKS(cudaMalloc(&s->partials, 2 * nblk * sizeof(double)));
  CKS(cudaMalloc(&s->partials2, (size_t)nload_max * kMeanBlocks * fh::MAXV * sizeof(double)));
  CKS(cudaMalloc(&s->hist, (size_t)nload_max * kHistCap * sizeof(double)));
  CKS(cudaMalloc(&s->mstress, FH_MAX_LOADS * fh::MAXV * sizeof(double)));
  CKS(cudaMalloc(&s->err, sizeof(int)));
  CKS(cudaMallocHost(&s->h_flag, sizeof(int)));
  CKS(cudaMallocHost(&s->h_states, FH_MAX_LOADS * sizeof(LoadState)));
  CKS(cudaMallocHost(&s->h_ms, FH_MAX_LOADS * fh::MAXV * sizeof(double)));
  CKS(cudaMalloc(&s->qtasks, FH_MAX_LOADS * sizeof(fh::ClusterTask)));
  CKS(cudaMalloc(&s->qnext, sizeof(unsigned int)));
  CKS(cudaMallocHost(&s->h_tasks, FH_MAX_LOADS * sizeof(fh::ClusterTask)));
  CKS(cudaMemset(s->ctl, 0, sizeof(Control)));
  CKS(cudaMemset(s->st, 0, FH_MAX_LOADS * sizeof(LoadState)));
  CKS(cudaMemset(s->err, 0, sizeof(int)));
  CKS(cudaMemset(s->E64, 0, nfield * sizeof(double)));
  // twiddles exp(-2 pi i t / L), evaluated in long double on the host
  for (int k = 0; k < g.nd; ++k) {
    const int L = s->ax[k].L;
    std::vector<double2> t64(L);
    std::vector<float2> t32(L);
    for (int t = 0; t < L; ++t) {
      const long double ang = 2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)L;
      t64[t].x = (double)cosl(ang);
      t64[t].y = (double)(-sinl(ang));
      t32[t].x = (float)t64[t].x;
      t32[t].y = (float)t64[t].y;
    }
    CKS(cudaMalloc(&s->ax[k].tw64, L * sizeof(double2)));
    CKS(cudaMalloc(&s->ax[k].tw32, L * sizeof(float2)));
    CKS(cudaMemcpy(s->ax[k].tw64, t64.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
    CKS(cudaMemcpy(s->ax[k].tw32, t32.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
  }
#undef CKS
  *out = s;
  return FH_OK;
}

void fh_solver_destroy(fh_solver* s) {
  if (!s) return;
  if (s->work) cudaStreamSynchronize(s->work);
  free_all(s);
  delete s;
}

fh_status fh_set_stiffness_phases(fh_solver* s, const uint8_t* phase, int nphase, const double* Cp) {
  if (!s || !phase || !Cp) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (nphase < 1 || nphase > kMaxPhases) { fh::set_error("nphase must be 1..16"); return FH_ERR_ARG; }
  const int nv = s->g.nv;
  for (int q = 0; q < nphase; ++q)
    for (int a = 0; a < nv; ++a)
      for (int b = 0; b < nv; ++b) {
        const double v = Cp[(q * nv + a) * nv + b];
        if (!std::isfinite(v)) { fh::set_error("non-finite stiffness"); return FH_ERR_ARG; }
        if (std::fabs(v - Cp[(q * nv + b) * nv + a]) > 1e-12 * (1.0 + std::fabs(v))) {
          fh::set_error("phase stiffness is not symmetric (major symmetry)");
          return FH_ERR_ARG;
        }
      }
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  CK(cudaMemcpyAsync(s->phase, phase, (size_t)s->g.m, cudaMemcpyDefault, s->work));
  CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->work));
  fh::check_phases<<<256, kThreads, 0, s->work>>>(s->phase, s->g.m, nphase, s->err);
  CK(cudaGetLastError());
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->work));
  CK(cudaStreamSynchronize(s->work));
  if (herr != 0) { fh::set_error("phase id >= nphase"); return FH_ERR_ARG; }
  s->field = false;
  s->nphase = nphase;
  std::memcpy(s->Cp, Cp, sizeof(double) * nphase * nv * nv);
  CK(cudaMemcpy(s->Cp64, s->Cp, sizeof(double) * nphase * nv * nv, cudaMemcpyHostToDevice));
  float cpf[kMaxPhases * 36];
  for (int q = 0; q < nphase * nv * nv; ++q) cpf[q] = (float)s->Cp[q];
  CK(cudaMemcpy(s->Cp32, cpf, sizeof(float) * nphase * nv * nv, cudaMemcpyHostToDevice));
  s->have_phases = true;
  s->have_table = false;
  return FH_OK;
}

}  // extern "C"

namespace {

// More than 16 distinct matrices: keep C(x) itself, upper triangle [tri][m] in
// FP64 on the device (the differences C(x) - C0 follow in fh_set_reference),
// after checking every matrix on the host.  Also records the ranges of lambda
// = C_1122 and mu = C_shear,shear / 2 over the points for the reference-medium
// rule.
fh_status set_field_pointwise(fh_solver* s, const double* Ch) {
  const int nv = s->g.nv, ntri = s->g.ntri;
  const size_t m = (size_t)s->g.m, per = (size_t)nv * nv;
  std::vector<double> tri((size_t)ntri * m);
  double lmin = 1e300, lmax = -1e300, mmin = 1e300, mmax = -1e300;
  for (size_t i = 0; i < m; ++i) {
    const double* c = Ch + i * per;
    int t = 0;
    for (int a = 0; a < nv; ++a)
      for (int b = a; b < nv; ++b, ++t) {
        const double v = c[a * nv + b];
        if (!std::isfinite(v)) { fh::set_error("non-finite stiffness"); return FH_ERR_ARG; }
        if (std::fabs(v - c[b * nv + a]) > 1e-12 * (1.0 + std::fabs(v))) {
          fh::set_error("stiffness is not symmetric (major symmetry)");
          return FH_ERR_ARG;
        }
        tri[(size_t)t * m + i] = v;
      }
    const double lam = c[1], mu = 0.5 * c[(nv - 1) * nv + nv - 1];
    lmin = std::min(lmin, lam); lmax = std::max(lmax, lam);
    mmin = std::min(mmin, mu); mmax = std::max(mmax, mu);
  }
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  const size_t n = (size_t)ntri * m;
  if (!s->Cf64) {
    CK(cudaMalloc(&s->Cf64, n * sizeof(double)));
    CK(cudaMalloc(&s->dCf64, n * sizeof(double)));
    CK(cudaMalloc(&s->dCf32, n * sizeof(float)));
    CK(cudaMalloc(&s->Cf32, n * sizeof(float)));
  }
  CK(cudaMemcpyAsync(s->Cf64, tri.data(), n * sizeof(double), cudaMemcpyHostToDevice, s->work));
  CK(cudaMemsetAsync(s->phase, 0, m, s->work));
  CK(cudaStreamSynchronize(s->work));
  // the phase table holds the first point's matrix (read by nothing on this path)
  s->nphase = 1;
  std::memcpy(s->Cp, Ch, sizeof(double) * per);
  CK(cudaMemcpy(s->Cp64, s->Cp, sizeof(double) * per, cudaMemcpyHostToDevice));
  s->field_lam[0] = lmin; s->field_lam[1] = lmax;
  s->field_mu[0] = mmin; s->field_mu[1] = mmax;
  s->field = true;
  s->have_phases = true;
  s->have_table = false;
  return FH_OK;
}

}  // namespace

extern "C" {

fh_status fh_set_stiffness_field(fh_solver* s, const double* C) {
  if (!s || !C) { fh::set_error("null argument"); return FH_ERR_ARG; }
  const int nv = s->g.nv;
  const size_t per = (size_t)nv * nv;
  const size_t m = (size_t)s->g.m;
  // the field on the host (it may live in device memory)
  std::vector<double> host;
  const double* Ch = C;
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, C) == cudaSuccess && attr.type == cudaMemoryTypeDevice) {
    host.resize(m * per);
    CK(cudaMemcpy(host.data(), C, m * per * sizeof(double), cudaMemcpyDeviceToHost));
    Ch = host.data();
  }
  cudaGetLastError();   // a host pointer may leave an error behind on some drivers
  std::vector<uint8_t> ids(m);
  double table[kMaxPhases * 36];
  int nphase = 0;
  for (size_t i = 0; i < m; ++i) {
    const double* c = Ch + i * per;
    int q = 0;
    while (q < nphase && std::memcmp(table + q * per, c, per * sizeof(double)) != 0) ++q;
    if (q == nphase) {
      if (nphase == kMaxPhases) return set_field_pointwise(s, Ch);
      std::memcpy(table + q * per, c, per * sizeof(double));
      ++nphase;
    }
    ids[i] = (uint8_t)q;
  }
  return fh_set_stiffness_phases(s, ids.data(), nphase, table);
}

static fh_status fh_set_reference_impl(fh_solver* s, const double* C0) {
  NvtxRange range("fh_set_reference (Gamma^p table)");
  if (!s) { fh::set_error("null solver"); return FH_ERR_ARG; }
  if (!s->have_phases) { fh::set_error("set the stiffness before the reference medium"); return FH_ERR_STATE; }
  const int nv = s->g.nv, d = s->g.d;
  double c0[36] = {};
  if (C0) {
    std::memcpy(c0, C0, sizeof(double) * nv * nv);
  } else {
    // Moulinec-Suquet rule on isotropic phases: lambda = C_1122, 2 mu = C_shear,shear (Mandel)
    double lmin = 1e300, lmax = -1e300, mmin = 1e300, mmax = -1e300;
    for (int q = 0; q < s->nphase; ++q) {
      const double* C = s->Cp + q * nv * nv;
      const double lam = C[0 * nv + 1];
      const double mu = 0.5 * C[(nv - 1) * nv + (nv - 1)];
      lmin = std::min(lmin, lam); lmax = std::max(lmax, lam);
      mmin = std::min(mmin, mu); mmax = std::max(mmax, mu);
    }
    if (s->field) {
      lmin = s->field_lam[0]; lmax = s->field_lam[1];
      mmin = s->field_mu[0]; mmax = s->field_mu[1];
    }
    const double lam0 = 0.5 * (lmin + lmax), mu0 = 0.5 * (mmin + mmax);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) c0[a * nv + b] = lam0 + (a == b ? 2.0 * mu0 : 0.0);
    for (int a = d; a < nv; ++a) c0[a * nv + a] = 2.0 * mu0;
  }
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b)
      if (!std::isfinite(c0[a * nv + b]) || std::fabs(c0[a * nv + b] - c0[b * nv + a]) > 1e-12 * (1 + std::fabs(c0[a * nv + b]))) {
        fh::set_error("C0 not finite/symmetric");
        return FH_ERR_ARG;
      }
  if (!cholesky_ok(c0, nv)) { fh::set_error("C0 is not positive definite"); return FH_ERR_ARG; }
  std::memcpy(s->C0, c0, sizeof(c0));
  fh::GreenParams GP{};
  GP.d = d; GP.nv = nv; GP.ntri = s->g.ntri; GP.nd = s->g.nd;
  for (int k = 0; k < 3; ++k) GP.dims[k] = s->g.dims[k];
  GP.H = s->g.H; GP.nhalf = s->g.nhalf; GP.D = s->P.D; GP.sign = s->P.sign;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      GP.M[i][j] = s->P.M[i][j];
      GP.adjT[i][j] = s->P.adjT[i][j];
      GP.Fmap[i][j] = s->P.Fmap[i][j];
    }
  GP.kind = s->gen.kind;
  for (int i = 0; i < 3; ++i) GP.alpha[i] = s->gen.alpha[i];
  GP.n_xi = s->gen.n_xi;
  for (int q = 0; q < 3 * 16; ++q) GP.xi[q] = s->gen.xi[q];
  GP.radius = s->gen.alias_radius;
  mandel_to_c4(c0, d, GP.C4);
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  CK(cudaMemsetAsync(s->err, 0, sizeof(int), s->work));
  const int blocks = (int)((s->g.nhalf + 127) / 128);
  if (closed_form_table(s, c0, &GP)) {
    int geo[2] = {-1, -1};
    const bool mirror = mirror_axes(s, geo);
    const bool cubic = mirror && cubic_axes(s, GP);
    long long nthreads = s->g.nhalf;
    if (mirror) nthreads = (long long)(s->g.dims[0] / 2 + 1) * (d == 3 ? s->g.dims[1] / 2 + 1 : 1) * s->g.H;
    if (cubic) {   // storage triples N/2 >= l0 >= l1 >= l2 >= 0
      const long long n = s->g.dims[0] / 2 + 1;
      nthreads = n * (n + 1) * (n + 2) / 6;
    }
    // 64-thread blocks: the cubic grid is small (47 905 threads at 128^3)
    const int tpb = cubic ? 64 : 128;
    const int mblocks = (int)((nthreads + tpb - 1) / tpb);
    if (d == 2)
      fh::green_table_iso<2><<<mblocks, tpb, 0, s->work>>>(GP, s->G64, s->G32, s->err, mirror, geo[0], geo[1], 0);
    else
      fh::green_table_iso<3><<<mblocks, tpb, 0, s->work>>>(GP, s->G64, s->G32, s->err, mirror, geo[0], geo[1],
                                                           cubic ? 1 : 0);
  } else {
    fh::green_table<<<blocks, 128, 0, s->work>>>(GP, s->G64, s->G32, s->err);
  }
  CK(cudaGetLastError());
  // the constitutive stage of the 3-D row passes skips structural zeros when
  // every phase matrix and C0 have them (then C_p - C0 has them too)
  s->dc_decoupled = nv == 6 && !s->field && decoupled6(c0);
  for (int q = 0; q < s->nphase && s->dc_decoupled; ++q) s->dc_decoupled = decoupled6(s->Cp + q * 36);
  // stiffness differences C_p - C0
  double dc[kMaxPhases * 36];
  float dcf[kMaxPhases * 36];
  for (int q = 0; q < s->nphase; ++q)
    for (int e = 0; e < nv * nv; ++e) {
      dc[q * nv * nv + e] = s->Cp[q * nv * nv + e] - c0[e];
      dcf[q * nv * nv + e] = (float)dc[q * nv * nv + e];
    }
  if (s->field) {   // point-by-point stiffness: C(x) - C0 and the FP32 copies
    fh::Tri21 c0t{};
    int t = 0;
    for (int a = 0; a < nv; ++a)
      for (int b = a; b < nv; ++b) c0t.v[t++] = c0[a * nv + b];
    fh::field_prepare<<<1024, kThreads, 0, s->work>>>(s->Cf64, c0t, s->g.ntri, s->g.m, s->dCf64, s->dCf32, s->Cf32);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(s->dC64, dc, sizeof(double) * s->nphase * nv * nv, cudaMemcpyHostToDevice, s->work));
  CK(cudaMemcpyAsync(s->dC32, dcf, sizeof(float) * s->nphase * nv * nv, cudaMemcpyHostToDevice, s->work));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->work));
  CK(cudaStreamSynchronize(s->work));
  if (herr != 0) {
    fh::set_error("alias sum of |c_k(f)|^2 vanishes: translates cannot be orthonormalised");
    return (fh_status)herr;
  }
  s->have_table = true;
  return FH_OK;
}

fh_status fh_set_reference(fh_solver* s, const double* C0) {
  return checked(fh_set_reference_impl(s, C0));
}

}  // extern "C"

namespace {

struct PhaseOut {
  int nload = 0;
  LoadState hs[FH_MAX_LOADS];
  double ms[FH_MAX_LOADS * fh::MAXV];
  float elapsed = 0.f;
  long long launches = 0;
  int path = 1, cs = 0;
};

// One run of the fixed point in one precision, in two halves so that a batch
// of solvers can have their cluster-resident solves in flight together.
// begin_phase enqueues the work; for the cluster path it returns without
// waiting (the results are copied to pinned host memory on the solver's
// stream), for the pass path it runs the host-driven loop to completion.
// end_phase waits for the solver's stream and collects the results.
// `start` (may be null) gives the per-load state to continue from.
fh_status begin_phase(fh_solver* s, int nload, const double* eps0, double tol, int max_iter, int prec, int init,
                      int chunk, int want_path, int want_cs, const LoadState* start, PhaseOut* out,
                      int stall_window = 0, bool defer_cluster = false) {
  const int nv = s->g.nv;
  Control h{};
  h.stall_window = stall_window;
  h.form = s->form;
  h.decoupled = s->dc_decoupled ? 1 : 0;
  for (int l = 0; l < nload; ++l)
    for (int c = 0; c < nv; ++c) h.eps0[l][c] = eps0[l * nv + c];
  h.tol = tol;
  h.max_iter = max_iter;
  h.nload = nload;
  h.hist_cap = kHistCap;
  CK(cudaMemcpyAsync(s->ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s->work));
  if (start) CK(cudaMemcpyAsync(s->st, start, nload * sizeof(LoadState), cudaMemcpyHostToDevice, s->work));
  else CK(cudaMemsetAsync(s->st, 0, FH_MAX_LOADS * sizeof(LoadState), s->work));
  const size_t nfield = (size_t)nload * nv * s->g.m;
  const unsigned conv_blocks = 1024;
  if (init == 0) {
    if (prec == FH_PREC_FP64) CK(cudaMemsetAsync(s->E64, 0, nfield * sizeof(double), s->work));
    else CK(cudaMemsetAsync(s->E32, 0, nfield * sizeof(float), s->work));
  } else if (s->E_prec != prec) {
    if (prec == FH_PREC_FP64) fh::convert_copy<double, float><<<conv_blocks, kThreads, 0, s->work>>>(s->E64, s->E32, (long long)nfield);
    else fh::convert_copy<float, double><<<conv_blocks, kThreads, 0, s->work>>>(s->E32, s->E64, (long long)nfield);
    CK(cudaGetLastError());
  }
  s->E_prec = prec;
  fh_status rc = prec == FH_PREC_FP64 ? choose_path<double>(s, want_path, want_cs, &out->path, &out->cs)
                                      : choose_path<float>(s, want_path, want_cs, &out->path, &out->cs);
  if (rc != FH_OK) return rc;
  if (out->path == 2 && defer_cluster) {
    // the cluster solve itself is queued by the caller (batched solves)
    out->nload = nload;
    CK(cudaEventRecord(s->ev0, s->work));
    return FH_OK;
  }
  if (out->path == 2)
    rc = prec == FH_PREC_FP64 ? run_solve_cluster<double>(s, nload, out->cs, &out->launches)
                              : run_solve_cluster<float>(s, nload, out->cs, &out->launches);
  else if (s->method == 1)
    rc = prec == FH_PREC_FP64 ? run_bicgstab<double>(s, prec, nload, chunk, max_iter, &out->launches)
                              : run_bicgstab<float>(s, prec, nload, chunk, max_iter, &out->launches);
  else
    rc = prec == FH_PREC_FP64 ? run_solve<double>(s, prec, nload, chunk, max_iter, &out->launches)
                              : run_solve<float>(s, prec, nload, chunk, max_iter, &out->launches);
  if (rc != FH_OK) return rc;
  CK(cudaMemcpyAsync(s->h_states, s->st, sizeof(LoadState) * nload, cudaMemcpyDeviceToHost, s->work));
  CK(cudaMemcpyAsync(s->h_ms, s->mstress, sizeof(double) * nload * fh::MAXV, cudaMemcpyDeviceToHost, s->work));
  out->nload = nload;
  return FH_OK;
}

fh_status end_phase(fh_solver* s, PhaseOut* out) {
  CK(cudaStreamSynchronize(s->work));
  std::memcpy(out->hs, s->h_states, sizeof(LoadState) * out->nload);
  std::memcpy(out->ms, s->h_ms, sizeof(double) * out->nload * fh::MAXV);
  CK(cudaEventElapsedTime(&out->elapsed, s->ev0, s->ev1));
  return FH_OK;
}

fh_status solve_phase(fh_solver* s, int nload, const double* eps0, double tol, int max_iter, int prec, int init,
                      int chunk, int want_path, int want_cs, const LoadState* start, PhaseOut* out,
                      int stall_window = 0) {
  NvtxRange range(s->method == 1 ? (prec == FH_PREC_FP64 ? "BiCGStab FP64" : "BiCGStab FP32")
                                 : (prec == FH_PREC_FP64 ? "fixed point FP64" : "fixed point FP32"));
  fh_status rc = begin_phase(s, nload, eps0, tol, max_iter, prec, init, chunk, want_path, want_cs, start, out,
                             stall_window);
  if (rc != FH_OK) return rc;
  return end_phase(s, out);
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

fh_status validate_solve(fh_solver* s, int nload, const double* eps0, const fh_solve_opts* opts) {
  if (!s || !eps0 || !opts) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (!s->have_table) { fh::set_error("set stiffness and reference medium first"); return FH_ERR_STATE; }
  if (nload < 1 || nload > s->nload_max) { fh::set_error("nload out of range"); return FH_ERR_ARG; }
  if (opts->max_iter < 1 || opts->max_iter > 10000000 || !(opts->tol >= 0.0)) { fh::set_error("bad tol/max_iter"); return FH_ERR_ARG; }
  if (opts->precision != FH_PREC_FP64 && opts->precision != FH_PREC_FP32 && opts->precision != FH_PREC_MIXED) {
    fh::set_error("unknown precision");
    return FH_ERR_ARG;
  }
  if (opts->init != 0 && opts->init != 1) { fh::set_error("init must be 0 or 1"); return FH_ERR_ARG; }
  if (opts->form != 0 && opts->form != 1) { fh::set_error("form must be 0 or 1"); return FH_ERR_ARG; }
  if (opts->tune < 0 || opts->tune >= 2 + FH_TUNE_CANDIDATES) {
    fh::set_error("tune must be 0, 1, or 2 + a candidate index");
    return FH_ERR_ARG;
  }
  if (opts->path < 0 || opts->path > 3 || (opts->cluster != 0 && opts->cluster != 8 && opts->cluster != 16)) {
    fh::set_error("path must be 0..3 and cluster 0, 8 or 16");
    return FH_ERR_ARG;
  }
  if (opts->method != 0 && opts->method != 1) { fh::set_error("method must be 0 or 1"); return FH_ERR_ARG; }
  if (opts->method == 1 && (opts->form != 0 || opts->tune != 0)) {
    fh::set_error("BiCGStab (method 1) solves form 0 and takes no tuning");
    return FH_ERR_ARG;
  }
  if (opts->method == 1 && opts->path == 2) {
    fh::set_error("BiCGStab (method 1) runs on the whole-GPU passes (path 1)");
    return FH_ERR_UNSUPPORTED;
  }
  for (int i = 0; i < nload * s->g.nv; ++i)
    if (!std::isfinite(eps0[i])) { fh::set_error("non-finite eps0"); return FH_ERR_ARG; }
  return FH_OK;
}

int chunk_of(const fh_solve_opts* opts) { return opts->chunk > 0 ? std::min(opts->chunk, 1024) : 32; }

// The FP64 phase of the mixed mode usually needs one or two iterations: its
// graph replays two at a time, so that the loads that have stopped do not run
// through a long chunk of early-exit passes (each FP64 row pass still
// launches its blocks and reduces their partial sums)
int polish_chunk(int chunk) { return std::min(chunk, 2); }

// start states of the FP64 step of the mixed mode: continue every load's count
void polish_start(const PhaseOut& A, LoadState* st0) {
  for (int l = 0; l < A.nload; ++l) {
    st0[l] = A.hs[l];
    st0[l].done = 0;
    st0[l].inc = 0;
    st0[l].r_best = 0.0;
    st0[l].since_best = 0;
    st0[l].status = 0;
  }
}

// mixed mode: the FP32 phase stops a load whose residual has not improved by 1%
// for this many iterations (its FP32 rounding floor), and the FP64 phase
// continues every load until its FP64 Cauchy residual meets the tolerance
constexpr int kStallWindow = 50;

fh_status finish_solve(fh_solver* s, int nload, const double* eps0, const PhaseOut& A, PhaseOut* B, bool mixed,
                       fh_result* res) {
  const int nv = s->g.nv;
  const PhaseOut* fin = &A;
  if (mixed) {
    B->elapsed += A.elapsed;
    B->launches += A.launches;
    fin = B;
  }
  fh_status worst = FH_OK;
  auto rank = [](int st) { return st == FH_NONFINITE ? 3 : st == FH_DIVERGED ? 2 : st == FH_NOT_CONVERGED ? 1 : 0; };
  if (res) std::memset(res, 0, sizeof(*res));
  for (int l = 0; l < nload; ++l) {
    const LoadState& hs = fin->hs[l];
    if (rank(hs.status) > rank(worst)) worst = (fh_status)hs.status;
    s->last_iters[l] = hs.iter;
    if (res) {
      res->iterations[l] = hs.iter;
      res->residual[l] = hs.r;
      res->status[l] = hs.status;
      for (int c = 0; c < nv; ++c) res->mean_stress[l * 6 + c] = fin->ms[l * fh::MAXV + c];
    }
    for (int c = 0; c < nv; ++c) {
      s->last_ms[l * 6 + c] = fin->ms[l * fh::MAXV + c];
      s->last_eps0[l * 6 + c] = eps0[l * nv + c];
    }
  }
  if (res) {
    res->elapsed_ms = fin->elapsed;
    res->kernel_launches = fin->launches;
    res->path = A.path;
    res->cluster = A.cs;
  }
  s->last_nload = nload;
  s->have_solution = true;
  return worst;
}

int status_rank(fh_status st) {
  return st == FH_NONFINITE ? 3 : st == FH_DIVERGED ? 2 : st == FH_NOT_CONVERGED ? 1 : 0;
}

// Autotuner: time every eligible launch configuration (whole-GPU passes,
// cluster-resident with 8 or 16 CTAs) for a few iterations of the actual loads
// in the given bulk precision and keep the fastest per iteration.  The trials
// overwrite the solver's strain, so they run only for solves that start from
// E = 0.
// Autotuner variants of the whole-GPU passes for one bulk precision; each
// starts from the shapes and radix schedules choose_shapes and make_plan gave.
// Returns false where the variant does not apply (or changes nothing).
//   0 the defaults
//   4 the block row pass with twice the rows per block
//   5 the block line passes with twice the tile width (columns per block);
//     rows and 3-D FP32 columns of 32-128 points by the earlier passes (warp
//     exchange in FP32, the block row pass in FP64) in place of the two-step
//     passes
//   6 every axis's radix schedule in reverse order
//   7 radix-4 stages in place of radix-8 and radix-2 pairs
bool apply_variant(fh_solver* s, int prec, int var) {
  const fh_solver::PassShapes& d = s->shape_def[prec];
  const GridInfo& g = s->g;
  s->rpb_gen[prec] = d.rpb_gen;
  s->row_bpl_gen[prec] = d.row_bpl_gen;
  s->row_smem_gen[prec] = d.row_smem_gen;
  for (int a = 0; a < 3; ++a) {
    s->lineW[prec][a] = d.lineW[a];
    s->ntiles[prec][a] = d.ntiles[a];
    s->line_smem[prec][a] = d.line_smem[a];
    s->ax[a].planp[prec] = d.plans[a];
  }
  s->col2s = true;
  if (var == 0) return true;
  if (var == 4) {
    if (s->row_warp[prec] > 0 && !s->field) return false;   // the warp row pass runs instead
    if (s->row2[prec] > 0 && !s->field) return false;       // the two-step row pass runs instead
    const int rpb = 2 * d.rpb_gen;
    if (rpb > g.nrows) return false;
    const int Lp = prec == FH_PREC_FP64 ? fh::padded_len<3>(g.L) : fh::padded_len<4>(g.L);
    const size_t sm = (size_t)2 * ((rpb * g.nv + 1) / 2) * Lp * csize(prec);
    if (sm > kMaxSmem) return false;
    s->rpb_gen[prec] = rpb;
    s->row_bpl_gen[prec] = (int)((g.nrows + rpb - 1) / rpb);
    s->row_smem_gen[prec] = sm;
    return true;
  }
  if (var == 5) {
    bool any = false;
    if (s->row2[prec] > 0 && !s->field) {
      s->col2s = false;
      any = true;
    }
    for (int a = 0; a + 1 < g.nd; ++a) {
      if (col2_len(s, prec, a) > 0) {
        s->col2s = false;
        any = true;
      }
      if (col_warp_p(s, prec, a) > 0) continue;
      const int W = 2 * d.lineW[a];
      const size_t sm = (size_t)2 * g.nv * W * (g.dims[a] + 1) * csize(prec);
      if (W > g.H || sm > kMaxSmem) continue;
      s->lineW[prec][a] = W;
      s->ntiles[prec][a] = (g.H + W - 1) / W;
      s->line_smem[prec][a] = sm;
      any = true;
    }
    return any;
  }
  bool any = false;
  for (int a = 0; a < g.nd; ++a) {
    fh::DevPlan p = d.plans[a];
    if (var == 6) {
      std::reverse(p.r, p.r + p.np);
    } else {   // var 7: the power of two as radix-4 stages (and one radix 2), the odd radices as before
      int e = 0, odd[24], no = 0;
      for (int q = 0; q < p.np; ++q) {
        const int r = p.r[q];
        if (r == 2) e += 1;
        else if (r == 4) e += 2;
        else if (r == 8) e += 3;
        else odd[no++] = r;
      }
      int np = 0;
      for (int k = 0; k < e / 2 && np < 24; ++k) p.r[np++] = 4;
      if ((e & 1) && np < 24) p.r[np++] = 2;
      for (int k = 0; k < no && np < 24; ++k) p.r[np++] = odd[k];
      if (np != (e / 2) + (e & 1) + no) continue;
      p.np = np;
    }
    bool same = p.np == d.plans[a].np;
    for (int q = 0; same && q < p.np; ++q) same = p.r[q] == d.plans[a].r[q];
    if (same) continue;
    s->ax[a].planp[prec] = p;
    any = true;
  }
  return any;
}

// Autotuner: time every candidate -- whole-GPU passes (with the default
// shapes, the fused plane pass, and variants 4-7 of apply_variant) and
// cluster-resident solves of 8 and 16 CTAs -- for 24 iterations of the actual
// loads, keep the fastest (its shapes stay with the solver).
constexpr int kCandPath[FH_TUNE_CANDIDATES] = {1, 2, 2, 3, 1, 1, 1, 1};
constexpr int kCandCs[FH_TUNE_CANDIDATES] = {0, 8, 16, 0, 0, 0, 0, 0};
constexpr int kCandVar[FH_TUNE_CANDIDATES] = {0, 0, 0, 0, 4, 5, 6, 7};

fh_status autotune(fh_solver* s, int nload, const double* eps0, int prec, int chunk) {
  const int slot = prec == FH_PREC_FP64 ? 0 : 1;
  const int* cand_path = kCandPath;
  const int* cand_cs = kCandCs;
  const int* cand_var = kCandVar;
  const int iters = 24;
  float best = 1e30f;
  int best_c = 0;
  for (int c = 0; c < FH_TUNE_CANDIDATES; ++c) {
    s->tuned_us[slot][c] = -1.f;
    if (!apply_variant(s, prec, cand_var[c])) continue;
    if (c == 3 && !(prec == FH_PREC_FP32 && s->plane[1] > 0 && !s->field)) continue;
    clear_graphs(s);
    int path = 1, cs = 0;
    fh_status rc = prec == FH_PREC_FP64 ? choose_path<double>(s, cand_path[c], cand_cs[c], &path, &cs)
                                        : choose_path<float>(s, cand_path[c], cand_cs[c], &path, &cs);
    if (rc == FH_ERR_UNSUPPORTED) { fh::set_error(""); continue; }
    if (rc != FH_OK) return rc;
    PhaseOut P;
    for (int rep = 0; rep < 2; ++rep) {  // the first run pays one-time set-up
      rc = solve_phase(s, nload, eps0, 0.0, iters, prec, 0, chunk, cand_path[c], cand_cs[c], nullptr, &P);
      if (rc != FH_OK) return rc;
    }
    const float us = 1e3f * P.elapsed / iters;
    s->tuned_us[slot][c] = us;
    if (us < best) {
      best = us;
      best_c = c;
      s->tuned_path[slot] = cand_path[c] == 3 ? 3 : P.path;
      s->tuned_cs[slot] = P.cs;
    }
  }
  apply_variant(s, prec, cand_var[best_c]);
  clear_graphs(s);
  s->tuned_cand[slot] = best_c;
  return FH_OK;
}

}  // namespace

namespace {

// After a queued cluster solve: the mean stresses and the read-back that
// begin_phase does for a solve it runs itself.
template <typename T>
fh_status finish_deferred(fh_solver* s, int nload, PhaseOut* out) {
  const int bpl = std::max(1, (int)std::min<long long>((s->g.m + kThreads - 1) / kThreads, kMeanBlocks));
  if (!s->skip_mean)
    fh::mean_stress<T><<<nload * bpl, kThreads, 0, s->work>>>(s->g, Eptr<T>(s), s->phase, s->Cp64, s->ctl, s->partials2,
                                                              s->mstress, bpl, s->field ? s->Cf64 : nullptr, s->nphase);
  CK(cudaGetLastError());
  CK(cudaEventRecord(s->ev1, s->work));
  CK(cudaMemcpyAsync(s->h_states, s->st, sizeof(LoadState) * nload, cudaMemcpyDeviceToHost, s->work));
  CK(cudaMemcpyAsync(s->h_ms, s->mstress, sizeof(double) * nload * fh::MAXV, cudaMemcpyDeviceToHost, s->work));
  out->launches = s->skip_mean ? 1 : 2;   // its share of the queue launch, and the mean stress
  return FH_OK;
}

// One queue launch for every (solver, load) of a group of deferred cluster
// solves that share precision, n_v, cluster size and radix variant; tasks are
// ordered largest pattern first, and as many clusters as fit stay resident.
struct QueueGroup {
  int prec, nv, cs;
  bool pow2;
  std::vector<int> members;   // indices into the batch
};

template <typename T, int NV, int CS, bool POW2>
fh_status launch_queue(fh_solver* const* solvers, const std::vector<int>& members, const int* nload,
                       cudaStream_t stream, fh::ClusterTask** dtasks, unsigned int** dnext) {
  std::vector<fh::ClusterTask> tasks;
  size_t smem = 0;
  for (int i : members) {
    fh_solver* s = solvers[i];
    const bool gs = s->cl_gsmem[sizeof(T) == 8 ? 0 : 1][CS == 16 ? 1 : 0];
    smem = std::max(smem, fh::cluster_layout<T>(s->g.dims[0], s->g.L, s->g.nv, CS, gs).total);
    for (int l = 0; l < nload[i]; ++l) tasks.push_back(cluster_task<T, CS>(s, l));
  }
  std::stable_sort(tasks.begin(), tasks.end(),
                   [](const fh::ClusterTask& a, const fh::ClusterTask& b) { return a.g.m > b.g.m; });
  auto kern = fh::cluster_solve_2d<T, NV, CS, POW2>;
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (CS > 8) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<T, NV, CS, POW2>(smem, 1, stream, attr);
  int resident = 0;
  CK(cudaOccupancyMaxActiveClusters(&resident, kern, &cfg));
  const int nclusters = std::max(1, std::min<int>((int)tasks.size(), resident));
  cfg.gridDim = dim3(nclusters * CS);
  CK(cudaMalloc(dtasks, tasks.size() * sizeof(fh::ClusterTask)));
  CK(cudaMalloc(dnext, sizeof(unsigned int)));
  CK(cudaMemcpyAsync(*dtasks, tasks.data(), tasks.size() * sizeof(fh::ClusterTask), cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(*dnext, 0, sizeof(unsigned int), stream));
  const fh::ClusterTask* tp = *dtasks;
  const int nt = (int)tasks.size();
  unsigned int* np = *dnext;
  CK(cudaLaunchKernelEx(&cfg, kern, tp, nt, np));
  return FH_OK;
}

template <typename T, int NV>
fh_status launch_queue_nv(const QueueGroup& q, fh_solver* const* solvers, const int* nload, cudaStream_t stream,
                          fh::ClusterTask** dt, unsigned int** dn) {
  if (q.cs == 16)
    return q.pow2 ? launch_queue<T, NV, 16, true>(solvers, q.members, nload, stream, dt, dn)
                  : launch_queue<T, NV, 16, false>(solvers, q.members, nload, stream, dt, dn);
  return q.pow2 ? launch_queue<T, NV, 8, true>(solvers, q.members, nload, stream, dt, dn)
                : launch_queue<T, NV, 8, false>(solvers, q.members, nload, stream, dt, dn);
}

// Queue the deferred cluster solves of a phase: group them, let one stream
// per group wait for the set-up of its members, launch one queue kernel per
// group (the groups run concurrently), and let every solver's stream wait for
// its group's kernel before finishing its phase.
fh_status run_queued(fh_solver* const* solvers, const int* nload, const std::vector<int>& deferred, int prec,
                     std::vector<PhaseOut>& out) {
  if (deferred.empty()) return FH_OK;
  std::vector<QueueGroup> groups;
  for (int i : deferred) {
    const QueueGroup key{prec, solvers[i]->g.nv, out[i].cs, pow2_plans(solvers[i]), {}};
    auto it = std::find_if(groups.begin(), groups.end(), [&](const QueueGroup& q) {
      return q.nv == key.nv && q.cs == key.cs && q.pow2 == key.pow2;
    });
    if (it == groups.end()) { groups.push_back(key); it = groups.end() - 1; }
    it->members.push_back(i);
  }
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> evs;
  std::vector<void*> bufs;
  auto cleanup = [&]() {
    for (cudaStream_t q : streams) cudaStreamSynchronize(q);
    for (void* b : bufs) cudaFree(b);
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    for (cudaStream_t q : streams) cudaStreamDestroy(q);
  };
  auto new_event = [&](cudaEvent_t* e) {
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
    evs.push_back(*e);
    return true;
  };
  for (const QueueGroup& q : groups) {
    cudaStream_t qs;
    if (cudaStreamCreateWithFlags(&qs, cudaStreamNonBlocking) != cudaSuccess) { cleanup(); return FH_ERR_CUDA; }
    streams.push_back(qs);
    for (int i : q.members) {
      cudaEvent_t e;
      if (!new_event(&e) || cudaEventRecord(e, solvers[i]->work) != cudaSuccess ||
          cudaStreamWaitEvent(qs, e, 0) != cudaSuccess) {
        cleanup();
        return FH_ERR_CUDA;
      }
    }
    fh::ClusterTask* dt = nullptr;
    unsigned int* dn = nullptr;
    fh_status rc;
    if (prec == FH_PREC_FP64)
      rc = q.nv == 3 ? launch_queue_nv<double, 3>(q, solvers, nload, qs, &dt, &dn)
                     : launch_queue_nv<double, 6>(q, solvers, nload, qs, &dt, &dn);
    else
      rc = q.nv == 3 ? launch_queue_nv<float, 3>(q, solvers, nload, qs, &dt, &dn)
                     : launch_queue_nv<float, 6>(q, solvers, nload, qs, &dt, &dn);
    if (dt) bufs.push_back(dt);
    if (dn) bufs.push_back(dn);
    if (rc != FH_OK) { cleanup(); return rc; }
    cudaEvent_t done;
    if (!new_event(&done) || cudaEventRecord(done, qs) != cudaSuccess) { cleanup(); return FH_ERR_CUDA; }
    for (int i : q.members) {
      fh_solver* s = solvers[i];
      if (cudaStreamWaitEvent(s->work, done, 0) != cudaSuccess) { cleanup(); return FH_ERR_CUDA; }
      rc = prec == FH_PREC_FP64 ? finish_deferred<double>(s, nload[i], &out[i])
                                : finish_deferred<float>(s, nload[i], &out[i]);
      if (rc != FH_OK) { cleanup(); return rc; }
    }
  }
  cleanup();   // waits for the queue kernels; the solvers' streams carry on
  return FH_OK;
}

// Cluster size for a batched solve left to the library: a 16-CTA cluster has
// to sit inside one GPC, so at most one runs per GPC; 8-CTA clusters pack two
// per GPC.  A batch is throughput-bound, so it takes the 8-CTA cluster
// wherever the fields fit, else the usual choice (16, or the pass path).
fh_status batch_cluster_choice(fh_solver* s, int prec, int* path, int* cs) {
  bool ok8 = false;
  fh_status rc = prec == FH_PREC_FP64 ? cluster_fits<double, 8>(s, &ok8) : cluster_fits<float, 8>(s, &ok8);
  if (rc != FH_OK) return rc;
  if (ok8) { *path = 2; *cs = 8; }
  return FH_OK;
}

}  // namespace

extern "C" {

static fh_status fh_solve_impl(fh_solver* s, int nload, const double* eps0, const fh_solve_opts* opts, fh_result* res) {
  if (s) s->skip_mean = false;
  NvtxRange range("fh_solve");
  fh_status rc = validate_solve(s, nload, eps0, opts);
  if (rc != FH_OK) return rc;
  rc = join_user(s);
  if (rc != FH_OK) return rc;
  s->form = opts->form;
  const int chunk = chunk_of(opts);
  const bool mixed = opts->precision == FH_PREC_MIXED;
  const int prec1 = opts->precision == FH_PREC_FP64 ? FH_PREC_FP64 : FH_PREC_FP32;
  int path1 = opts->path, cs1 = opts->cluster, path2 = opts->path, cs2 = opts->cluster;
  if (opts->tune >= 2) {   // a given autotuner candidate, without timing
    const int c = opts->tune - 2;
    if (!apply_variant(s, prec1, kCandVar[c])) {
      fh::set_error("this autotuner candidate does not apply to the grid");
      return FH_ERR_UNSUPPORTED;
    }
    clear_graphs(s);
    path1 = kCandPath[c];
    cs1 = kCandCs[c];
  } else if (opts->tune && opts->path == 0 && opts->cluster == 0 && opts->init == 0) {
    for (int pr : {prec1, mixed ? (int)FH_PREC_FP64 : -1}) {
      if (pr < 0) continue;
      const int slot = pr == FH_PREC_FP64 ? 0 : 1;
      if (s->tuned_path[slot] == 0) {
        rc = autotune(s, nload, eps0, pr, chunk);
        if (rc != FH_OK) return rc;
      }
    }
    const int s1 = prec1 == FH_PREC_FP64 ? 0 : 1;
    path1 = s->tuned_path[s1];
    cs1 = s->tuned_cs[s1];
    path2 = s->tuned_path[0];
    cs2 = s->tuned_cs[0];
  }
  PhaseOut A, B;
  s->method = opts->method;
  if (s->method == 1) path1 = 1;
  // mixed BiCGStab: its FP32 phase stops on the recursively updated residual,
  // which drifts from the true one, so it aims at half the tolerance; the FP64
  // phase then usually needs a single fixed-point step to confirm it
  const double tol1 = (mixed && opts->method == 1) ? 0.5 * opts->tol : opts->tol;
  s->skip_mean = mixed;   // the FP64 phase computes the mean stress that is returned
  rc = solve_phase(s, nload, eps0, tol1, opts->max_iter, prec1, opts->init, chunk, path1, cs1, nullptr, &A,
                   mixed ? kStallWindow : 0);
  s->skip_mean = false;
  s->method = 0;
  if (rc != FH_OK) return rc;
  if (mixed) {
    // the FP64 phase is the fixed point in every method: its Cauchy residual is
    // the residual of the FP32 result, so it also removes the FP32 rounding
    LoadState st0[FH_MAX_LOADS];
    polish_start(A, st0);
    s->polish = true;
    rc = solve_phase(s, nload, eps0, opts->tol, opts->max_iter, FH_PREC_FP64, 1, polish_chunk(chunk), path2, cs2,
                     st0, &B);
    s->polish = false;
    if (rc != FH_OK) return rc;
  }
  return finish_solve(s, nload, eps0, A, &B, mixed, res);
}

fh_status fh_solve(fh_solver* s, int nload, const double* eps0, const fh_solve_opts* opts, fh_result* res) {
  return checked(fh_solve_impl(s, nload, eps0, opts, res));
}

static fh_status fh_solve_batch_impl(fh_solver* const* solvers, int n, const int* nload, const double* const* eps0,
                         const fh_solve_opts* opts, fh_result* res) {
  NvtxRange range("fh_solve_batch");
  if (!solvers || !nload || !eps0 || !opts || n < 1) { fh::set_error("null argument or empty batch"); return FH_ERR_ARG; }
  for (int i = 0; i < n; ++i) {
    fh_status rc = validate_solve(solvers[i], nload[i], eps0[i], opts);
    if (rc != FH_OK) return rc;
    solvers[i]->skip_mean = false;
    for (int j = 0; j < i; ++j)
      if (solvers[j] == solvers[i]) { fh::set_error("a solver appears twice in the batch"); return FH_ERR_ARG; }
  }
  const int chunk = chunk_of(opts);
  const bool mixed = opts->precision == FH_PREC_MIXED;
  const int prec1 = opts->precision == FH_PREC_FP64 ? FH_PREC_FP64 : FH_PREC_FP32;
  std::vector<PhaseOut> A(n), B(n);
  // largest problems first (longest-processing-time order): the small ones
  // fill the GPU at the end instead of leaving a long solve running alone
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)solvers[a]->g.m * nload[a] > (double)solvers[b]->g.m * nload[b];
  });
  // phase 1: every solver's work is enqueued before any is waited for; the
  // cluster-resident solves go through one persistent queue launch per
  // kernel variant
  std::vector<int> deferred1, deferred2;
  for (int i : order) {
    fh_status rc = join_user(solvers[i]);
    if (rc != FH_OK) return rc;
    solvers[i]->form = opts->form;
    int p1 = opts->path, c1 = opts->cluster;
    const int slot = prec1 == FH_PREC_FP64 ? 0 : 1;
    if (p1 == 0 && c1 == 0 && solvers[i]->tuned_path[slot] != 0) {   // keep an earlier tuning
      p1 = solvers[i]->tuned_path[slot];
      c1 = solvers[i]->tuned_cs[slot];
    } else if (p1 == 0 && c1 == 0) {
      fh_status rc = batch_cluster_choice(solvers[i], prec1, &p1, &c1);
      if (rc != FH_OK) return rc;
    }
    solvers[i]->method = opts->method;
    if (opts->method == 1) p1 = 1;
    solvers[i]->skip_mean = mixed;   // the FP64 phase computes the mean stress that is returned
    rc = begin_phase(solvers[i], nload[i], eps0[i], (mixed && opts->method == 1) ? 0.5 * opts->tol : opts->tol,
                     opts->max_iter, prec1, opts->init, chunk, p1, c1, nullptr, &A[i], mixed ? kStallWindow : 0, true);
    solvers[i]->method = 0;
    if (rc != FH_OK) return rc;
    if (A[i].path == 2) deferred1.push_back(i);
  }
  {
    fh_status rc = run_queued(solvers, nload, deferred1, prec1, A);
    for (int i = 0; i < n; ++i) solvers[i]->skip_mean = false;
    if (rc != FH_OK) return rc;
  }
  for (int i = 0; i < n; ++i) {
    fh_status rc = end_phase(solvers[i], &A[i]);
    if (rc != FH_OK) return rc;
  }
  if (mixed) {
    for (int i : order) {
      LoadState st0[FH_MAX_LOADS];
      polish_start(A[i], st0);
      int p2 = opts->path, c2 = opts->cluster;
      if (p2 == 0 && c2 == 0 && solvers[i]->tuned_path[0] != 0) {
        p2 = solvers[i]->tuned_path[0];
        c2 = solvers[i]->tuned_cs[0];
      } else if (p2 == 0 && c2 == 0) {
        fh_status rc = batch_cluster_choice(solvers[i], FH_PREC_FP64, &p2, &c2);
        if (rc != FH_OK) return rc;
      }
      fh_status rc = begin_phase(solvers[i], nload[i], eps0[i], opts->tol, opts->max_iter, FH_PREC_FP64, 1,
                                 polish_chunk(chunk), p2,
                                 c2, st0, &B[i], 0, true);
      if (rc != FH_OK) return rc;
      if (B[i].path == 2) deferred2.push_back(i);
    }
    {
      fh_status rc = run_queued(solvers, nload, deferred2, FH_PREC_FP64, B);
      if (rc != FH_OK) return rc;
    }
    for (int i = 0; i < n; ++i) {
      fh_status rc = end_phase(solvers[i], &B[i]);
      if (rc != FH_OK) return rc;
    }
  }
  fh_status worst = FH_OK;
  for (int i = 0; i < n; ++i) {
    fh_status st = finish_solve(solvers[i], nload[i], eps0[i], A[i], &B[i], mixed, res ? &res[i] : nullptr);
    if (status_rank(st) > status_rank(worst)) worst = st;
  }
  return worst;
}

fh_status fh_solve_batch(fh_solver* const* solvers, int n, const int* nload, const double* const* eps0,
                         const fh_solve_opts* opts, fh_result* res) {
  return checked(fh_solve_batch_impl(solvers, n, nload, eps0, opts, res));
}

fh_status fh_get_strain(const fh_solver* sc, int load, double* E) {
  fh_solver* s = const_cast<fh_solver*>(sc);
  if (!s || !E) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (load < 0 || load >= s->nload_max) { fh::set_error("load out of range"); return FH_ERR_ARG; }
  if (s->E_prec < 0) { fh::set_error("no strain available"); return FH_ERR_STATE; }
  const size_t n = (size_t)s->g.nv * s->g.m;
  const size_t off = (size_t)load * n;
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  if (s->E_prec == FH_PREC_FP64) {
    CK(cudaMemcpyAsync(E, s->E64 + off, n * sizeof(double), cudaMemcpyDefault, s->work));
  } else {
    if (!s->scratch64) CK(cudaMalloc(&s->scratch64, n * sizeof(double)));
    fh::convert_copy<double, float><<<1024, kThreads, 0, s->work>>>(s->scratch64, s->E32 + off, (long long)n);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(E, s->scratch64, n * sizeof(double), cudaMemcpyDefault, s->work));
  }
  CK(cudaStreamSynchronize(s->work));
  return FH_OK;
}

fh_status fh_set_strain(fh_solver* s, int load, const double* E) {
  if (!s || !E) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (load < 0 || load >= s->nload_max) { fh::set_error("load out of range"); return FH_ERR_ARG; }
  const size_t n = (size_t)s->g.nv * s->g.m;
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  if (s->E_prec == FH_PREC_FP32) {
    // keep every load in one precision: bring the others to FP64 first
    fh::convert_copy<double, float><<<1024, kThreads, 0, s->work>>>(s->E64, s->E32, (long long)(n * s->nload_max));
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(s->E64 + (size_t)load * n, E, n * sizeof(double), cudaMemcpyDefault, s->work));
  CK(cudaStreamSynchronize(s->work));
  s->E_prec = FH_PREC_FP64;
  return FH_OK;
}

fh_status fh_get_strain_f32(const fh_solver* sc, int load, float* E) {
  fh_solver* s = const_cast<fh_solver*>(sc);
  if (!s || !E) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (load < 0 || load >= s->nload_max) { fh::set_error("load out of range"); return FH_ERR_ARG; }
  if (s->E_prec < 0) { fh::set_error("no strain available"); return FH_ERR_STATE; }
  const size_t n = (size_t)s->g.nv * s->g.m;
  const size_t off = (size_t)load * n;
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  if (s->E_prec == FH_PREC_FP32) {
    CK(cudaMemcpyAsync(E, s->E32 + off, n * sizeof(float), cudaMemcpyDefault, s->work));
  } else {
    fh::convert_copy<float, double><<<1024, kThreads, 0, s->work>>>(s->E32 + off, s->E64 + off, (long long)n);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(E, s->E32 + off, n * sizeof(float), cudaMemcpyDefault, s->work));
  }
  CK(cudaStreamSynchronize(s->work));
  return FH_OK;
}

fh_status fh_set_strain_f32(fh_solver* s, int load, const float* E) {
  if (!s || !E) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (load < 0 || load >= s->nload_max) { fh::set_error("load out of range"); return FH_ERR_ARG; }
  const size_t n = (size_t)s->g.nv * s->g.m;
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  if (s->E_prec == FH_PREC_FP64) {
    // keep every load in one precision: bring the others to FP32 first
    fh::convert_copy<float, double><<<1024, kThreads, 0, s->work>>>(s->E32, s->E64, (long long)(n * s->nload_max));
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(s->E32 + (size_t)load * n, E, n * sizeof(float), cudaMemcpyDefault, s->work));
  CK(cudaStreamSynchronize(s->work));
  s->E_prec = FH_PREC_FP32;
  return FH_OK;
}

fh_status fh_get_ceff(const fh_solver* s, double* Ceff, int voigt) {
  if (!s || !Ceff) { fh::set_error("null argument"); return FH_ERR_ARG; }
  const int nv = s->g.nv;
  if (!s->have_solution || s->last_nload != nv) { fh::set_error("C_eff needs a solve with nload = n_v"); return FH_ERR_STATE; }
  // <sigma>_l = C_eff eps0_l  =>  S = E0 C^T  (rows l);  solve E0 X = S, C = X^T
  double A[36], X[36];
  for (int l = 0; l < nv; ++l)
    for (int c = 0; c < nv; ++c) {
      A[l * nv + c] = s->last_eps0[l * 6 + c];
      X[l * nv + c] = s->last_ms[l * 6 + c];
    }
  for (int col = 0; col < nv; ++col) {
    int piv = col;
    for (int r = col + 1; r < nv; ++r)
      if (std::fabs(A[r * nv + col]) > std::fabs(A[piv * nv + col])) piv = r;
    if (std::fabs(A[piv * nv + col]) < 1e-300) { fh::set_error("eps0 of the last solve is singular"); return FH_ERR_STATE; }
    for (int c = 0; c < nv; ++c) { std::swap(A[col * nv + c], A[piv * nv + c]); std::swap(X[col * nv + c], X[piv * nv + c]); }
    for (int r = 0; r < nv; ++r) {
      if (r == col) continue;
      const double f = A[r * nv + col] / A[col * nv + col];
      for (int c = 0; c < nv; ++c) { A[r * nv + c] -= f * A[col * nv + c]; X[r * nv + c] -= f * X[col * nv + c]; }
    }
  }
  for (int r = 0; r < nv; ++r)
    for (int c = 0; c < nv; ++c) X[r * nv + c] /= A[r * nv + r];
  const int d = s->g.d;
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      double v = X[b * nv + a];
      if (voigt) v /= ((a < d ? 1.0 : std::sqrt(2.0)) * (b < d ? 1.0 : std::sqrt(2.0)));
      Ceff[a * nv + b] = v;
    }
  return FH_OK;
}

fh_status fh_get_green(const fh_solver* s, double* G) {
  if (!s || !G) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (!s->have_table) { fh::set_error("no table"); return FH_ERR_STATE; }
  const int nv = s->g.nv, nt = s->g.ntri;
  const size_t nh = (size_t)s->g.nhalf;
  std::vector<double> t((size_t)nt * nh);
  CK(cudaMemcpy(t.data(), s->G64, t.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (size_t f = 0; f < nh; ++f) {
    int q = 0;
    for (int a = 0; a < nv; ++a)
      for (int b = a; b < nv; ++b) {
        const double v = t[(size_t)q * nh + f];
        G[f * nv * nv + a * nv + b] = v;
        G[f * nv * nv + b * nv + a] = v;
        ++q;
      }
  }
  return FH_OK;
}


static fh_status fh_profile_passes_impl(fh_solver* s, int nload, int precision, int reps, double* ms) {
  if (!s || !ms) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (!s->have_solution || nload != s->last_nload) { fh::set_error("profile needs a prior solve with the same nload"); return FH_ERR_STATE; }
  if (reps < 1 || reps > 100000) { fh::set_error("reps out of range"); return FH_ERR_ARG; }
  if (precision != FH_PREC_FP64 && precision != FH_PREC_FP32) { fh::set_error("unknown precision"); return FH_ERR_ARG; }
  if (precision != s->E_prec) { fh::set_error("profile precision must match the last solve"); return FH_ERR_STATE; }
  fh_status rc = join_user(s);
  if (rc != FH_OK) return rc;
  return precision == FH_PREC_FP64 ? profile_passes<double>(s, precision, nload, reps, ms)
                                   : profile_passes<float>(s, precision, nload, reps, ms);
}

fh_status fh_profile_passes(fh_solver* s, int nload, int precision, int reps, double* ms) {
  return checked(fh_profile_passes_impl(s, nload, precision, reps, ms));
}

fh_status fh_get_tuning(const fh_solver* s, int precision, int* path, int* cluster, int* candidate,
                        float* us_per_iter) {
  if (!s || !path || !cluster) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (precision != FH_PREC_FP64 && precision != FH_PREC_FP32) { fh::set_error("precision must be FP64 or FP32"); return FH_ERR_ARG; }
  const int slot = precision == FH_PREC_FP64 ? 0 : 1;
  *path = s->tuned_path[slot];
  *cluster = s->tuned_cs[slot];
  if (candidate) *candidate = s->tuned_cand[slot];
  if (us_per_iter)
    for (int c = 0; c < FH_TUNE_CANDIDATES; ++c) us_per_iter[c] = s->tuned_us[slot][c];
  return FH_OK;
}

fh_status fh_get_residuals(const fh_solver* s, int load, double* hist, int* n) {
  if (!s || !n) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (!s->have_solution || load < 0 || load >= s->last_nload) { fh::set_error("no such load in the last solve"); return FH_ERR_STATE; }
  const int cnt = std::min(s->last_iters[load], kHistCap);
  *n = cnt;
  if (hist && cnt > 0) CK(cudaMemcpy(hist, s->hist + (size_t)load * kHistCap, cnt * sizeof(double), cudaMemcpyDeviceToHost));
  return FH_OK;
}

}  // extern "C"
