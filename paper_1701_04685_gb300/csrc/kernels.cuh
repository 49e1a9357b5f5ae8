// Device kernels of the Basic-Scheme iteration on the Smith-normal-form grid.
//
// One iteration of the paper's fixed point (Eq. (pde_coefficients), Sec. 4)
// is split into passes over the stored fields:
//
//   row pass   (contiguous axis):  half spectrum -> inverse FFT -> E_new,
//              Cauchy-residual partial sums (FP64), store E_new, then
//              tau = (C(y) - C0):(E_new + eps0) -> forward FFT -> half spectrum.
//              Two real lines share one complex FFT (z = a + i b).
//   line pass  (every other axis): forward FFT, and on axis 0 the Green step
//              E^ = -Gamma^p tau^ (E^_0 = 0), then inverse FFT.
//   the last block of each row pass reduces the partial sums in a fixed order
//   and advances the per-load state (iteration count, r_n, stop flags).
//
// Layouts (all loads in one allocation):
//   E  [load][comp][m]              real, storage order (row-major grid)
//   S  [load][comp][rows][H]        complex half spectrum, H = L/2 + 1
//   G  [tri][n_half]                Gamma^p upper triangle, structure of arrays
#pragma once

#include <cstdint>

#include "fft.cuh"

namespace fh {

constexpr int MAXV = 6;  // n_v <= 6

// ---------------------------------------------------------------------------
// Checked build (compiled with -DFH_CHECKED): the global-memory and tile
// accesses of the solver's kernels test their index against the extent of
// the array they address (for the fields: the loads of the launch).  The
// first violation is recorded (site, index, extent, and a count of all of
// them) and the access is skipped, so that a wrong index becomes an error
// status instead of a fault; the host reads the record after each solve.
// Without FH_CHECKED the tests compile away.
// ---------------------------------------------------------------------------
enum CheckSite {
  CK_ROW_S = 1, CK_ROW_E, CK_ROW_PHASE, CK_ROW_SMEM, CK_FIELD, CK_PARTIALS,
  CK_LINE_S, CK_LINE_G, CK_LINE_SMEM,
  CK_WROW_S, CK_WROW_E, CK_WROW_PHASE, CK_WROW_SCRATCH,
  CK_COL_S, CK_COL_G, CK_COL_TILE,
  CK_C2_S, CK_C2_G, CK_C2_TILE,
  CK_GREEN1D, CK_MEAN, CK_KRY, CK_CLUSTER, CK_TABLE, CK_SELFTEST,
  CK_NSITES
};

struct CheckRecord {
  unsigned long long count;
  long long index, extent;
  int site, pad;
};

#ifdef FH_CHECKED
static __device__ CheckRecord g_check;
__device__ __noinline__ bool check_fail(int site, long long i, long long n) {
  if (atomicAdd(&g_check.count, 1ull) == 0ull) {
    g_check.site = site;
    g_check.index = i;
    g_check.extent = n;
  }
  return false;
}
#define FH_IN(site, i, n) \
  (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n)) || \
   ::fh::check_fail((site), (long long)(i), (long long)(n)))
#else
#define FH_IN(site, i, n) true
#endif

struct GridInfo {
  int d, nv, ntri, nd;
  int dims[3];
  int L, H;
  long long m, nrows, nhalf;
  double inv_m;
};

struct LoadState {
  int iter;
  int done;
  int status;
  int inc;          // consecutive growing residuals
  double r;         // last residual
  double r_first;
  double r_best;    // smallest residual so far
  int since_best;   // iterations since r_best last improved by 1%
  int pad_;
  double n_first;   // ||E_1 + eps0||^2 of the first iteration: the divergence test's scale
};

// internal status: the residual stopped improving (FP32 rounding floor); the
// mixed mode then continues in FP64
constexpr int kStatusStalled = 4;

struct Control {
  double eps0[16][6];
  double tol;
  int max_iter;
  int nload;
  int hist_cap;
  int all_done;
  unsigned int ticket;
  unsigned int ticket2;
  int err;
  int stall_window;  // > 0: stop a load whose residual has not improved by 1% for this many iterations
  int form;          // 0: Eq. (pde_coefficients), E <- -Gamma^p (C - C0)(E + eps0)
                     // 1: Eq. (pde_coefficients_variational), E <- E - Gamma^p C (E + eps0)
  int decoupled;     // 3-D phase tables with zero normal-shear blocks and a diagonal shear
                     // block (isotropic, cubic, orthotropic phases in the grid axes): the
                     // constitutive stage skips the structural zeros (stress6_decoupled)
  int no_forward;    // two-step row pass: stop after the E update and the residual (no tau,
                     // no forward transform); the spectra are then stale and a FIRST pass
                     // must precede the next iteration
  int pad3;
};

// tau = D x for a 6 x 6 Mandel matrix D whose normal-shear blocks are zero and
// whose shear block is diagonal, from its 12 nonzero entries
//   d = (D00, D01, D02, D10, D11, D12, D20, D21, D22, D33, D44, D55).
// The products are summed in the order of the full row-by-row product and the
// skipped terms are exact zeros, so the result has the value of the full
// 36-term product (12 FMAs instead of 36).
template <typename T>
__device__ __forceinline__ void stress6_decoupled(const T* d, const T* x, T* tau) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T t = T(0);
    t = fma(d[3 * a], x[0], t);
    t = fma(d[3 * a + 1], x[1], t);
    t = fma(d[3 * a + 2], x[2], t);
    tau[a] = t;
  }
#pragma unroll
  for (int a = 3; a < 6; ++a) tau[a] = fma(d[6 + a], x[a], T(0));
}

// the 12 entries stress6_decoupled reads, from a 6 x 6 row-major matrix
template <typename T>
__device__ __forceinline__ T decoupled_entry(const T* D, int q) {
  return q < 9 ? D[(q / 3) * 6 + q % 3] : D[(q - 6) * 7];
}

// ---------------------------------------------------------------------------
// block reductions (fixed order -> deterministic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// sum over the block; result valid in thread 0.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Per-thread accumulator of the Cauchy-residual sums.  FP64 kernels add in
// double.  FP32 kernels keep a double-float pair (hi, lo) built with the exact
// TwoSum / TwoProduct transformations (Knuth; Dekker), which carries about 48
// significant bits while using only FP32 instructions: GB300's FP64 pipe is
// narrow enough that per-point double arithmetic would dominate an FP32
// iteration.  The pair is rounded to double once per thread, before the FP64
// block reduction.
template <typename T> struct ResAcc;
template <> struct ResAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_sq(double a) { s = fma(a, a, s); }
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct ResAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_sq(float a) {
    const float p = a * a;
    const float e = fmaf(a, a, -p);        // a*a = p + e exactly
    const float s = hi + p;                 // TwoSum(hi, p)
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);        // a*b = p + e exactly
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err + e;
  }
  // add a short FP32 partial sum (TwoSum only)
  __device__ __forceinline__ void add(float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Block sum of the per-thread accumulators; result valid in thread 0.  The
// FP32 variant reduces the double-float pairs across each warp with exact
// TwoSum steps in FP32 and converts once per warp, so the narrow FP64 pipe
// sees a handful of operations per block instead of several per thread.
__device__ __forceinline__ double block_sum_acc(const ResAcc<double>& a, double* red) { return block_sum(a.value(), red); }
__device__ __forceinline__ double block_sum_acc(const ResAcc<float>& a, double* red) {
  float hi = a.hi, lo = a.lo;
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_down_sync(0xffffffffu, hi, o);
    const float olo = __shfl_down_sync(0xffffffffu, lo, o);
    const float s = hi + ohi;                 // TwoSum(hi, ohi)
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (ohi - bp);
    hi = s;
    lo = lo + olo + e;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = (double)hi + (double)lo;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t += red[i];
  }
  return t;
}

// Both residual accumulators of a block reduced in one pass (one block
// barrier); the sums are valid in every lane of warp 0.  `red2` holds >= 32
// double2.  Fixed order, so every launch of the same shape gives the same bits.
__device__ __forceinline__ void two_sum_merge(float& hi, float& lo, float ohi, float olo) {
  const float s = hi + ohi;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (ohi - bp);
  hi = s;
  lo = lo + olo + e;
}
__device__ __forceinline__ void block_sum_pair(const ResAcc<float>& a, const ResAcc<float>& b, double2* red2,
                                               double& d2, double& n2) {
  float ah = a.hi, al = a.lo, bh = b.hi, bl = b.lo;
  for (int o = 16; o > 0; o >>= 1) {
    two_sum_merge(ah, al, __shfl_down_sync(0xffffffffu, ah, o), __shfl_down_sync(0xffffffffu, al, o));
    two_sum_merge(bh, bl, __shfl_down_sync(0xffffffffu, bh, o), __shfl_down_sync(0xffffffffu, bl, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float4* red4 = reinterpret_cast<float4*>(red2);
  if (lane == 0) red4[w] = make_float4(ah, al, bh, bl);
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const float4 v = lane < nw ? red4[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    ah = v.x; al = v.y; bh = v.z; bl = v.w;
    for (int o = 16; o > 0; o >>= 1) {
      two_sum_merge(ah, al, __shfl_down_sync(0xffffffffu, ah, o), __shfl_down_sync(0xffffffffu, al, o));
      two_sum_merge(bh, bl, __shfl_down_sync(0xffffffffu, bh, o), __shfl_down_sync(0xffffffffu, bl, o));
    }
    ah = __shfl_sync(0xffffffffu, ah, 0); al = __shfl_sync(0xffffffffu, al, 0);
    bh = __shfl_sync(0xffffffffu, bh, 0); bl = __shfl_sync(0xffffffffu, bl, 0);
    d2 = (double)ah + (double)al;
    n2 = (double)bh + (double)bl;
  }
}
__device__ __forceinline__ void block_sum_pair(const ResAcc<double>& a, const ResAcc<double>& b, double2* red2,
                                               double& d2, double& n2) {
  double x = a.s, y = b.s;
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red2[w] = make_double2(x, y);
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const double2 v = lane < nw ? red2[lane] : make_double2(0.0, 0.0);
    x = v.x; y = v.y;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
    d2 = __shfl_sync(0xffffffffu, x, 0);
    n2 = __shfl_sync(0xffffffffu, y, 0);
  }
}

// Advance the per-load state after one iteration's residual is known:
// r_n = sqrt(d2 / n2) (Sec. 4's Cauchy criterion), then the stop tests.
__device__ __forceinline__ void update_state(LoadState& s, double d2, double n2, double tol, int max_iter,
                                             int stall_window) {
  const double r = (n2 > 0.0) ? sqrt(d2 / n2) : sqrt(d2);
  s.iter += 1;
  if (s.iter == 1) { s.r_first = r; s.n_first = n2; }
  s.inc = (s.iter > 1 && r > s.r) ? s.inc + 1 : 0;
  s.r = r;
  if (s.since_best == 0 && s.r_best == 0.0) s.r_best = r;  // first step of this phase
  if (r < 0.99 * s.r_best) { s.r_best = r; s.since_best = 0; }
  else s.since_best += 1;
  if (!isfinite(r)) { s.status = FH_NONFINITE; s.done = 1; }
  else if (r <= tol) { s.status = FH_OK; s.done = 1; }
  // diverged: the residual kept growing, or the iterate itself grew by a factor
  // 1e6 in norm (a geometric divergence keeps r_n roughly constant, so the
  // residual alone does not show it)
  else if (s.inc >= 100 || (s.iter > 10 && r > 1e6 * s.r_first && r > 1.0) ||
           (s.iter > 10 && s.n_first > 0.0 && n2 > 1e12 * s.n_first)) { s.status = FH_DIVERGED; s.done = 1; }
  else if (stall_window > 0 && s.since_best >= stall_window) { s.status = kStatusStalled; s.done = 1; }
  else if (s.iter >= max_iter) { s.status = FH_NOT_CONVERGED; s.done = 1; }
}

__device__ void advance_state(LoadState& s, Control* ctl, double* hist, int load, double d2, double n2) {
  update_state(s, d2, n2, ctl->tol, ctl->max_iter, ctl->stall_window);
  if (s.iter <= ctl->hist_cap) hist[(size_t)load * ctl->hist_cap + (s.iter - 1)] = s.r;
}

// ---------------------------------------------------------------------------
// row pass along the contiguous axis (length L), fused with the pointwise
// constitutive stage and the residual.
// ---------------------------------------------------------------------------
// resident blocks per SM requested from the compiler (more than one capped
// the registers and spilled, measured slower)
template <typename T> struct PassOcc { static constexpr int value = 1; };

// KINV (with FIRST = false): the inverse half of an operator application for
// the Krylov solver.  The inverse transform gives y = -Gamma^p tau of the
// field X (= E) whose stress the previous FIRST pass transformed; the pass
// writes W = X - y = (I + Gamma^p (C - C0)) X to Wout and the block sums of
// W . Yaux (Yaux = X when null) and W . W to partials, and does nothing else.
template <typename T, int NV, bool FIRST, bool KINV = false>
__global__ void __launch_bounds__(256, PassOcc<T>::value) row_pass(GridInfo g, DevPlan plan, const cplx<T>* __restrict__ tw,
                                                T* __restrict__ E, cplx<T>* __restrict__ S,
                                                const uint8_t* __restrict__ phase, const T* __restrict__ dC,
                                                Control* ctl, LoadState* st, double* __restrict__ partials,
                                                double* __restrict__ hist, int rpb, int blocks_per_load,
                                                T* __restrict__ Wout = nullptr, const T* __restrict__ Yaux = nullptr,
                                                const T* __restrict__ Cfld = nullptr) {
  static_assert(!(FIRST && KINV), "the inverse-only pass follows a transform");
  // Cfld (not null): the stiffness of the constitutive stage given point by
  // point, upper triangle of the Mandel matrix as [tri][m] (C - C0, or C for
  // the variational form), instead of the phase table
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int s_skip;
  const int load = blockIdx.x / blocks_per_load;
  const int rb = blockIdx.x - load * blocks_per_load;
  const long long row0 = (long long)rb * rpb;
  const int nrow = (int)min((long long)rpb, g.nrows - row0);
  const int L = g.L, H = g.H;
  const int nreal = nrow * NV;
  const int npair = (nreal + 1) >> 1;
  constexpr int PS = sizeof(T) == 4 ? 4 : 3;   // one spare slot per 128-byte wavefront
  const int Lp = padded_len<PS>(L);
  cplx<T>* W0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* W1 = W0 + (size_t)((rpb * NV + 1) >> 1) * Lp;
  const FDiv fL = make_fdiv(L), fH = make_fdiv(H);

  __shared__ T dcs[16 * NV * NV];   // stiffness table of the pointwise stage
  for (int i = threadIdx.x; i < 16 * NV * NV; i += blockDim.x) dcs[i] = dC[i];
  if (threadIdx.x == 0) s_skip = st[load].done;
  __syncthreads();
  ResAcc<T> acc_d, acc_n;
  if (!s_skip) {
    T e0[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) e0[c] = (T)ctl->eps0[load][c];
    T* Eb = E + (size_t)load * NV * g.m + row0 * L;              // row0 of component 0
    const cplx<T>* Sr = S + ((size_t)load * NV * g.nrows + row0) * H;  // row0 of component 0
    cplx<T>* Sw = S + ((size_t)load * NV * g.nrows + row0) * H;
    const size_t cstrE = (size_t)g.m, cstrS = (size_t)g.nrows * H;
    // extents for the checked build: offsets of Sr / Eb inside S / E, the
    // fields of the launch's loads, one work buffer
    const long long sbase = ((long long)load * NV * g.nrows + row0) * H;
    const long long ebase = (long long)load * NV * g.m + row0 * L;
    const long long nS = (long long)ctl->nload * NV * g.nhalf, nE = (long long)ctl->nload * NV * g.m;
    const long long nW = (long long)((rpb * NV + 1) >> 1) * Lp;
    (void)sbase; (void)ebase; (void)nS; (void)nE; (void)nW;
    cplx<T>* Z = W0;
    cplx<T>* Zo = W1;
    if (!FIRST) {
      // 1. rebuild the two-real-lines-in-one complex spectrum Z = A + i B
      // four independent element pairs per thread are loaded before any is
      // stored, to keep enough global loads in flight
      constexpr int U = 4;
      const int total = npair * L;
      for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
        cplx<T> A[U], B[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base + u * blockDim.x;
          A[u].x = A[u].y = B[u].x = B[u].y = T(0);
          if (idx < total) {
            const int p = fdiv(idx, fL), k = idx - p * L;
            const int fa = 2 * p, fb = 2 * p + 1;
            const int kk = k <= (L >> 1) ? k : L - k;
            const int ra = fa / NV, ca = fa - ra * NV;
            const long long oa = (long long)ca * cstrS + ra * H + kk;
            if (FH_IN(CK_ROW_S, sbase + oa, nS)) A[u] = Sr[oa];
            if (fb < nreal) {
              const int rbb = fb / NV, cb = fb - rbb * NV;
              const long long ob = (long long)cb * cstrS + rbb * H + kk;
              if (FH_IN(CK_ROW_S, sbase + ob, nS)) B[u] = Sr[ob];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base + u * blockDim.x;
          if (idx < total) {
            const int p = fdiv(idx, fL), k = idx - p * L;
            if (k > (L >> 1)) { A[u].y = -A[u].y; B[u].y = -B[u].y; }
            cplx<T> z;
            z.x = A[u].x - B[u].y;
            z.y = A[u].y + B[u].x;
            if (FH_IN(CK_ROW_SMEM, p * Lp + padi<PS>(k), nW)) W0[p * Lp + padi<PS>(k)] = z;
          }
        }
      }
      __syncthreads();
      // 2. inverse FFT (unnormalised)
      Z = fft_lines_pp<+1, T, PS>(W0, W1, npair, Lp, plan, tw);
      Zo = (Z == W0) ? W1 : W0;
    }
    // 3. pointwise: E_new, residual sums, tau = (C - C0):(E_new + eps0)
    //    (variational form: E_new = E_old + update, tau = C:(E_new + eps0))
    const T scale = (T)g.inv_m;
    const bool incremental = ctl->form == 1;
    if constexpr (KINV) {
      const size_t ob = (size_t)load * NV * g.m + row0 * L;
      for (int idx = threadIdx.x; idx < nrow * L; idx += blockDim.x) {
        const int r = fdiv(idx, fL), x = idx - r * L;
        if (!FH_IN(CK_ROW_SMEM, ((r * NV + NV - 1) >> 1) * Lp + padi<PS>(x), nW)) continue;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const int f = r * NV + c;
          const cplx<T> zz = Z[(f >> 1) * Lp + padi<PS>(x)];
          const size_t o = ob + (size_t)c * cstrE + r * L + x;
          if (!FH_IN(CK_ROW_E, (long long)o, nE)) continue;
          const T w = E[o] - ((f & 1) ? zz.y : zz.x) * scale;
          Wout[o] = w;
          acc_d.add_prod(w, Yaux ? Yaux[o] : E[o]);
          acc_n.add_sq(w);
        }
      }
    }
    for (int idx = threadIdx.x; idx < (KINV ? 0 : nrow * L); idx += blockDim.x) {
      const int r = fdiv(idx, fL), x = idx - r * L;
      if (!(FH_IN(CK_ROW_E, ebase + r * L + x, nE) && FH_IN(CK_ROW_E, ebase + r * L + x + (NV - 1) * (long long)cstrE, nE) &&
            FH_IN(CK_ROW_SMEM, ((r * NV + NV - 1) >> 1) * Lp + padi<PS>(x), nW) &&
            FH_IN(Cfld ? CK_FIELD : CK_ROW_PHASE, (row0 + r) * L + x, g.m)))
        continue;
      T* ep = Eb + r * L + x;
      T en[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        const int f = r * NV + c;
        if (FIRST) {
          en[c] = ep[c * cstrE];
        } else {
          const cplx<T> zz = Z[(f >> 1) * Lp + padi<PS>(x)];
          en[c] = ((f & 1) ? zz.y : zz.x) * scale;
          const T eo = ep[c * cstrE];
          if (incremental) en[c] += eo;
          acc_d.add_sq(en[c] - eo);
          acc_n.add_sq(en[c] + e0[c]);
          ep[c * cstrE] = en[c];
        }
      }
      T tau[NV];
      if (Cfld) {
        const size_t pt = (size_t)(row0 + r) * L + x;
#pragma unroll
        for (int a = 0; a < NV; ++a) tau[a] = T(0);
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
          for (int b = a; b < NV; ++b) {
            const T cab = Cfld[(size_t)(a * NV - (a * (a - 1)) / 2 + (b - a)) * g.m + pt];
            tau[a] += cab * (en[b] + e0[b]);
            if (b != a) tau[b] += cab * (en[a] + e0[a]);
          }
      } else {
        const T* dc = dcs + (size_t)phase[(row0 + r) * L + x] * NV * NV;
#pragma unroll
        for (int a = 0; a < NV; ++a) {
          T t = T(0);
#pragma unroll
          for (int b = 0; b < NV; ++b) t += dc[a * NV + b] * (en[b] + e0[b]);
          tau[a] = t;
        }
      }
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const int f = r * NV + a;
        if (f & 1) Z[(f >> 1) * Lp + padi<PS>(x)].y = tau[a];
        else Z[(f >> 1) * Lp + padi<PS>(x)].x = tau[a];
      }
    }
    // odd number of real lines: the last pair's imaginary part is zero
    if (!KINV && (nreal & 1)) {
      for (int x = threadIdx.x; x < L; x += blockDim.x) Z[(npair - 1) * Lp + padi<PS>(x)].y = T(0);
    }
    __syncthreads();
    if (KINV) goto partial_sums;
    {
    // 4. forward FFT
    cplx<T>* Zf = fft_lines_pp<-1, T, PS>(Z, Zo, npair, Lp, plan, tw);
    // 5. split into the two half spectra A = (Z_k + conj Z_{L-k})/2, B = (Z_k - conj Z_{L-k})/(2i)
    for (int idx = threadIdx.x; idx < npair * H; idx += blockDim.x) {
      const int p = fdiv(idx, fH), k = idx - p * H;
      if (!FH_IN(CK_ROW_SMEM, p * Lp + padi<PS>(k == 0 ? 0 : L - k), nW) || !FH_IN(CK_ROW_SMEM, p * Lp + padi<PS>(k), nW))
        continue;
      const cplx<T> zk = Zf[p * Lp + padi<PS>(k)];
      const cplx<T> zm = Zf[p * Lp + padi<PS>(k == 0 ? 0 : L - k)];
      cplx<T> A, B;
      A.x = T(0.5) * (zk.x + zm.x);
      A.y = T(0.5) * (zk.y - zm.y);
      B.x = T(0.5) * (zk.y + zm.y);
      B.y = T(-0.5) * (zk.x - zm.x);
      const int fa = 2 * p, fb = 2 * p + 1;
      const int ra = fa / NV, ca = fa - ra * NV;
      const long long oa = (long long)ca * cstrS + ra * H + k;
      if (FH_IN(CK_ROW_S, sbase + oa, nS)) Sw[oa] = A;
      if (fb < nreal) {
        const int rbb = fb / NV, cb = fb - rbb * NV;
        const long long ob = (long long)cb * cstrS + rbb * H + k;
        if (FH_IN(CK_ROW_S, sbase + ob, nS)) Sw[ob] = B;
      }
    }
    }
  }
partial_sums:
  if (FIRST) return;
  // 6. partial sums of this block
  const double d2 = block_sum_acc(acc_d, red);
  const double n2 = block_sum_acc(acc_n, red);
  if (KINV) {
    if (threadIdx.x == 0) {
      partials[2 * (size_t)blockIdx.x] = d2;
      partials[2 * (size_t)blockIdx.x + 1] = n2;
    }
    return;
  }
  __shared__ unsigned int s_ticket;
  if (threadIdx.x == 0) {
    partials[2 * (size_t)blockIdx.x] = d2;
    partials[2 * (size_t)blockIdx.x + 1] = n2;
    __threadfence();
    s_ticket = atomicAdd(&ctl->ticket, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  // 7. last block: fixed-order reduction per load, state update
  __threadfence();
  for (int load2 = 0; load2 < ctl->nload; ++load2) {
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < blocks_per_load; q += blockDim.x) {
      const size_t blk = (size_t)load2 * blocks_per_load + q;
      a += __ldcg(&partials[2 * blk]);
      b += __ldcg(&partials[2 * blk + 1]);
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0 && !st[load2].done) advance_state(st[load2], ctl, hist, load2, a, b);
  }
  if (threadIdx.x == 0) {
    int all = 1;
    for (int l = 0; l < ctl->nload; ++l) all &= st[l].done;
    ctl->all_done = all;
    ctl->ticket = 0u;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------
// line pass along a non-contiguous axis `ax` of the half spectrum.
// MODE 0: forward FFT; MODE 1: inverse FFT; MODE 2 (ax = 0 only): forward,
// Green step, inverse.  Lines sit in shared memory with stride N + 1 (odd,
// against bank conflicts).
// ---------------------------------------------------------------------------
template <typename T, int NV, int MODE>
__global__ void __launch_bounds__(256, PassOcc<T>::value) line_pass(GridInfo g, DevPlan plan, const cplx<T>* __restrict__ tw,
                                                 cplx<T>* __restrict__ S, const T* __restrict__ Gt,
                                                 const LoadState* st, int ax, int W, int ntiles,
                                                 int n_outer, int n_inner) {
  constexpr int NTRI = NV * (NV + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int b = blockIdx.x;
  const int tile = b % ntiles; b /= ntiles;
  const int inner = b % n_inner; b /= n_inner;
  const int outer = b % n_outer; b /= n_outer;
  const int load = b;
  if (st[load].done) return;
  const int N = g.dims[ax];
  const int ls = N + 1;
  const int H = g.H;
  // element stride of axis ax inside one component's half spectrum
  long long stride = H;
  for (int k = ax + 1; k < g.nd - 1; ++k) stride *= g.dims[k];
  const long long base = (long long)outer * N * stride + (long long)inner * H;
  const int w0 = tile * W;
  const int nl = NV * W;
  cplx<T>* X0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* X1 = X0 + (size_t)nl * ls;
  const size_t comp_stride = (size_t)g.nhalf;
  cplx<T>* Sb = S + (size_t)load * NV * comp_stride + base + w0;
  const FDiv fW = make_fdiv(W), fN = make_fdiv(N);
  const int wlim = min(W, H - w0);
  // extents for the checked build: the launch's loads, one line buffer
  const long long sb0 = (long long)load * NV * comp_stride + base + w0;
  const long long nS = (long long)(gridDim.x / ((unsigned)ntiles * n_inner * n_outer)) * NV * g.nhalf;
  const long long nX = (long long)nl * ls;
  (void)sb0; (void)nS; (void)nX;

  {
    constexpr int U = 4;   // loads in flight per thread
    const int total = NV * N * W;
    for (int base0 = threadIdx.x; base0 < total; base0 += U * blockDim.x) {
      cplx<T> v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base0 + u * blockDim.x;
        v[u].x = v[u].y = T(0);
        if (idx < total) {
          const int t = fdiv(idx, fW);
          const int w = idx - t * W;
          const int c = fdiv(t, fN);
          const int n = t - c * N;
          if (w < wlim && FH_IN(CK_LINE_S, sb0 + c * comp_stride + n * stride + w, nS))
            v[u] = Sb[c * comp_stride + n * stride + w];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base0 + u * blockDim.x;
        if (idx < total) {
          const int t = fdiv(idx, fW);
          const int w = idx - t * W;
          const int c = fdiv(t, fN);
          const int n = t - c * N;
          if (FH_IN(CK_LINE_SMEM, (c * W + w) * ls + n, nX)) X0[(c * W + w) * ls + n] = v[u];
        }
      }
    }
  }
  __syncthreads();
  cplx<T>* X = X0;
  if (MODE == 0 || MODE == 2) X = fft_lines_pp<-1, T>(X0, X1, nl, ls, plan, tw);
  if (MODE == 2) {
    // Green step at frequency (l_0 = n, inner axes, l_last = w0 + w)
    for (int idx = threadIdx.x; idx < N * W; idx += blockDim.x) {
      const int n = fdiv(idx, fW);
      const int w = idx - n * W;
      if (w >= wlim) continue;
      const long long f = (long long)n * stride + (long long)inner * H + w0 + w;
      if (!FH_IN(CK_LINE_G, f + (long long)(NTRI - 1) * g.nhalf, (long long)NTRI * g.nhalf) ||
          !FH_IN(CK_LINE_SMEM, ((NV - 1) * W + w) * ls + n, nX))
        continue;
      cplx<T> tv[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) tv[c] = X[(c * W + w) * ls + n];
      T gm[NTRI];
#pragma unroll
      for (int t = 0; t < NTRI; ++t) gm[t] = Gt[(size_t)t * g.nhalf + f];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        T re = T(0), im = T(0);
#pragma unroll
        for (int bb = 0; bb < NV; ++bb) {
          const int lo = a < bb ? a : bb, hi = a < bb ? bb : a;
          const T gv = gm[lo * NV - (lo * (lo - 1)) / 2 + (hi - lo)];
          re -= gv * tv[bb].x;
          im -= gv * tv[bb].y;
        }
        cplx<T> e;
        e.x = (f == 0) ? T(0) : re;
        e.y = (f == 0) ? T(0) : im;
        X[(a * W + w) * ls + n] = e;
      }
    }
    __syncthreads();
  }
  if (MODE == 1 || MODE == 2) X = fft_lines_pp<+1, T>(X, X == X0 ? X1 : X0, nl, ls, plan, tw);
  for (int idx = threadIdx.x; idx < NV * N * W; idx += blockDim.x) {
    const int t = fdiv(idx, fW);
    const int w = idx - t * W;
    const int c = fdiv(t, fN);
    const int n = t - c * N;
    if (w < wlim && FH_IN(CK_LINE_S, sb0 + c * comp_stride + n * stride + w, nS) &&
        FH_IN(CK_LINE_SMEM, (c * W + w) * ls + n, nX))
      Sb[c * comp_stride + n * stride + w] = X[(c * W + w) * ls + n];
  }
}

// Green step alone, for 1-D grids (the row pass already transformed the only axis).
template <typename T>
__global__ void green_1d(GridInfo g, cplx<T>* __restrict__ S, const T* __restrict__ Gt, const LoadState* st,
                         int nload) {
  const long long total = (long long)nload * g.nhalf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int load = (int)(i / g.nhalf);
    const long long f = i - (long long)load * g.nhalf;
    if (st[load].done) continue;
    const int nv = g.nv;
    const size_t base = (size_t)load * nv * g.nhalf + f;
    if (!FH_IN(CK_GREEN1D, (long long)base + (long long)(nv - 1) * g.nhalf, (long long)nload * nv * g.nhalf)) continue;
    cplx<T> tv[MAXV];
    for (int c = 0; c < nv; ++c) tv[c] = S[base + c * g.nhalf];
    int t = 0;
    T Gm[MAXV][MAXV];
    for (int a = 0; a < nv; ++a)
      for (int bb = a; bb < nv; ++bb) { const T v = Gt[(size_t)t * g.nhalf + f]; Gm[a][bb] = v; Gm[bb][a] = v; ++t; }
    for (int a = 0; a < nv; ++a) {
      cplx<T> e;
      e.x = T(0); e.y = T(0);
      if (f != 0)
        for (int bb = 0; bb < nv; ++bb) { e.x -= Gm[a][bb] * tv[bb].x; e.y -= Gm[a][bb] * tv[bb].y; }
      S[base + a * g.nhalf] = e;
    }
  }
}

// ---------------------------------------------------------------------------
// mean stress <C:(E + eps0)> per load, FP64, fixed-order reduction.
// With at most four phases (and no point-by-point stiffness) C is constant on
// each phase, so the block sums E + eps0 over the points of every phase
// (additions only) and applies the phase matrices to those sums:
// sum_x C(x):(E(x) + eps0) = sum_p C_p : sum_{x in phase p} (E(x) + eps0).
// ---------------------------------------------------------------------------
constexpr int kMeanPhaseSums = 4;

template <typename T>
__global__ void __launch_bounds__(256) mean_stress(GridInfo g, const T* __restrict__ E,
                                                   const uint8_t* __restrict__ phase,
                                                   const double* __restrict__ Cp, Control* ctl,
                                                   double* __restrict__ partials, double* __restrict__ out,
                                                   int blocks_per_load, const double* __restrict__ Cfld = nullptr,
                                                   int nphase = 16) {
  __shared__ double red[32];
  __shared__ unsigned int s_ticket;
  const int load = blockIdx.x / blocks_per_load;
  const int q = blockIdx.x - load * blocks_per_load;
  const int nv = g.nv;
  double acc[MAXV] = {0, 0, 0, 0, 0, 0};
  double e0[MAXV];
  for (int c = 0; c < nv; ++c) e0[c] = ctl->eps0[load][c];
  const size_t Ebase = (size_t)load * nv * g.m;
  if (!Cfld && nphase <= kMeanPhaseSums) {
    // per thread: the sum of E over its points of each phase and the point
    // counts (eps0 enters through the counts).  Each phase's sum covers the
    // same points whatever label the phase carries, and the phases'
    // contributions are added last, so relabelling two phases (a stiffness
    // field reduced to its distinct matrices) gives the same bits.
    double sp[kMeanPhaseSums][MAXV];
    long long cnt[kMeanPhaseSums] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < MAXV; ++c)
#pragma unroll
      for (int p = 0; p < kMeanPhaseSums; ++p) sp[p][c] = 0.0;
    for (long long i = (long long)q * blockDim.x + threadIdx.x; i < g.m; i += (long long)blocks_per_load * blockDim.x) {
      if (!FH_IN(CK_MEAN, (long long)Ebase + (long long)(nv - 1) * g.m + i, (long long)ctl->nload * nv * g.m)) continue;
      const int ph = phase[i];
#pragma unroll
      for (int p = 0; p < kMeanPhaseSums; ++p) cnt[p] += (ph == p);
#pragma unroll
      for (int c = 0; c < MAXV; ++c) {
        if (c >= nv) break;
        const double e = (double)E[Ebase + (size_t)c * g.m + i];
        // the phase selects the addend, not the addition (FP64 additions are
        // the scarce resource here: one per phase and component)
#pragma unroll
        for (int p = 0; p < kMeanPhaseSums; ++p)
          if (p < nphase) sp[p][c] += (ph == p) ? e : 0.0;
      }
    }
    // block sums; thread 0 forms sum_p C_p : (sum over phase p of E + n_p eps0)
    double n[kMeanPhaseSums], S[kMeanPhaseSums][MAXV];
    for (int p = 0; p < nphase; ++p) {
      n[p] = block_sum((double)cnt[p], red);
      for (int c = 0; c < nv; ++c) S[p][c] = block_sum(sp[p][c], red);
    }
    if (threadIdx.x == 0) {
      for (int p = 0; p < nphase; ++p) {
        double v[MAXV];
        for (int a = 0; a < nv; ++a) {
          double t = 0.0;
          for (int c = 0; c < nv; ++c) t += Cp[((size_t)p * nv + a) * nv + c] * (S[p][c] + n[p] * e0[c]);
          v[a] = t;
        }
        for (int a = 0; a < nv; ++a) acc[a] += v[a];
      }
    }
  } else
  for (long long i = (long long)q * blockDim.x + threadIdx.x; i < g.m; i += (long long)blocks_per_load * blockDim.x) {
    double e[MAXV];
    if (!FH_IN(CK_MEAN, (long long)Ebase + (long long)(nv - 1) * g.m + i, (long long)ctl->nload * nv * g.m)) continue;
    if (!Cfld && !FH_IN(CK_MEAN, phase[i], 16)) continue;
    for (int c = 0; c < nv; ++c) e[c] = (double)E[Ebase + (size_t)c * g.m + i] + e0[c];
    if (Cfld) {   // point-by-point stiffness, upper triangle [tri][m]
      int t = 0;
      for (int a = 0; a < nv; ++a)
        for (int b = a; b < nv; ++b, ++t) {
          const double cab = Cfld[(size_t)t * g.m + i];
          acc[a] += cab * e[b];
          if (b != a) acc[b] += cab * e[a];
        }
    } else {
      const double* C = Cp + (size_t)phase[i] * nv * nv;
      for (int a = 0; a < nv; ++a) {
        double s = 0.0;
        for (int b = 0; b < nv; ++b) s += C[a * nv + b] * e[b];
        acc[a] += s;
      }
    }
  }
  for (int a = 0; a < nv; ++a) {
    const double v = block_sum(acc[a], red);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * MAXV + a] = v;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_ticket = atomicAdd(&ctl->ticket2, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  for (int l = 0; l < ctl->nload; ++l)
    for (int a = 0; a < nv; ++a) {
      double s = 0.0;
      for (int qq = threadIdx.x; qq < blocks_per_load; qq += blockDim.x)
        s += __ldcg(&partials[((size_t)l * blocks_per_load + qq) * MAXV + a]);
      s = block_sum(s, red);
      if (threadIdx.x == 0) out[l * MAXV + a] = s * g.inv_m;
    }
  if (threadIdx.x == 0) ctl->ticket2 = 0u;
}

// ---------------------------------------------------------------------------
// Gamma^p table (Def. gamma_tilde_fourier), FP64, one thread per stored
// frequency of the half spectrum.
// ---------------------------------------------------------------------------
struct GreenParams {
  int d, nv, ntri, nd;
  int dims[3];
  int H;
  long long nhalf;
  long long D;
  int sign;
  long long M[3][3];
  long long adjT[3][3];
  long long Fmap[3][3];
  int kind;
  double alpha[3];
  int n_xi;
  double xi[3 * 16];
  int radius;
  double C4[81];  // C0_ijkl, index ((i*3 + j)*3 + k)*3 + l
  // closed-form path (green_table_iso): C0 isotropic with Lame constants
  // lam0, mu0, and a symbol that is a product of per-axis factors; for a box
  // spline whose directions are all +-e_i, xcount[i] is how often e_i occurs
  double lam0, mu0;
  int xcount[3];
};

__device__ __forceinline__ long long floordiv_ll(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// symbol g at u = unum / D  (see fh_generator)
__device__ double gen_symbol(const GreenParams& P, const long long* unum) {
  double g = 1.0;
  if (P.kind == FH_GEN_BOXSPLINE) {
    for (int s = 0; s < P.n_xi; ++s) {
      double t = 0.0;
      for (int i = 0; i < P.d; ++i) t += P.xi[3 * s + i] * ((double)unum[i] / (double)P.D);
      double f;
      if (t == 0.0) f = 1.0;
      else if (t == rint(t)) f = 0.0;
      else f = sinpi(t) / (3.14159265358979323846 * t);
      g *= f;
    }
    return g;
  }
  for (int i = 0; i < P.d; ++i) {
    const long long two = unum[i] < 0 ? -2 * unum[i] : 2 * unum[i];
    const double a = (P.kind == FH_GEN_DLVP) ? P.alpha[i] : 0.0;
    double gi;
    if (a == 0.0) gi = two < P.D ? 1.0 : (two == P.D ? 0.5 : 0.0);
    else {
      const double u = fabs((double)unum[i] / (double)P.D);
      gi = fmin(1.0, fmax(0.0, (0.5 + a - u) / (2.0 * a)));
    }
    g *= gi;
  }
  return g;
}

__device__ void mandel_pair(int d, int a, int& i, int& j) {
  if (d == 2) {
    const int I[3] = {0, 1, 0}, J[3] = {0, 1, 1};
    i = I[a]; j = J[a];
  } else {
    const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
    i = I[a]; j = J[a];
  }
}

// storage frequency f -> h = V^-T l, reduced into G(M^T), and the numerators
// u = D M^-T h of the reduced frequency (|u_i| <= D/2)
__device__ __forceinline__ void reduce_frequency(const GreenParams& P, long long f, long long* h, long long* u) {
  const int d = P.d;
  long long l[3] = {0, 0, 0};
  long long rem = f;
  l[P.nd - 1] = rem % P.H;
  rem /= P.H;
  for (int k = P.nd - 2; k >= 0; --k) { l[k] = rem % P.dims[k]; rem /= P.dims[k]; }
  for (int i = 0; i < 3; ++i) h[i] = u[i] = 0;
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < P.nd; ++k) h[i] += l[k] * P.Fmap[k][i];
  for (int i = 0; i < d; ++i) {
    long long s = 0;
    for (int c = 0; c < d; ++c) s += P.adjT[i][c] * h[c];
    u[i] = P.sign * s;
  }
  long long z0[3];
  for (int i = 0; i < d; ++i) z0[i] = floordiv_ll(2 * u[i] + P.D, 2 * P.D);
  for (int i = 0; i < d; ++i) {
    for (int c = 0; c < d; ++c) h[i] -= P.M[c][i] * z0[c];
    u[i] -= P.D * z0[i];
  }
}

__global__ void green_table(GreenParams P, double* __restrict__ G64, float* __restrict__ G32, int* err) {
  const long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (f >= P.nhalf) return;
  const int d = P.d;
  // storage frequency l -> h = V^-T l, reduced into G(M^T)
  long long l[3] = {0, 0, 0};
  long long rem = f;
  l[P.nd - 1] = rem % P.H;
  rem /= P.H;
  for (int k = P.nd - 2; k >= 0; --k) { l[k] = rem % P.dims[k]; rem /= P.dims[k]; }
  long long h[3] = {0, 0, 0}, u[3] = {0, 0, 0};
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < P.nd; ++k) h[i] += l[k] * P.Fmap[k][i];
  for (int i = 0; i < d; ++i) {
    long long s = 0;
    for (int c = 0; c < d; ++c) s += P.adjT[i][c] * h[c];
    u[i] = P.sign * s;
  }
  long long z0[3];
  for (int i = 0; i < d; ++i) z0[i] = floordiv_ll(2 * u[i] + P.D, 2 * P.D);
  for (int i = 0; i < d; ++i) {
    for (int c = 0; c < d; ++c) h[i] -= P.M[c][i] * z0[c];
    u[i] -= P.D * z0[i];
  }
  // aliases k = h + M^T z with |u_i + z_i| <= R + 1/2: z_i in {-R..R+1}, the
  // last one only where u_i = -1/2 (a cube symmetric in M^-T k, so that
  // Gamma^p_{-h} = Gamma^p_h).  Dirichlet and dlVP symbols vanish beyond
  // |u_i| = 1, so R = 1 covers them exactly.
  const int R = (P.kind == FH_GEN_BOXSPLINE) ? P.radius : 1;
  const int span = 2 * R + 2;
  int nal = 1;
  for (int i = 0; i < d; ++i) nal *= span;
  const double s2 = 1.41421356237309504880;
  double acc[21];
  for (int t = 0; t < P.ntri; ++t) acc[t] = 0.0;
  double wsum = 0.0;
  for (int ai = 0; ai < nal; ++ai) {
    long long z[3] = {0, 0, 0};
    int q = ai;
    for (int i = 0; i < d; ++i) { z[i] = (q % span) - R; q /= span; }
    long long un[3];
    bool inside = true;
    for (int i = 0; i < d; ++i) {
      un[i] = u[i] + P.D * z[i];
      const long long t = un[i] < 0 ? -2 * un[i] : 2 * un[i];
      inside = inside && t <= (2 * R + 1) * P.D;
    }
    if (!inside) continue;
    const double gv = gen_symbol(P, un);
    if (gv == 0.0) continue;
    const double w = gv * gv;
    wsum += w;
    double k[3] = {0, 0, 0};
    bool nonzero = false;
    for (int i = 0; i < d; ++i) {
      long long s = h[i];
      for (int c = 0; c < d; ++c) s += P.M[c][i] * z[c];
      k[i] = (double)s;
      nonzero = nonzero || (s != 0);
    }
    if (!nonzero) continue;  // Gamma^0(0) = 0
    // acoustic tensor K_ik = C0_ijkl k_j k_l and its inverse N
    double K[3][3];
    for (int i = 0; i < d; ++i)
      for (int kk = 0; kk < d; ++kk) {
        double s = 0.0;
        for (int j = 0; j < d; ++j)
          for (int ll = 0; ll < d; ++ll) s += P.C4[((i * 3 + j) * 3 + kk) * 3 + ll] * k[j] * k[ll];
        K[i][kk] = s;
      }
    double N[3][3];
    if (d == 2) {
      const double det = K[0][0] * K[1][1] - K[0][1] * K[1][0];
      N[0][0] = K[1][1] / det; N[0][1] = -K[0][1] / det;
      N[1][0] = -K[1][0] / det; N[1][1] = K[0][0] / det;
    } else {
      const double c00 = K[1][1] * K[2][2] - K[1][2] * K[2][1];
      const double c01 = K[1][2] * K[2][0] - K[1][0] * K[2][2];
      const double c02 = K[1][0] * K[2][1] - K[1][1] * K[2][0];
      const double det = K[0][0] * c00 + K[0][1] * c01 + K[0][2] * c02;
      N[0][0] = c00 / det;
      N[1][0] = c01 / det;
      N[2][0] = c02 / det;
      N[0][1] = (K[0][2] * K[2][1] - K[0][1] * K[2][2]) / det;
      N[1][1] = (K[0][0] * K[2][2] - K[0][2] * K[2][0]) / det;
      N[2][1] = (K[0][1] * K[2][0] - K[0][0] * K[2][1]) / det;
      N[0][2] = (K[0][1] * K[1][2] - K[0][2] * K[1][1]) / det;
      N[1][2] = (K[0][2] * K[1][0] - K[0][0] * K[1][2]) / det;
      N[2][2] = (K[0][0] * K[1][1] - K[0][1] * K[1][0]) / det;
    }
    // Gamma^0 Mandel entry (a, b): s_a s_b / 4 (k_i N_jp k_q + k_i N_jq k_p + k_j N_ip k_q + k_j N_iq k_p)
    int t = 0;
    for (int a = 0; a < P.nv; ++a) {
      int i, j;
      mandel_pair(d, a, i, j);
      const double sa = (i == j) ? 1.0 : s2;
      for (int bb = a; bb < P.nv; ++bb) {
        int p, qq;
        mandel_pair(d, bb, p, qq);
        const double sb = (p == qq) ? 1.0 : s2;
        const double v = 0.25 * sa * sb *
                         (k[i] * N[j][p] * k[qq] + k[i] * N[j][qq] * k[p] + k[j] * N[i][p] * k[qq] + k[j] * N[i][qq] * k[p]);
        acc[t++] += w * v;
      }
    }
  }
  if (!(wsum > 0.0)) {
    atomicExch(err, (int)FH_ERR_NO_ONB);
    wsum = 1.0;
  }
  for (int t = 0; t < P.ntri; ++t) {
    const double v = acc[t] / wsum;
    if (!FH_IN(CK_TABLE, (long long)t * P.nhalf + f, (long long)P.ntri * P.nhalf)) continue;
    G64[(size_t)t * P.nhalf + f] = v;
    G32[(size_t)t * P.nhalf + f] = (float)v;
  }
}

// ---------------------------------------------------------------------------
// Gamma^p table, closed form for an isotropic C0 and a separable symbol.
//
// For isotropic C0 (Lame constants lam0, mu0) Gamma^0 has the closed form of
// Moulinec & Suquet (1998); with n = k/|k|,
//   Gamma^0_ijpq(k) = (d_ip n_j n_q + d_iq n_j n_p + d_jp n_i n_q + d_jq n_i n_p) / (4 mu0)
//                     - (lam0 + mu0) / (mu0 (lam0 + 2 mu0)) n_i n_j n_p n_q,
// so the alias sum of Def. gamma_tilde_fourier, Gamma^p_h = sum_z w_z Gamma^0(h + M^T z),
// needs only the fourth moment B_ijpq = sum_z w_z n_i n_j n_p n_q (15 numbers in
// 3-D, 5 in 2-D); the second moment follows from it, sum_z w_z n_i n_j = sum_p B_ijpp.
// When the symbol is a product of per-axis factors g(u) = prod_i g_i(u_i)
// (Dirichlet, dlVP, box splines whose directions are unit vectors) and the
// alias set is the product of per-axis sets |u_i + z_i| <= R + 1/2, the
// orthonormalised weights (Lemma FI:Props (iii)) factor too:
//   w_z = prod_i g_i(u_i + z_i)^2 / sum_{z_i'} g_i(u_i + z_i')^2,
// so they cost a few symbol evaluations per axis instead of one per alias, and
// aliases of zero weight are skipped.  One thread per stored frequency, aliases
// in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int kMaxAxisAliases = 34;  // 2R + 2 per axis, R <= 16

// per-axis factor g_i at u_i = un / D
__device__ __forceinline__ double axis_symbol(const GreenParams& P, int i, long long un) {
  if (P.kind == FH_GEN_BOXSPLINE) {
    const int c = P.xcount[i];
    if (c == 0) return 1.0;
    double f;
    if (un == 0) f = 1.0;
    else if (un % P.D == 0) f = 0.0;  // sinc vanishes at the nonzero integers
    else {
      const double v = (double)un / (double)P.D;
      f = sinpi(v) / (3.14159265358979323846 * v);
    }
    double g = 1.0;
    for (int e = 0; e < c; ++e) g *= f;
    return g;
  }
  const long long two = un < 0 ? -2 * un : 2 * un;
  const double a = (P.kind == FH_GEN_DLVP) ? P.alpha[i] : 0.0;
  if (a == 0.0) return two < P.D ? 1.0 : (two == P.D ? 0.5 : 0.0);
  const double u = fabs((double)un / (double)P.D);
  return fmin(1.0, fmax(0.0, (0.5 + a - u) / (2.0 * a)));
}

// index of the fourth moment with exponents (e0, e1, e2) of n_0, n_1, n_2 in
// the accumulation order of green_table_iso<3>
__device__ __forceinline__ int moment_index3(int e1, int e2) {
  // rows e1 = 0..4, columns e2 = 0..4 (e0 = 4 - e1 - e2)
  const signed char T[5][5] = {{0, 2, 5, 12, 14}, {1, 4, 8, 13, -1}, {3, 7, 11, -1, -1},
                               {6, 10, -1, -1, -1}, {9, -1, -1, -1, -1}};
  return T[e1][e2];
}

// Gamma^p entries of one storage frequency f (coordinates l0, l1, l2 when
// mirroring) from its moments Bm, written to f and, when mirroring, to its
// mirror images.
//
// mirror: M diagonal and the Smith grid's axes are M's axes (Fmap a signed
// permutation, mirror_geo[k] = the geometric axis of storage axis k).  The
// symbols are even per axis and the alias sets mirror with u_i -> -u_i, so
// reflecting h_g -> -h_g multiplies the Mandel entry of (i,j),(p,q) by
// (-1)^(how often g occurs among i, j, p, q).  Threads then cover only the
// storage frequencies with l_k <= dims_k / 2 on the full (non-half) axes and
// write every mirror image: 1/2 (2-D) or 1/4 (3-D) of the alias sums.
template <int DIM>
__device__ void iso_emit(const GreenParams& P, const double* Bm, long long f, long long l0, long long l1, long long l2,
                         int mirror, int mirror_geo0, int mirror_geo1, double* __restrict__ G64,
                         float* __restrict__ G32) {
  auto moment = [&](int i, int j, int p, int q) -> double {
    int e[3] = {0, 0, 0};
    ++e[i]; ++e[j]; ++e[p]; ++e[q];
    if (DIM == 2) return Bm[e[1]];
    return Bm[moment_index3(e[1], e[2])];
  };
  // second moment A_ij = sum_p B_ijpp
  double A[3][3];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      double s = 0.0;
      for (int p = 0; p < DIM; ++p) s += moment(i, j, p, p);
      A[i][j] = s;
    }
  const double c4 = 0.25 / P.mu0;
  const double cb = (P.lam0 + P.mu0) / (P.mu0 * (P.lam0 + 2.0 * P.mu0));
  const double s2 = 1.41421356237309504880;
  // mirror images (s0, s1) of the storage frequency; (0, 0) is f itself
  long long fm[4];
  fm[0] = f;
  fm[1] = fm[2] = fm[3] = -1;
  if (mirror) {
    const long long m0 = (P.dims[0] - l0) % P.dims[0];
    const long long m1 = DIM == 3 ? (P.dims[1] - l1) % P.dims[1] : 0;
    const bool d0 = m0 != l0, d1 = DIM == 3 && m1 != l1;
    if (DIM == 3) {
      if (d0) fm[1] = (m0 * P.dims[1] + l1) * P.H + l2;
      if (d1) fm[2] = (l0 * P.dims[1] + m1) * P.H + l2;
      if (d0 && d1) fm[3] = (m0 * P.dims[1] + m1) * P.H + l2;
    } else if (d0) {
      fm[1] = m0 * P.H + l2;
    }
  }
  int t = 0;
  for (int a = 0; a < P.nv; ++a) {
    int i, j;
    mandel_pair(DIM, a, i, j);
    const double sa = (i == j) ? 1.0 : s2;
    for (int b = a; b < P.nv; ++b) {
      int p, q;
      mandel_pair(DIM, b, p, q);
      const double sb = (p == q) ? 1.0 : s2;
      const double lin = (i == p ? A[j][q] : 0.0) + (i == q ? A[j][p] : 0.0) + (j == p ? A[i][q] : 0.0) +
                         (j == q ? A[i][p] : 0.0);
      const double v = sa * sb * (c4 * lin - cb * moment(i, j, p, q));
      const int c0 = (i == mirror_geo0) + (j == mirror_geo0) + (p == mirror_geo0) + (q == mirror_geo0);
      const int c1 = (i == mirror_geo1) + (j == mirror_geo1) + (p == mirror_geo1) + (q == mirror_geo1);
      for (int r = 0; r < 4; ++r) {
        if (fm[r] < 0) continue;
        const int flips = ((r & 1) ? c0 : 0) + ((r & 2) ? c1 : 0);
        const double vr = (flips & 1) ? -v : v;
        if (!FH_IN(CK_TABLE, (long long)t * P.nhalf + fm[r], (long long)P.ntri * P.nhalf)) continue;
        G64[(size_t)t * P.nhalf + fm[r]] = vr;
        G32[(size_t)t * P.nhalf + fm[r]] = (float)vr;
      }
      ++t;
    }
  }
}

// exponents (e1, e2) of moment t in the accumulation order of green_table_iso<3>
// (inverse of moment_index3; e0 = 4 - e1 - e2)
__device__ __forceinline__ void moment_exponents3(int t, int& e1, int& e2) {
  const signed char E1[15] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 4, 3, 2, 0, 1, 0};
  const signed char E2[15] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 0, 1, 2, 3, 3, 4};
  e1 = E1[t];
  e2 = E2[t];
}

// cubic: in addition to the mirror conditions, the three storage axes have the
// same length N, |M_00| = |M_11| = |M_22| and the per-axis symbols are the same
// function (Dirichlet, dlVP with equal ramps, a box spline with the same count
// of each e_i).  Permuting the geometric axes then maps the alias set and the
// weights onto themselves, so the moments at a permuted frequency are the
// moments at the original one with their exponents permuted:
//   sum_z w_z n'^e = sum_z w_z prod_g n_{pi(g)}^{e_g}   when |h'_g| = |h_{pi(g)}|.
// Threads take the storage frequencies with N/2 >= l0 >= l1 >= l2 >= 0 (thread
// index -> the triple by tetrahedral numbers), sum the aliases once, and write
// every distinct permutation of (l0, l1, l2) with its mirror images: 1/6 of the
// alias sums of the mirror path.  Signs go through |h|: the moments at the
// reduced frequency h carry prod_g sign(h_g)^(e_g) relative to those at |h|
// (the alias sets of the reduced u are symmetric).
__device__ __forceinline__ long long tet3(long long a) { return a * (a + 1) * (a + 2) / 6; }

__device__ __forceinline__ void cubic_triple(long long idx, long long& L0, long long& L1, long long& L2) {
  long long a = (long long)cbrt(6.0 * (double)idx);
  while (tet3(a + 1) <= idx) ++a;
  while (a > 0 && tet3(a) > idx) --a;
  const long long r = idx - tet3(a);
  long long b = (long long)((sqrt(8.0 * (double)r + 1.0) - 1.0) * 0.5);
  while ((b + 1) * (b + 2) / 2 <= r) ++b;
  while (b > 0 && b * (b + 1) / 2 > r) --b;
  L0 = a;
  L1 = b;
  L2 = r - b * (b + 1) / 2;
}

template <int DIM>
__global__ void __launch_bounds__(128) green_table_iso(GreenParams P, double* __restrict__ G64,
                                                       float* __restrict__ G32, int* err, int mirror,
                                                       int mirror_geo0, int mirror_geo1, int cubic) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long f = idx;
  long long l0 = 0, l1 = 0, l2 = 0;  // storage coordinates when mirroring
  if (DIM == 3 && cubic) {
    const long long n = P.dims[0] / 2 + 1;
    if (idx >= tet3(n)) return;
    cubic_triple(idx, l0, l1, l2);
    f = (l0 * P.dims[1] + l1) * P.H + l2;
  } else if (mirror) {
    const long long n0 = P.dims[0] / 2 + 1, n1 = DIM == 3 ? P.dims[1] / 2 + 1 : 1;
    if (idx >= n0 * n1 * P.H) return;
    l2 = idx % P.H;
    const long long t = idx / P.H;
    l1 = DIM == 3 ? t % n1 : 0;
    l0 = DIM == 3 ? t / n1 : t;
    f = DIM == 3 ? (l0 * P.dims[1] + l1) * P.H + l2 : l0 * P.H + l2;
  } else if (f >= P.nhalf) {
    return;
  }
  long long h[3], u[3];
  reduce_frequency(P, f, h, u);
  const int R = (P.kind == FH_GEN_BOXSPLINE) ? P.radius : 1;
  int nal[DIM];
  int zl[DIM][kMaxAxisAliases];
  double wl[DIM][kMaxAxisAliases];
  bool onb = true;
  for (int i = 0; i < DIM; ++i) {
    double sum = 0.0;
    int n = 0;
    for (int z = -R; z <= R + 1; ++z) {
      const long long un = u[i] + P.D * z;
      const long long t = un < 0 ? -2 * un : 2 * un;
      if (t > (2 * R + 1) * P.D) continue;
      const double g = axis_symbol(P, i, un);
      if (g == 0.0) continue;
      zl[i][n] = z;
      wl[i][n] = g * g;
      sum += g * g;
      ++n;
    }
    if (!(sum > 0.0)) onb = false;
    for (int q = 0; q < n; ++q) wl[i][q] /= sum;
    nal[i] = n;
  }
  constexpr int NB = DIM == 2 ? 5 : 15;
  double B[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) B[t] = 0.0;
  if (!onb) {
    atomicExch(err, (int)FH_ERR_NO_ONB);
  } else if (DIM == 2) {
    for (int a = 0; a < nal[0]; ++a) {
      const double za = (double)zl[0][a], wa = wl[0][a];
      const double ka0 = (double)h[0] + (double)P.M[0][0] * za, ka1 = (double)h[1] + (double)P.M[0][1] * za;
      const double m0 = (double)P.M[1][0], m1 = (double)P.M[1][1];
      for (int b = 0; b < nal[1]; ++b) {
        const double zb = (double)zl[1][b];
        const double k0 = fma(m0, zb, ka0), k1 = fma(m1, zb, ka1);  // integers: exact
        const double p00 = k0 * k0, p11 = k1 * k1, p01 = k0 * k1;
        const double r2 = p00 + p11;
        if (r2 == 0.0) continue;  // Gamma^0(0) = 0
        const double inv = __drcp_rn(r2);
        const double q = wa * wl[1][b] * inv * inv;
        const double q00 = q * p00, q01 = q * p01, q11 = q * p11;
        B[0] = fma(q00, p00, B[0]);  // n0^4
        B[1] = fma(q00, p01, B[1]);  // n0^3 n1
        B[2] = fma(q00, p11, B[2]);  // n0^2 n1^2
        B[3] = fma(q01, p11, B[3]);  // n0 n1^3
        B[4] = fma(q11, p11, B[4]);  // n1^4
      }
    }
  } else {
    for (int a = 0; a < nal[0]; ++a) {
      const double za = (double)zl[0][a], wa = wl[0][a];
      double ka[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) ka[i] = (double)h[i] + (double)P.M[0][i] * za;
      for (int b = 0; b < nal[1]; ++b) {
        const double zb = (double)zl[1][b], wab = wa * wl[1][b];
        double kb[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) kb[i] = fma((double)P.M[1][i], zb, ka[i]);
        const double m0 = (double)P.M[2][0], m1 = (double)P.M[2][1], m2 = (double)P.M[2][2];
        for (int c = 0; c < nal[2]; ++c) {
          const double zc = (double)zl[2][c];
          const double k0 = fma(m0, zc, kb[0]), k1 = fma(m1, zc, kb[1]), k2 = fma(m2, zc, kb[2]);
          const double p00 = k0 * k0, p11 = k1 * k1, p22 = k2 * k2;
          const double r2 = p00 + p11 + p22;
          if (r2 == 0.0) continue;  // Gamma^0(0) = 0
          const double p01 = k0 * k1, p02 = k0 * k2, p12 = k1 * k2;
          const double inv = __drcp_rn(r2);
          const double q = wab * wl[2][c] * inv * inv;
          const double q00 = q * p00, q01 = q * p01, q02 = q * p02, q11 = q * p11, q12 = q * p12, q22 = q * p22;
          B[0] = fma(q00, p00, B[0]);    // (4,0,0)
          B[1] = fma(q00, p01, B[1]);    // (3,1,0)
          B[2] = fma(q00, p02, B[2]);    // (3,0,1)
          B[3] = fma(q00, p11, B[3]);    // (2,2,0)
          B[4] = fma(q00, p12, B[4]);    // (2,1,1)
          B[5] = fma(q00, p22, B[5]);    // (2,0,2)
          B[6] = fma(q01, p11, B[6]);    // (1,3,0)
          B[7] = fma(q01, p12, B[7]);    // (1,2,1)
          B[8] = fma(q01, p22, B[8]);    // (1,1,2)
          B[9] = fma(q11, p11, B[9]);    // (0,4,0)
          B[10] = fma(q11, p12, B[10]);  // (0,3,1)
          B[11] = fma(q11, p22, B[11]);  // (0,2,2)
          B[12] = fma(q02, p22, B[12]);  // (1,0,3)
          B[13] = fma(q12, p22, B[13]);  // (0,1,3)
          B[14] = fma(q22, p22, B[14]);  // (0,0,4)
        }
      }
    }
  }
  // fourth moment B_ijpq by exponents (a copy is indexed at run time, so that
  // B itself stays in registers in the loops)
  double Bm[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) Bm[t] = B[t];
  if constexpr (DIM == 2) {
    iso_emit<DIM>(P, Bm, f, l0, l1, l2, mirror, mirror_geo0, mirror_geo1, G64, G32);
  } else {
  if (!cubic) {
    iso_emit<DIM>(P, Bm, f, l0, l1, l2, mirror, mirror_geo0, mirror_geo1, G64, G32);
    return;
  }
  // every distinct permutation (l0', l1', l2') of the storage triple
  const long long L[3] = {l0, l1, l2};
  const signed char PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  long long seen[6][3];
  int nseen = 0;
  for (int pi = 0; pi < 6; ++pi) {
    const long long lp[3] = {L[PERM[pi][0]], L[PERM[pi][1]], L[PERM[pi][2]]};
    bool dup = false;
    for (int q = 0; q < nseen; ++q)
      dup = dup || (seen[q][0] == lp[0] && seen[q][1] == lp[1] && seen[q][2] == lp[2]);
    if (dup) continue;
    seen[nseen][0] = lp[0];
    seen[nseen][1] = lp[1];
    seen[nseen][2] = lp[2];
    ++nseen;
    const long long fp = (lp[0] * P.dims[1] + lp[1]) * P.H + lp[2];
    long long hp[3], up[3];
    reduce_frequency(P, fp, hp, up);
    // geometric axis map: |h'_g| = |h_{ax[g]}|
    int ax[3] = {-1, -1, -1};
    bool used[3] = {false, false, false};
    for (int g = 0; g < 3; ++g) {
      const long long want = hp[g] < 0 ? -hp[g] : hp[g];
      for (int g2 = 0; g2 < 3 && ax[g] < 0; ++g2) {
        const long long have = h[g2] < 0 ? -h[g2] : h[g2];
        if (!used[g2] && have == want) { ax[g] = g2; used[g2] = true; }
      }
    }
    if (ax[0] < 0 || ax[1] < 0 || ax[2] < 0) {  // cannot happen when the cubic conditions hold
      atomicExch(err, (int)FH_ERR_INTERNAL);
      return;
    }
    double Bp[NB];
    for (int t = 0; t < NB; ++t) {
      int e[3];
      moment_exponents3(t, e[1], e[2]);
      e[0] = 4 - e[1] - e[2];
      int src[3] = {0, 0, 0};
      for (int g = 0; g < 3; ++g) src[ax[g]] = e[g];
      int par = 0;
      for (int g = 0; g < 3; ++g) par += (h[g] < 0 ? src[g] : 0) + (hp[g] < 0 ? e[g] : 0);
      const double v = Bm[moment_index3(src[1], src[2])];
      Bp[t] = (par & 1) ? -v : v;
    }
    iso_emit<DIM>(P, Bp, fp, lp[0], lp[1], lp[2], mirror, mirror_geo0, mirror_geo1, G64, G32);
  }
  }
}

// Point-by-point stiffness after the reference medium is known: from C(x)
// (upper triangle [tri][m], FP64) the differences C(x) - C0 in FP64 and FP32
// and C(x) in FP32 (variational form), same layout
struct Tri21 {
  double v[21];
};
__global__ void field_prepare(const double* __restrict__ C, Tri21 c0, int ntri, long long m,
                              double* __restrict__ dC64, float* __restrict__ dC32, float* __restrict__ C32) {
  const long long n = (long long)ntri * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / m);
    const double d = C[i] - c0.v[t];
    dC64[i] = d;
    dC32[i] = (float)d;
    C32[i] = (float)C[i];
  }
}

// phase ids must index the phase table
__global__ void check_phases(const uint8_t* __restrict__ phase, long long m, int nphase, int* err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    if (phase[i] >= nphase) atomicExch(err, (int)FH_ERR_ARG);
}

template <typename TO, typename TI>
__global__ void convert_copy(TO* __restrict__ out, const TI* __restrict__ in, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

}  // namespace fh
