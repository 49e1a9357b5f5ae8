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
};

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
  int pad;
};

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

// Advance the per-load state after one iteration's residual is known.
__device__ void advance_state(LoadState& s, Control* ctl, double* hist, int load, double d2, double n2) {
  const double r = (n2 > 0.0) ? sqrt(d2 / n2) : sqrt(d2);
  s.iter += 1;
  if (s.iter <= ctl->hist_cap) hist[(size_t)load * ctl->hist_cap + (s.iter - 1)] = r;
  if (s.iter == 1) s.r_first = r;
  s.inc = (s.iter > 1 && r > s.r) ? s.inc + 1 : 0;
  s.r = r;
  if (!isfinite(r)) { s.status = FH_NONFINITE; s.done = 1; }
  else if (r <= ctl->tol) { s.status = FH_OK; s.done = 1; }
  else if (s.inc >= 100 || (s.iter > 10 && r > 1e6 * s.r_first && r > 1.0)) { s.status = FH_DIVERGED; s.done = 1; }
  else if (s.iter >= ctl->max_iter) { s.status = FH_NOT_CONVERGED; s.done = 1; }
}

// ---------------------------------------------------------------------------
// row pass along the contiguous axis (length L), fused with the pointwise
// constitutive stage and the residual.
// ---------------------------------------------------------------------------
template <typename T, bool FIRST>
__global__ void __launch_bounds__(256) row_pass(GridInfo g, DevPlan plan, const cplx<T>* __restrict__ tw,
                                                T* __restrict__ E, cplx<T>* __restrict__ S,
                                                const uint8_t* __restrict__ phase, const T* __restrict__ dC,
                                                Control* ctl, LoadState* st, double* __restrict__ partials,
                                                double* __restrict__ hist, int rpb, int blocks_per_load) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int s_skip;
  const int load = blockIdx.x / blocks_per_load;
  const int rb = blockIdx.x - load * blocks_per_load;
  const long long row0 = (long long)rb * rpb;
  const int nrow = (int)min((long long)rpb, g.nrows - row0);
  const int L = g.L, H = g.H, nv = g.nv;
  const int nreal = nrow * nv;
  const int npair = (nreal + 1) >> 1;
  cplx<T>* Z = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tmp = Z + (size_t)((rpb * nv + 1) >> 1) * L;

  if (threadIdx.x == 0) s_skip = st[load].done;
  __syncthreads();
  double d2 = 0.0, n2 = 0.0;
  if (!s_skip) {
    T e0[MAXV];
    for (int c = 0; c < nv; ++c) e0[c] = (T)ctl->eps0[load][c];
    const size_t Ebase = (size_t)load * nv * g.m;
    const size_t Sbase = (size_t)load * nv * g.nrows * H;
    if (!FIRST) {
      // 1. rebuild the two-real-lines-in-one complex spectrum Z = A + i B
      for (int idx = threadIdx.x; idx < npair * L; idx += blockDim.x) {
        const int p = idx / L, k = idx - p * L;
        const int fa = 2 * p, fb = 2 * p + 1;
        const int kk = k <= L / 2 ? k : L - k;
        const T sg = k <= L / 2 ? T(1) : T(-1);  // conjugate for k > L/2
        const int ra = fa / nv, ca = fa - ra * nv;
        cplx<T> A = S[Sbase + ((size_t)ca * g.nrows + row0 + ra) * H + kk];
        cplx<T> B;
        B.x = T(0); B.y = T(0);
        if (fb < nreal) {
          const int rbb = fb / nv, cb = fb - rbb * nv;
          B = S[Sbase + ((size_t)cb * g.nrows + row0 + rbb) * H + kk];
        }
        A.y *= sg;
        B.y *= sg;
        cplx<T> z;
        z.x = A.x - B.y;
        z.y = A.y + B.x;
        Z[(size_t)p * L + k] = z;
      }
      __syncthreads();
      // 2. inverse FFT (unnormalised)
      fft_lines<+1, T>(Z, tmp, npair, L, plan, tw);
    }
    // 3. pointwise: E_new, residual sums, tau = (C - C0):(E_new + eps0)
    const T scale = (T)g.inv_m;
    for (int idx = threadIdx.x; idx < nrow * L; idx += blockDim.x) {
      const int r = idx / L, x = idx - r * L;
      const size_t gi = (size_t)(row0 + r) * L + x;
      T en[MAXV];
      for (int c = 0; c < nv; ++c) {
        const int f = r * nv + c;
        if (FIRST) {
          en[c] = E[Ebase + (size_t)c * g.m + gi];
        } else {
          const cplx<T> zz = Z[(size_t)(f >> 1) * L + x];
          en[c] = ((f & 1) ? zz.y : zz.x) * scale;
          const T eo = E[Ebase + (size_t)c * g.m + gi];
          const double df = (double)en[c] - (double)eo;
          const double tf = (double)en[c] + (double)e0[c];
          d2 += df * df;
          n2 += tf * tf;
          E[Ebase + (size_t)c * g.m + gi] = en[c];
        }
      }
      const T* dc = dC + (size_t)phase[gi] * nv * nv;
      for (int a = 0; a < nv; ++a) {
        T t = T(0);
        for (int b = 0; b < nv; ++b) t += dc[a * nv + b] * (en[b] + e0[b]);
        const int f = r * nv + a;
        if (f & 1) Z[(size_t)(f >> 1) * L + x].y = t;
        else Z[(size_t)(f >> 1) * L + x].x = t;
      }
    }
    // odd number of real lines: the last pair's imaginary part is zero
    if (nreal & 1) {
      for (int x = threadIdx.x; x < L; x += blockDim.x) Z[(size_t)(npair - 1) * L + x].y = T(0);
    }
    __syncthreads();
    // 4. forward FFT
    fft_lines<-1, T>(Z, tmp, npair, L, plan, tw);
    // 5. split into the two half spectra A = (Z_k + conj Z_{L-k})/2, B = (Z_k - conj Z_{L-k})/(2i)
    for (int idx = threadIdx.x; idx < npair * H; idx += blockDim.x) {
      const int p = idx / H, k = idx - p * H;
      const cplx<T> zk = Z[(size_t)p * L + k];
      const cplx<T> zm = Z[(size_t)p * L + (k == 0 ? 0 : L - k)];
      cplx<T> A, B;
      A.x = T(0.5) * (zk.x + zm.x);
      A.y = T(0.5) * (zk.y - zm.y);
      B.x = T(0.5) * (zk.y + zm.y);
      B.y = T(-0.5) * (zk.x - zm.x);
      const int fa = 2 * p, fb = 2 * p + 1;
      const int ra = fa / nv, ca = fa - ra * nv;
      S[Sbase + ((size_t)ca * g.nrows + row0 + ra) * H + k] = A;
      if (fb < nreal) {
        const int rbb = fb / nv, cb = fb - rbb * nv;
        S[Sbase + ((size_t)cb * g.nrows + row0 + rbb) * H + k] = B;
      }
    }
  }
  if (FIRST) return;
  // 6. partial sums of this block
  d2 = block_sum(d2, red);
  n2 = block_sum(n2, red);
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
// Green step, inverse.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(256) line_pass(GridInfo g, DevPlan plan, const cplx<T>* __restrict__ tw,
                                                 cplx<T>* __restrict__ S, const T* __restrict__ Gt,
                                                 const LoadState* st, int ax, int W, int ntiles,
                                                 int n_outer, int n_inner) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int b = blockIdx.x;
  const int tile = b % ntiles; b /= ntiles;
  const int inner = b % n_inner; b /= n_inner;
  const int outer = b % n_outer; b /= n_outer;
  const int load = b;
  if (st[load].done) return;
  const int N = g.dims[ax];
  const int nv = g.nv, H = g.H;
  // element stride of axis ax inside one component's half spectrum
  long long stride = H;
  for (int k = ax + 1; k < g.nd - 1; ++k) stride *= g.dims[k];
  const long long base = (long long)outer * N * stride + (long long)inner * H;
  const int w0 = tile * W;
  const int nl = nv * W;
  cplx<T>* X = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* tmp = X + (size_t)nl * N;
  const size_t comp_stride = (size_t)g.nhalf;
  const size_t Sbase = (size_t)load * nv * comp_stride;

  for (int idx = threadIdx.x; idx < nv * N * W; idx += blockDim.x) {
    const int w = idx % W;
    const int t = idx / W;
    const int n = t % N;
    const int c = t / N;
    cplx<T> v;
    v.x = T(0); v.y = T(0);
    if (w0 + w < H) v = S[Sbase + c * comp_stride + base + n * stride + w0 + w];
    X[(size_t)(c * W + w) * N + n] = v;
  }
  __syncthreads();
  if (MODE == 0 || MODE == 2) fft_lines<-1, T>(X, tmp, nl, N, plan, tw);
  if (MODE == 2) {
    // Green step at frequency (l_0 = n, inner axes, l_last = w0 + w)
    for (int idx = threadIdx.x; idx < N * W; idx += blockDim.x) {
      const int w = idx % W;
      const int n = idx / W;
      if (w0 + w >= H) continue;
      const long long f = (long long)n * stride + (long long)inner * H + w0 + w;
      cplx<T> tv[MAXV], ev[MAXV];
      for (int c = 0; c < nv; ++c) tv[c] = X[(size_t)(c * W + w) * N + n];
      T Gm[MAXV][MAXV];
      int t = 0;
      for (int a = 0; a < nv; ++a)
        for (int bb = a; bb < nv; ++bb) {
          const T v = Gt[(size_t)t * g.nhalf + f];
          Gm[a][bb] = v;
          Gm[bb][a] = v;
          ++t;
        }
      for (int a = 0; a < nv; ++a) {
        T re = T(0), im = T(0);
        for (int bb = 0; bb < nv; ++bb) { re -= Gm[a][bb] * tv[bb].x; im -= Gm[a][bb] * tv[bb].y; }
        ev[a].x = re;
        ev[a].y = im;
      }
      if (f == 0)
        for (int a = 0; a < nv; ++a) { ev[a].x = T(0); ev[a].y = T(0); }
      for (int c = 0; c < nv; ++c) X[(size_t)(c * W + w) * N + n] = ev[c];
    }
    __syncthreads();
  }
  if (MODE == 1 || MODE == 2) fft_lines<+1, T>(X, tmp, nl, N, plan, tw);
  for (int idx = threadIdx.x; idx < nv * N * W; idx += blockDim.x) {
    const int w = idx % W;
    const int t = idx / W;
    const int n = t % N;
    const int c = t / N;
    if (w0 + w < H) S[Sbase + c * comp_stride + base + n * stride + w0 + w] = X[(size_t)(c * W + w) * N + n];
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
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) mean_stress(GridInfo g, const T* __restrict__ E,
                                                   const uint8_t* __restrict__ phase,
                                                   const double* __restrict__ Cp, Control* ctl,
                                                   double* __restrict__ partials, double* __restrict__ out,
                                                   int blocks_per_load) {
  __shared__ double red[32];
  __shared__ unsigned int s_ticket;
  const int load = blockIdx.x / blocks_per_load;
  const int q = blockIdx.x - load * blocks_per_load;
  const int nv = g.nv;
  double acc[MAXV] = {0, 0, 0, 0, 0, 0};
  double e0[MAXV];
  for (int c = 0; c < nv; ++c) e0[c] = ctl->eps0[load][c];
  const size_t Ebase = (size_t)load * nv * g.m;
  for (long long i = (long long)q * blockDim.x + threadIdx.x; i < g.m; i += (long long)blocks_per_load * blockDim.x) {
    double e[MAXV];
    for (int c = 0; c < nv; ++c) e[c] = (double)E[Ebase + (size_t)c * g.m + i] + e0[c];
    const double* C = Cp + (size_t)phase[i] * nv * nv;
    for (int a = 0; a < nv; ++a) {
      double s = 0.0;
      for (int b = 0; b < nv; ++b) s += C[a * nv + b] * e[b];
      acc[a] += s;
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
    G64[(size_t)t * P.nhalf + f] = v;
    G32[(size_t)t * P.nhalf + f] = (float)v;
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
