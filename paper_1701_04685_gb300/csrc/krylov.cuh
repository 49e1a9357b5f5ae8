// BiCGStab on the discrete equation of the fixed point.
//
// The paper's introduction names Krylov methods as faster solvers of the same
// discretised Lippmann-Schwinger equation.  Eq. (pde_coefficients) is the
// linear system
//
//     A E = b,   A = I + Gamma^p (C - C0),   b = -Gamma^p (C - C0) eps0,
//
// and the Basic Scheme's step from E is E' - E = b - A E: the Cauchy
// criterion of Sec. 4 measures exactly the residual of E.  BiCGStab (van der
// Vorst, 1992) runs on the same operator, with the same stopping rule
// |b - A E| <= tol |E + eps0|, per load case:
//
//   r = b - A E0, rhat = r;  then per iteration
//   p = r (first) or r + beta (p - omega v);   v = A p;   alpha = rho / (rhat . v);
//   s = r - alpha v;   t = A s;   omega = (t . s) / (t . t);
//   E += alpha p + omega s;   r = s - omega t;
//   rho' = rhat . r,  beta = (rho' / rho)(alpha / omega),  rho = rho'.
//
// Operator applications reuse the iteration's passes: the FIRST row pass takes
// the stress of a field (with a zero macroscopic strain) to the half spectrum,
// the line passes apply the Green step, and the inverse-only row pass (KINV)
// writes A X = X - (inverse transform) together with the block sums of two dot
// products.  The vector updates below stream the fields once each; their dot
// products are block partial sums (FP64, or exact FP32 double-float pairs)
// reduced in a fixed order by kry_scalars, which also advances the per-load
// state (iteration count, residual history, stop flags) with the fixed
// point's rules.  Every kernel skips the loads that have stopped.
#pragma once

#include "kernels.cuh"

namespace fh {

struct KrylovScal {
  double rho, alpha, omega, beta;
  int first;  // 1 until the first direction p = r is formed
  int pad;
};

constexpr int kKryThreads = 256;

// p = r (first iteration) or r + beta (p - omega v)
template <typename T>
__global__ void __launch_bounds__(kKryThreads) kry_update_p(T* __restrict__ p, const T* __restrict__ r,
                                                            const T* __restrict__ v, const KrylovScal* sc,
                                                            const LoadState* st, long long n, int bpl) {
  const int load = blockIdx.x / bpl, q = blockIdx.x - load * bpl;
  if (st[load].done) return;
  const KrylovScal k = sc[load];
  const T beta = (T)k.beta, omega = (T)k.omega;
  const size_t base = (size_t)load * n;
  for (long long i = (long long)q * blockDim.x + threadIdx.x; i < n; i += (long long)bpl * blockDim.x) {
    const size_t o = base + i;
    p[o] = k.first ? r[o] : r[o] + beta * (p[o] - omega * v[o]);
  }
}

// s = r - alpha v
template <typename T>
__global__ void __launch_bounds__(kKryThreads) kry_update_s(T* __restrict__ s, const T* __restrict__ r,
                                                            const T* __restrict__ v, const KrylovScal* sc,
                                                            const LoadState* st, long long n, int bpl) {
  const int load = blockIdx.x / bpl, q = blockIdx.x - load * bpl;
  if (st[load].done) return;
  const T alpha = (T)sc[load].alpha;
  const size_t base = (size_t)load * n;
  for (long long i = (long long)q * blockDim.x + threadIdx.x; i < n; i += (long long)bpl * blockDim.x) {
    const size_t o = base + i;
    s[o] = r[o] - alpha * v[o];
  }
}

// three block sums of one load to part[3 * block + j]
template <typename T>
__device__ __forceinline__ void kry_block_sums(const ResAcc<T>& a0, const ResAcc<T>& a1, const ResAcc<T>& a2,
                                               double* part) {
  __shared__ double red[32];
  const double v0 = block_sum_acc(a0, red);
  __syncthreads();
  const double v1 = block_sum_acc(a1, red);
  __syncthreads();
  const double v2 = block_sum_acc(a2, red);
  if (threadIdx.x == 0) {
    part[3 * (size_t)blockIdx.x] = v0;
    part[3 * (size_t)blockIdx.x + 1] = v1;
    part[3 * (size_t)blockIdx.x + 2] = v2;
  }
}

// E += alpha p + omega s;  r = s - omega t;  block sums of |r|^2, rhat . r and
// |E + eps0|^2.  Fields are [load][component][m].
template <typename T>
__global__ void __launch_bounds__(kKryThreads) kry_update_xr(T* __restrict__ x, T* __restrict__ r,
                                                             const T* __restrict__ p, const T* __restrict__ s,
                                                             const T* __restrict__ t, const T* __restrict__ rhat,
                                                             const KrylovScal* sc, const LoadState* st,
                                                             const Control* ctl, long long m, int nv, int bpl,
                                                             double* __restrict__ part) {
  const int load = blockIdx.x / bpl, q = blockIdx.x - load * bpl;
  ResAcc<T> arr, arh, axx;
  if (FH_IN(CK_KRY, load, ctl->nload) && !st[load].done) {
    const T alpha = (T)sc[load].alpha, omega = (T)sc[load].omega;
    const size_t base = (size_t)load * nv * m;
    for (int c = 0; c < nv; ++c) {
      const T e0 = (T)ctl->eps0[load][c];
      for (long long i = (long long)q * blockDim.x + threadIdx.x; i < m; i += (long long)bpl * blockDim.x) {
        const size_t o = base + (size_t)c * m + i;
        const T sv = s[o];
        const T xn = x[o] + alpha * p[o] + omega * sv;
        const T rn = sv - omega * t[o];
        x[o] = xn;
        r[o] = rn;
        arr.add_sq(rn);
        arh.add_prod(rhat[o], rn);
        axx.add_sq(xn + e0);
      }
    }
  }
  kry_block_sums<T>(arr, arh, axx, part);
}

// start: the inverse-only pass wrote W = E0 - y with y = b - Gamma^p (C - C0) E0
// (stress of E0 + eps0), so r = b - A E0 = -W; rhat = r; block sums of |r|^2
// and |E0 + eps0|^2
template <typename T>
__global__ void __launch_bounds__(kKryThreads) kry_init(T* __restrict__ r, T* __restrict__ rhat,
                                                        const T* __restrict__ x, const LoadState* st,
                                                        const Control* ctl, long long m, int nv, int bpl,
                                                        double* __restrict__ part) {
  const int load = blockIdx.x / bpl, q = blockIdx.x - load * bpl;
  ResAcc<T> arr, axx, unused;
  if (FH_IN(CK_KRY, load, ctl->nload) && !st[load].done) {
    const size_t base = (size_t)load * nv * m;
    for (int c = 0; c < nv; ++c) {
      const T e0 = (T)ctl->eps0[load][c];
      for (long long i = (long long)q * blockDim.x + threadIdx.x; i < m; i += (long long)bpl * blockDim.x) {
        const size_t o = base + (size_t)c * m + i;
        const T rv = -r[o];
        r[o] = rv;
        rhat[o] = rv;
        arr.add_sq(rv);
        axx.add_sq(x[o] + e0);
      }
    }
  }
  kry_block_sums<T>(arr, unused, axx, part);
}

// Fixed-order reduction of the block sums of every load and the scalar step
// of BiCGStab; one block.
//   STEP 0 (after kry_init):      rho = |r|^2 = rhat . r; first = 1
//   STEP 1 (after v = A p; sums (v . rhat, v . v)):   alpha = rho / (rhat . v)
//   STEP 2 (after t = A s; sums (t . s, t . t)):      omega = (t . s) / (t . t)
//   STEP 3 (after kry_update_xr): rho' = rhat . r, beta = (rho'/rho)(alpha/omega),
//          residual |r| / |E + eps0| -> iteration count, history, stop flags
// A zero denominator (breakdown, or an exact solution) sets that scalar to 0.
template <int STEP>
__global__ void __launch_bounds__(kKryThreads) kry_scalars(KrylovScal* sc, LoadState* st, Control* ctl,
                                                           double* __restrict__ hist,
                                                           const double* __restrict__ part, int nsum, int bpl) {
  __shared__ double red[32];
  for (int l = 0; l < ctl->nload; ++l) {
    if (st[l].done) continue;
    double v[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < nsum; ++j) {
      double a = 0.0;
      for (int qq = threadIdx.x; qq < bpl; qq += blockDim.x) a += part[(size_t)nsum * ((size_t)l * bpl + qq) + j];
      v[j] = block_sum(a, red);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      KrylovScal& k = sc[l];
      if (STEP == 0) {
        k.rho = v[0];
        k.alpha = k.omega = 1.0;
        k.beta = 0.0;
        k.first = 1;
        if (!(v[0] > 0.0)) {  // E0 solves the system (or the residual is not finite)
          st[l].status = isfinite(v[0]) ? FH_OK : FH_NONFINITE;
          st[l].done = 1;
        }
      } else if (STEP == 1) {
        k.alpha = v[0] != 0.0 ? k.rho / v[0] : 0.0;
      } else if (STEP == 2) {
        k.omega = v[1] != 0.0 ? v[0] / v[1] : 0.0;
      } else {
        const double rho_new = v[1];
        k.beta = (k.rho != 0.0 && k.omega != 0.0) ? (rho_new / k.rho) * (k.alpha / k.omega) : 0.0;
        k.rho = rho_new;
        k.first = 0;
        advance_state(st[l], ctl, hist, l, v[0], v[2]);
      }
    }
    __syncthreads();
  }
  if (STEP == 3 && threadIdx.x == 0) {
    int all = 1;
    for (int l = 0; l < ctl->nload; ++l) all &= st[l].done;
    ctl->all_done = all;
  }
}

}  // namespace fh
