// Two-step row pass for 3-D grids (n_v = 6) whose contiguous axis has
// L = R1 R2 points (32 = 4 x 8, 64 = 8 x 8, 128 = 8 x 16), FP32 or FP64.
//
// The stages of row_pass_warp6 (inverse transform of the half spectra, E
// update and Cauchy-residual sums, tau = (C - C0):(E + eps0), forward
// transform), with each row's complex line DFTs split as in the two-step
// column pass (j = j2 + R2 j1, k = k1 + R1 k2):
//   X[k1 + R1 k2] = sum_j2 w_R2^{j2 k2} w_L^{j2 k1} sum_j1 w_R1^{j1 k1} x[j2 + R2 j1],
// on shared-memory lines instead of lane exchanges.  A block owns RB rows of
// one load; each row's six components form three complex lines (components
// 2p and 2p + 1 as real and imaginary parts).
//   inverse   stage A: thread (line, j2) gathers Z[j2 + R2 j1] = A + i B from
//             the two half spectra in global memory (the conjugate mirror for
//             k > L/2; sixteen lanes read 128 contiguous bytes), R1-point DFT,
//             twiddles; stage B: thread (line, k1) the R2-point DFT of row k1,
//             points k1 + R1 k2 back in natural order;
//   pointwise thread (row, point): the three lines' values there are the six
//             components of the new strain; E_old from global memory, the
//             residual sums, E_new out, tau into the same line positions;
//   forward   the same two steps on tau, then thread (line, k) splits Z[k],
//             Z[L - k] into the half spectra of the line's two components.
// Results of a stage go back to the positions another thread reads, so each
// stage reads into registers, meets a block barrier, then writes.  Line
// stride LS = 8 mod 16 elements: every half-warp access of the FP32 form (and
// quarter-warp access of the FP64 form) is free of bank conflicts for
// L = 64 and 128.  FIRST: no inverse (the strain itself is transformed);
// KINV: no forward (Wout = X - inverse transform and the block sums of
// Wout . Yaux, Wout . Wout, as in row_pass).  The last block reduces the
// residual partials of every load in a fixed order and advances the states.
#pragma once

#include "colpass2.cuh"

namespace fh {

template <int R1, int R2>
struct Row2 {
  static constexpr int L = R1 * R2;
  static constexpr int H = L / 2 + 1;
  static constexpr int RMIN = R1 < R2 ? R1 : R2;
  static constexpr int THREADS = 384;
  static constexpr int RB = THREADS / (3 * RMIN);            // rows per block
  static constexpr int LINES = 3 * RB;
  static constexpr int A_PER = LINES * R2 / THREADS;         // stage A tasks per thread
  static constexpr int B_PER = LINES * R1 / THREADS;         // stage B tasks per thread
  static constexpr int OFF = R1 == 4 ? 4 : 8;
  static constexpr int LS = ((L + R1 - 1 - OFF + 15) / 16) * 16 + OFF;
  static_assert(A_PER * THREADS == LINES * R2 && B_PER * THREADS == LINES * R1, "uneven task split");
  static_assert(LS >= L + R1 - 1 && LS % 16 == OFF, "line stride");
};

template <typename T, int R1, int R2>
__host__ inline size_t row2_smem() {
  return (size_t)(R1 * R2 + Row2<R1, R2>::LINES * Row2<R1, R2>::LS) * 2 * sizeof(T);
}

template <typename T, int R1, int R2, bool FIRST, bool KINV = false>
__global__ void __launch_bounds__(Row2<R1, R2>::THREADS, sizeof(T) == 4 ? 3 : 1)
    row_pass_2s(GridInfo g, const cplx<T>* __restrict__ twg, T* __restrict__ E, cplx<T>* __restrict__ S,
                const uint8_t* __restrict__ phase, const T* __restrict__ dC, Control* ctl, LoadState* st,
                double* __restrict__ partials, double* __restrict__ hist, int blocks_per_load,
                T* __restrict__ Wout = nullptr, const T* __restrict__ Yaux = nullptr) {
  static_assert(!(FIRST && KINV), "the inverse-only pass follows a transform");
  using K = Row2<R1, R2>;
  using C = cplx<T>;
  constexpr int NV = 6, L = K::L, H = K::H, LS = K::LS, RB = K::RB, NT = K::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);   // tw[t] = exp(-2 pi i t / L)
  C* buf = tw + L;                          // [LINES][LS]: line 3 r + p = row r, components 2p, 2p + 1
  __shared__ __align__(16) T dcs[16 * NV * NV];
  __shared__ __align__(16) T dcp[16 * 12];   // the 12 nonzeros of decoupled phase matrices
  __shared__ double red[32];
  __shared__ int s_skip;
  const bool decoupled = ctl->decoupled != 0;
  const bool no_fwd = !FIRST && !KINV && ctl->no_forward != 0;
  const int load = blockIdx.x / blocks_per_load;
  const int qb = blockIdx.x - load * blocks_per_load;
  const long long row0 = (long long)qb * RB;
  for (int i = threadIdx.x; i < L; i += NT) tw[i] = twg[i];
  if (!KINV) {
    for (int i = threadIdx.x; i < 16 * NV * NV; i += NT) dcs[i] = dC[i];
    if (decoupled)
      for (int i = threadIdx.x; i < 16 * 12; i += NT) dcp[i] = decoupled_entry(dC + (i / 12) * NV * NV, i % 12);
  }
  if (threadIdx.x == 0) s_skip = st[load].done;
  __syncthreads();
  ResAcc<T> acc_d, acc_n;
  const size_t cstrS = (size_t)g.nrows * H, cstrE = (size_t)g.m;
  // extents for the checked build
  const long long nS = (long long)ctl->nload * NV * g.nhalf, nE = (long long)ctl->nload * NV * g.m;
  constexpr long long nB = (long long)K::LINES * LS;
  (void)nS; (void)nE;
  if (!s_skip) {
    T e0[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) e0[c] = (T)ctl->eps0[load][c];
    const T scale = (T)g.inv_m;
    const bool incremental = ctl->form == 1;
    const C* Sload = S + (size_t)load * NV * cstrS;
    C* Sw = S + (size_t)load * NV * cstrS;
    const T* Eload = E + (size_t)load * NV * cstrE;
    T* Ew = E + (size_t)load * NV * cstrE;

    // ---- inverse: half spectra -> points, natural order in buf
    if (!FIRST) {
      C v[K::A_PER][R1];
#pragma unroll
      for (int i = 0; i < K::A_PER; ++i) {
        const int a = threadIdx.x + NT * i;
        const int j2 = a % R2, line = a / R2;
        const int r = line / 3, p = line - 3 * r;
        const long long row = row0 + r;
        const bool ok = row < g.nrows &&
                        FH_IN(CK_ROW_S, ((long long)load * NV + 2 * p + 1) * (long long)cstrS + row * H + H - 1, nS);
#pragma unroll
        for (int j1 = 0; j1 < R1; ++j1) {
          const int k = j2 + R2 * j1;
          const bool lo = k <= L / 2;
          const int kk = lo ? k : L - k;
          C A, B;
          A.x = A.y = B.x = B.y = T(0);
          if (ok) {
            A = Sload[(size_t)(2 * p) * cstrS + row * H + kk];
            B = Sload[(size_t)(2 * p + 1) * cstrS + row * H + kk];
          }
          if (!lo) { A.y = -A.y; B.y = -B.y; }
          v[i][j1].x = A.x - B.y;
          v[i][j1].y = A.y + B.x;
        }
      }
#pragma unroll
      for (int i = 0; i < K::A_PER; ++i) {
        const int a = threadIdx.x + NT * i;
        const int j2 = a % R2, line = a / R2;
        small_dft<R1, 1, T>(v[i]);
        C twv[R1];
        twiddle_powers<R1, 1, T>(tw, j2, twv);
        C* ln = buf + line * LS;
        if (!FH_IN(CK_ROW_SMEM, line * LS + c2off<R2>(R1 - 1, j2), nB)) continue;
        ln[c2off<R2>(0, j2)] = v[i][0];
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) ln[c2off<R2>(k1, j2)] = cmul(v[i][k1], twv[k1]);
      }
      __syncthreads();
      C w[K::B_PER][R2];
#pragma unroll
      for (int i = 0; i < K::B_PER; ++i) {
        const int b = threadIdx.x + NT * i;
        const int k1 = b % R1, line = b / R1;
        const C* ln = buf + line * LS;
#pragma unroll
        for (int j2 = 0; j2 < R2; ++j2) w[i][j2] = ln[c2off<R2>(k1, j2)];
        small_dft<R2, 1, T>(w[i]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < K::B_PER; ++i) {
        const int b = threadIdx.x + NT * i;
        const int k1 = b % R1, line = b / R1;
        C* ln = buf + line * LS;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) ln[k1 + R1 * k2] = w[i][k2];
      }
      __syncthreads();
    }

    // ---- pointwise
    for (int idx = threadIdx.x; idx < RB * L; idx += NT) {
      const int r = idx / L, x = idx - r * L;
      const long long row = row0 + r;
      if (row >= g.nrows) continue;
      const size_t pt = (size_t)row * L + x;
      if (!(FH_IN(CK_ROW_E, (long long)load * NV * (long long)cstrE + (NV - 1) * (long long)cstrE + (long long)pt, nE) &&
            FH_IN(CK_ROW_PHASE, (long long)pt, g.m)))
        continue;
      C* ln = buf + (3 * r) * LS + x;
      T ev[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) ev[c] = Eload[c * cstrE + pt];
      if constexpr (KINV) {
        const T* Yl = Yaux ? Yaux + (size_t)load * NV * cstrE : Eload;
        T* Wl = Wout + (size_t)load * NV * cstrE;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const C z = ln[p * LS];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = 2 * p + h;
            const T wv = ev[c] - (h ? z.y : z.x) * scale;
            Wl[c * cstrE + pt] = wv;
            acc_d.add_prod(wv, Yaux ? Yl[c * cstrE + pt] : ev[c]);
            acc_n.add_sq(wv);
          }
        }
        continue;
      }
      T en[NV];
      if (FIRST) {
#pragma unroll
        for (int c = 0; c < NV; ++c) en[c] = ev[c];
      } else {
        T rd = T(0), rn = T(0);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const C z = ln[p * LS];
          en[2 * p] = z.x * scale;
          en[2 * p + 1] = z.y * scale;
        }
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          if (incremental) en[c] += ev[c];
          const T dd = en[c] - ev[c], nn = en[c] + e0[c];
          rd = fma(dd, dd, rd);
          rn = fma(nn, nn, rn);
          Ew[c * cstrE + pt] = en[c];
        }
        acc_d.add(rd);
        acc_n.add(rn);
      }
      if (no_fwd) continue;
      int ph = phase[pt];
      if (!FH_IN(CK_ROW_PHASE, ph, 16)) ph = 0;
      if (decoupled) {
        T xv[NV], tau[NV];
#pragma unroll
        for (int b = 0; b < NV; ++b) xv[b] = en[b] + e0[b];
        stress6_decoupled<T>(dcp + ph * 12, xv, tau);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          C z;
          z.x = tau[2 * p];
          z.y = tau[2 * p + 1];
          ln[p * LS] = z;
        }
      } else {
      const T* dc = dcs + ph * NV * NV;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        T t0 = T(0), t1 = T(0);
#pragma unroll
        for (int b = 0; b < NV; ++b) {
          t0 = fma(dc[(2 * p) * NV + b], en[b] + e0[b], t0);
          t1 = fma(dc[(2 * p + 1) * NV + b], en[b] + e0[b], t1);
        }
        C z;
        z.x = t0;
        z.y = t1;
        ln[p * LS] = z;
      }
      }
    }

    // ---- forward: tau -> half spectra
    if (!KINV && !no_fwd) {
      __syncthreads();
      C v[K::A_PER][R1];
#pragma unroll
      for (int i = 0; i < K::A_PER; ++i) {
        const int a = threadIdx.x + NT * i;
        const int j2 = a % R2, line = a / R2;
        const C* ln = buf + line * LS;
#pragma unroll
        for (int j1 = 0; j1 < R1; ++j1) v[i][j1] = ln[j2 + R2 * j1];
        small_dft<R1, -1, T>(v[i]);
        C twv[R1];
        twiddle_powers<R1, -1, T>(tw, j2, twv);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[i][k1] = cmul(v[i][k1], twv[k1]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < K::A_PER; ++i) {
        const int a = threadIdx.x + NT * i;
        const int j2 = a % R2, line = a / R2;
        C* ln = buf + line * LS;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) ln[c2off<R2>(k1, j2)] = v[i][k1];
      }
      __syncthreads();
      C w[K::B_PER][R2];
#pragma unroll
      for (int i = 0; i < K::B_PER; ++i) {
        const int b = threadIdx.x + NT * i;
        const int k1 = b % R1, line = b / R1;
        const C* ln = buf + line * LS;
#pragma unroll
        for (int j2 = 0; j2 < R2; ++j2) w[i][j2] = ln[c2off<R2>(k1, j2)];
        small_dft<R2, -1, T>(w[i]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < K::B_PER; ++i) {
        const int b = threadIdx.x + NT * i;
        const int k1 = b % R1, line = b / R1;
        C* ln = buf + line * LS;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) ln[k1 + R1 * k2] = w[i][k2];
      }
      __syncthreads();
      // split each line's spectrum into its two components' half spectra
      for (int idx = threadIdx.x; idx < K::LINES * H; idx += NT) {
        const int line = idx / H, k = idx - line * H;
        const int r = line / 3, p = line - 3 * r;
        const long long row = row0 + r;
        if (row >= g.nrows) continue;
        if (!FH_IN(CK_ROW_S, ((long long)load * NV + 2 * p + 1) * (long long)cstrS + row * H + k, nS)) continue;
        const C* ln = buf + line * LS;
        const C zk = ln[k];
        const C zm = ln[k == 0 ? 0 : L - k];
        C A, B;
        A.x = T(0.5) * (zk.x + zm.x);
        A.y = T(0.5) * (zk.y - zm.y);
        B.x = T(0.5) * (zk.y + zm.y);
        B.y = T(-0.5) * (zk.x - zm.x);
        Sw[(size_t)(2 * p) * cstrS + row * H + k] = A;
        Sw[(size_t)(2 * p + 1) * cstrS + row * H + k] = B;
      }
    }
  }
  if (FIRST) return;
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

}  // namespace fh
