// Two-step column pass for 3-D grids (n_v = 6) in FP32 or FP64, for axes of
// N = R1 R2 points (32 = 4 x 8, 64 = 8 x 8, 128 = 8 x 16).
//
// Same job as line_pass_warp6 (forward, inverse, or forward + Green step +
// inverse along one strided axis of the half spectra, CT = 8 or 4 adjacent
// columns of one load and all six components per block), with the length-N
// DFT of each column split as N = R1 R2 (the four-step factorisation):
// with j = j2 + R2 j1 and k = k1 + R1 k2,
//   X[k1 + R1 k2] = sum_j2 w_R2^{j2 k2} w_N^{j2 k1} sum_j1 w_R1^{j1 k1} x[j2 + R2 j1].
//   stage A - one thread per (column, j2): the R1 points x[j2 + R2 j1] come
//             straight from global memory (the eight columns of a tile are
//             adjacent, so eight lanes read 64 contiguous bytes), an R1-point
//             DFT in registers, the twiddles w_N^{j2 k1}, one store to shared
//             memory;
//   stage B - one thread per (column, k1): the R2 values of row k1 from
//             shared memory, an R2-point DFT in registers, and the
//             frequencies k1 + R1 k2 straight to global memory.
// Each value passes through shared memory once (one store, one load) and no
// lane exchange is needed.  MODE 2 (axis 0) keeps the spectrum in shared
// memory, runs the Green step E^ = -Gamma^p tau^ (E^_0 = 0) with one thread
// per (frequency, column), and takes the inverse in the mirror order (stage B
// inverse with the twiddles after it, then stage A inverse, writing the
// points in natural order).  Inverse transforms are unnormalised.
//
// Shared memory: line (component c, column w) = c CT + w holds the R1 rows
// of R2 values at padded offsets j2 + (R2 + 1) k1, LS entries per line.  In
// FP32 LS = 16 / CT mod 16: eight-byte accesses are served per half-warp (CT
// columns x 16 / CT values of j2, or x 16 / CT rows k1), the columns land
// 32 / CT banks apart and the values or rows 2 banks apart.  In FP64 (CT = 4)
// LS = 2 mod 16: sixteen-byte accesses are served per quarter-warp (4 columns
// x 2 values or rows), the columns land 8 banks apart and the values or rows
// 4.  So the stage A stores, the stage B loads and the Green step's accesses
// are free of bank conflicts.
#pragma once

#include "linewarp.cuh"

namespace fh {

template <int R1, int R2, int CT = kColTile, typename T = float>
struct Col2 {
  static constexpr int N = R1 * R2;
  static constexpr int RMIN = R1 < R2 ? R1 : R2;
  static constexpr int LINES = 6 * CT;                       // lines per block (48 for 8 columns)
  static constexpr int THREADS = LINES * RMIN;
  static constexpr int A_PER = LINES * R2 / THREADS;         // stage A tasks per thread
  static constexpr int B_PER = LINES * R1 / THREADS;         // stage B tasks per thread
  static constexpr int OFF = sizeof(T) == 4 ? 16 / CT : 2;   // line stride mod 16
  static constexpr int LS = ((N + R1 - OFF + 15) / 16) * 16 + OFF;
  static_assert(CT == 4 || CT == 8, "4 or 8 columns per block");
  static_assert(A_PER * THREADS == LINES * R2 && B_PER * THREADS == LINES * R1, "uneven task split");
  static_assert(LS >= N + R1 && LS % 16 == OFF, "line stride");
};

template <int R1, int R2, int CT = kColTile, typename T = float>
__host__ inline size_t col2_smem() {
  return (size_t)(R1 * R2 + 6 * CT * Col2<R1, R2, CT, T>::LS) * 2 * sizeof(T);
}

// padded offset of (row k1, entry j2) inside a line
template <int R2>
__device__ __forceinline__ int c2off(int k1, int j2) { return j2 + (R2 + 1) * k1; }

// w[t] = w_N^{DIR base t} for t < R (R = 4, 8 or 16): the powers t = 1, 2, 4, 8
// come from the table tw[t] = exp(-2 pi i t / N), every other one is the
// product of two earlier ones (at most three roundings deep)
template <int R, int DIR, typename T = float>
__device__ __forceinline__ void twiddle_powers(const cplx<T>* tw, int base, cplx<T>* w) {
  w[0].x = T(1);
  w[0].y = T(0);
#pragma unroll
  for (int p = 1; p < R; p <<= 1) w[p] = twl<DIR, T>(tw, base * p);
#pragma unroll
  for (int t = 3; t < R; ++t) {
    if ((t & (t - 1)) == 0) continue;
    const int hi = t >= 8 ? 8 : (t >= 4 ? 4 : 2);
    w[t] = cmul(w[hi], w[t - hi]);
  }
}

// resident blocks per SM the register budget is set for: three for the
// single transforms, two for MODE 2 (whose Green step wants more registers;
// measured faster at two)
template <int MODE>
constexpr int col2_minb() { return MODE == 2 ? 2 : 3; }

template <int R1, int R2, int MODE, int CT = kColTile, int MINB = col2_minb<MODE>(), typename T = float>
__global__ void __launch_bounds__(Col2<R1, R2, CT, T>::THREADS, MINB)
    line_pass_2s(GridInfo g, const cplx<T>* __restrict__ twg, cplx<T>* __restrict__ S, const T* __restrict__ Gt,
                 const LoadState* st, long long stride, long long ncols, int nload) {
  using K = Col2<R1, R2, CT, T>;
  using C = cplx<T>;
  const C czero = {T(0), T(0)};
  constexpr int NV = 6, NTRI = 21, N = K::N, LS = K::LS;
  // forward transforms take w = exp(-2 pi i / N); MODE 1 is an inverse
  constexpr int DIR = MODE == 1 ? 1 : -1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);   // tw[t] = exp(-2 pi i t / N)
  C* tile = tw + N;                          // [NV * CT][LS]
  __shared__ long long colbase[CT];
  const int load = blockIdx.x % nload;
  const long long q0 = (long long)(blockIdx.x / nload) * CT;
  if (st[load].done) return;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  if (threadIdx.x < CT) {
    const long long q = q0 + threadIdx.x;
    const long long outer = q / stride;
    colbase[threadIdx.x] = outer * N * stride + (q - outer * stride);
  }
  __syncthreads();
  C* Sl = S + (size_t)load * NV * g.nhalf;
  auto gidx = [&](int c, int w, int n) -> size_t { return (size_t)c * g.nhalf + colbase[w] + (long long)n * stride; };
  // extents for the checked build: the launch's loads, the tile
  const long long sl0 = (long long)load * NV * g.nhalf, nS = (long long)nload * NV * g.nhalf;
  constexpr long long nT = (long long)NV * CT * LS;
  (void)sl0; (void)nS; (void)nT;

  // stage A (first step in natural order): task a -> column w, entry j2, component c
  {
    C v[K::A_PER][R1];
#pragma unroll
    for (int i = 0; i < K::A_PER; ++i) {
      const int a = threadIdx.x + K::THREADS * i;
      const int w = a % CT, j2 = (a / CT) % R2, c = a / (CT * R2);
      const bool ok = q0 + w < ncols;
#pragma unroll
      for (int j1 = 0; j1 < R1; ++j1)
        v[i][j1] = ok && FH_IN(CK_C2_S, sl0 + (long long)gidx(c, w, j2 + R2 * j1), nS) ? Sl[gidx(c, w, j2 + R2 * j1)]
                                                                                    : czero;
    }
#pragma unroll
    for (int i = 0; i < K::A_PER; ++i) {
      const int a = threadIdx.x + K::THREADS * i;
      const int w = a % CT, j2 = (a / CT) % R2, c = a / (CT * R2);
      small_dft<R1, DIR, T>(v[i]);
      C twv[R1];
      twiddle_powers<R1, DIR, T>(tw, j2, twv);
      if (!FH_IN(CK_C2_TILE, (c * CT + w) * LS + c2off<R2>(R1 - 1, j2), nT)) continue;
      C* line = tile + (c * CT + w) * LS;
      line[c2off<R2>(0, j2)] = v[i][0];
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) line[c2off<R2>(k1, j2)] = cmul(v[i][k1], twv[k1]);
    }
  }
  __syncthreads();

  if constexpr (MODE != 2) {
    // stage B, results to global memory in natural frequency order
#pragma unroll
    for (int i = 0; i < K::B_PER; ++i) {
      const int b = threadIdx.x + K::THREADS * i;
      const int w = b % CT, k1 = (b / CT) % R1, c = b / (CT * R1);
      if (!FH_IN(CK_C2_TILE, (c * CT + w) * LS + c2off<R2>(k1, R2 - 1), nT)) continue;
      const C* line = tile + (c * CT + w) * LS;
      C v[R2];
#pragma unroll
      for (int j2 = 0; j2 < R2; ++j2) v[j2] = line[c2off<R2>(k1, j2)];
      small_dft<R2, DIR, T>(v);
      if (q0 + w < ncols) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
          if (FH_IN(CK_C2_S, sl0 + (long long)gidx(c, w, k1 + R1 * k2), nS)) Sl[gidx(c, w, k1 + R1 * k2)] = v[k2];
      }
    }
  } else {
  // MODE 2: stage B forward in place (row k1 now holds X[k1 + R1 k2] at entry k2)
#pragma unroll
  for (int i = 0; i < K::B_PER; ++i) {
    const int b = threadIdx.x + K::THREADS * i;
    const int w = b % CT, k1 = (b / CT) % R1, c = b / (CT * R1);
    if (!FH_IN(CK_C2_TILE, (c * CT + w) * LS + c2off<R2>(k1, R2 - 1), nT)) continue;
    C* line = tile + (c * CT + w) * LS;
    C v[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) v[j2] = line[c2off<R2>(k1, j2)];
    small_dft<R2, -1, T>(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) line[c2off<R2>(k1, k2)] = v[k2];
  }
  __syncthreads();

  // Green step at frequency (n along this axis, column q): f = n * stride + q
  for (int idx = threadIdx.x; idx < N * CT; idx += K::THREADS) {
    const int w = idx % CT, n = idx / CT;
    const long long q = q0 + w;
    if (q >= ncols) continue;
    const long long f = (long long)n * stride + q;
    const int off = c2off<R2>(n % R1, n / R1);
    if (!FH_IN(CK_C2_G, f, g.nhalf) || !FH_IN(CK_C2_TILE, ((NV - 1) * CT + w) * LS + off, nT)) continue;
    C tv[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) tv[c] = tile[(c * CT + w) * LS + off];
    T gm[NTRI];
#pragma unroll
    for (int t = 0; t < NTRI; ++t) gm[t] = Gt[(size_t)t * g.nhalf + f];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      T re = T(0), im = T(0);
#pragma unroll
      for (int b = 0; b < NV; ++b) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const T gv = gm[lo * NV - (lo * (lo - 1)) / 2 + (hi - lo)];
        re = fma(-gv, tv[b].x, re);
        im = fma(-gv, tv[b].y, im);
      }
      C e;
      e.x = (f == 0) ? T(0) : re;
      e.y = (f == 0) ? T(0) : im;
      tile[(a * CT + w) * LS + off] = e;
    }
  }
  __syncthreads();

  // inverse, stage B: row k1, sum over k2, then the twiddles w_N^{+j2 k1}
#pragma unroll
  for (int i = 0; i < K::B_PER; ++i) {
    const int b = threadIdx.x + K::THREADS * i;
    const int w = b % CT, k1 = (b / CT) % R1, c = b / (CT * R1);
    if (!FH_IN(CK_C2_TILE, (c * CT + w) * LS + c2off<R2>(k1, R2 - 1), nT)) continue;
    C* line = tile + (c * CT + w) * LS;
    C v[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k2] = line[c2off<R2>(k1, k2)];
    small_dft<R2, 1, T>(v);
    C twv[R2];
    twiddle_powers<R2, 1, T>(tw, k1, twv);
    line[c2off<R2>(k1, 0)] = v[0];
#pragma unroll
    for (int j2 = 1; j2 < R2; ++j2) line[c2off<R2>(k1, j2)] = cmul(v[j2], twv[j2]);
  }
  __syncthreads();

  // inverse, stage A: entry j2, sum over k1, points j2 + R2 j1 to global memory
#pragma unroll
  for (int i = 0; i < K::A_PER; ++i) {
    const int a = threadIdx.x + K::THREADS * i;
    const int w = a % CT, j2 = (a / CT) % R2, c = a / (CT * R2);
    if (!FH_IN(CK_C2_TILE, (c * CT + w) * LS + c2off<R2>(R1 - 1, j2), nT)) continue;
    const C* line = tile + (c * CT + w) * LS;
    C v[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = line[c2off<R2>(k1, j2)];
    small_dft<R1, 1, T>(v);
    if (q0 + w < ncols) {
#pragma unroll
      for (int j1 = 0; j1 < R1; ++j1)
        if (FH_IN(CK_C2_S, sl0 + (long long)gidx(c, w, j2 + R2 * j1), nS)) Sl[gidx(c, w, j2 + R2 * j1)] = v[j1];
    }
  }
  }
}

}  // namespace fh

