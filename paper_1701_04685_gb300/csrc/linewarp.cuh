// Warp-per-column variant of the line pass for 3-D grids (n_v = 6) in FP32,
// for axes of N = 32 P points, P in {1, 2, 4, 8}.
//
// The half spectrum of one component is a set of columns along axis `ax`:
// column q (the flattened indices of every other axis, the contiguous
// frequency axis fastest) holds N points at stride `stride`.  A block owns
// kColTile adjacent columns of one load, all six components:
//   1. the tile moves from global memory into shared memory in chunks of
//      kColTile contiguous entries per (component, point), every load of a
//      thread issued before any store;
//   2. warp w transforms column w, three complex lines at a time, in
//      registers (length-P DFT, then a 32-point exchange across lanes, as in
//      the warp row pass), reading and writing only its own column;
//   3. MODE 2 (axis 0): after the forward transform, the Green step
//      E^ = -Gamma^p tau^ (E^_0 = 0) runs with one thread per (point, column),
//      so that a warp's table reads cover whole 32-byte sectors, then the
//      inverse transform;
//   4. the tile goes back to global memory.
// Blocks are numbered load-fastest: the blocks of all loads that read the
// same table tile run close together and share it through L2.
#pragma once

#include "warprow.cuh"

namespace fh {

constexpr int kColTile = 8;                      // columns per block = warps per block
constexpr int kColThreads = 32 * kColTile;

// padded line length in shared memory: holds wpad(N - 1) + 1 entries and is
// 2 mod 16, so that the tile copy (8 columns x 4 points per warp) and the
// lane-strided line accesses both spread over all banks
__host__ __device__ constexpr int col_ls(int N) {
  return ((N + (N - 1) / 16 + 1 + 13) / 16) * 16 + 2;
}

template <int P>
__host__ inline size_t colpass_smem() {
  return (size_t)(32 * P + 6 * kColTile * col_ls(32 * P)) * sizeof(float2);
}

template <int P, int MODE>
__global__ void __launch_bounds__(kColThreads) line_pass_warp6(GridInfo g, const float2* __restrict__ twg,
                                                               float2* __restrict__ S, const float* __restrict__ Gt,
                                                               const LoadState* st, long long stride,
                                                               long long ncols, int nload) {
  constexpr int NV = 6, NTRI = 21, N = 32 * P, LS = col_ls(N);
  constexpr int PER = NV * N * kColTile / kColThreads;    // tile entries per thread (= 6 P)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);       // N
  float2* tile = tw + N;                                   // [NV][kColTile][LS]
  __shared__ long long colbase[kColTile];
  const int load = blockIdx.x % nload;
  const long long q0 = (long long)(blockIdx.x / nload) * kColTile;
  if (st[load].done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  // offset of point 0 of each column inside one component (column q = outer
  // * stride + r lives at outer * N * stride + r)
  if (threadIdx.x < kColTile) {
    const long long q = q0 + threadIdx.x;
    const long long outer = q / stride;
    colbase[threadIdx.x] = outer * N * stride + (q - outer * stride);
  }
  __syncthreads();
  float2* Sl = S + (size_t)load * NV * g.nhalf;
  auto goff = [&](int w, int n) -> long long { return colbase[w] + (long long)n * stride; };
  // extents for the checked build: the launch's loads, the tile
  const long long sl0 = (long long)load * NV * g.nhalf, nS = (long long)nload * NV * g.nhalf;
  constexpr long long nT = (long long)NV * kColTile * LS;
  (void)sl0; (void)nS;

  // 1. tile in: thread t takes entries t + kColThreads * i, column fastest
  {
    float2 v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = threadIdx.x + kColThreads * i;
      const int w = idx % kColTile, t = idx / kColTile;
      const int n = t % N, c = t / N;
      v[i] = make_float2(0.f, 0.f);
      if (q0 + w < ncols && FH_IN(CK_COL_S, sl0 + (long long)c * g.nhalf + goff(w, n), nS))
        v[i] = Sl[(size_t)c * g.nhalf + goff(w, n)];
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = threadIdx.x + kColThreads * i;
      const int w = idx % kColTile, t = idx / kColTile;
      const int n = t % N, c = t / N;
      if (FH_IN(CK_COL_TILE, (c * kColTile + w) * LS + wpad(n), nT)) tile[(c * kColTile + w) * LS + wpad(n)] = v[i];
    }
  }
  __syncthreads();

  // 2. warp transforms of column `warp`, three components at a time
  auto forward = [&]() {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float2 z[3][P];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const float2* col = tile + ((3 * half + p) * kColTile + warp) * LS;
#pragma unroll
        for (int j = 0; j < P; ++j) z[p][j] = col[wpad(lane + 32 * j)];
      }
      warp_fft_fwd_any<P, 3, float>(z, tw, lane);
      __syncwarp();
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        float2* col = tile + ((3 * half + p) * kColTile + warp) * LS;
#pragma unroll
        for (int q = 0; q < P; ++q) col[wpad(warp_freq<P>(lane, q))] = z[p][q];
      }
    }
  };
  auto inverse = [&]() {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float2 z[3][P];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const float2* col = tile + ((3 * half + p) * kColTile + warp) * LS;
#pragma unroll
        for (int q = 0; q < P; ++q) z[p][q] = col[wpad(warp_freq<P>(lane, q))];
      }
      warp_fft_inv_any<P, 3, float>(z, tw, lane);
      __syncwarp();
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        float2* col = tile + ((3 * half + p) * kColTile + warp) * LS;
#pragma unroll
        for (int j = 0; j < P; ++j) col[wpad(lane + 32 * j)] = z[p][j];
      }
    }
  };

  if (MODE == 1) {
    inverse();
  } else {
    forward();
  }
  if (MODE == 2) {
    __syncthreads();
    // 3. Green step at frequency (n along axis 0, column q): f = n * stride + q
    for (int idx = threadIdx.x; idx < N * kColTile; idx += blockDim.x) {
      const int w = idx % kColTile, n = idx / kColTile;
      const long long q = q0 + w;
      if (q >= ncols) continue;
      const long long f = (long long)n * stride + q;
      if (!FH_IN(CK_COL_G, f, g.nhalf) || !FH_IN(CK_COL_TILE, ((NV - 1) * kColTile + w) * LS + wpad(n), nT)) continue;
      float2 tv[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) tv[c] = tile[(c * kColTile + w) * LS + wpad(n)];
      float gm[NTRI];
#pragma unroll
      for (int t = 0; t < NTRI; ++t) gm[t] = Gt[(size_t)t * g.nhalf + f];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int b = 0; b < NV; ++b) {
          const int lo = a < b ? a : b, hi = a < b ? b : a;
          const float gv = gm[lo * NV - (lo * (lo - 1)) / 2 + (hi - lo)];
          re = fmaf(-gv, tv[b].x, re);
          im = fmaf(-gv, tv[b].y, im);
        }
        tile[(a * kColTile + w) * LS + wpad(n)] = (f == 0) ? make_float2(0.f, 0.f) : make_float2(re, im);
      }
    }
    __syncthreads();
    inverse();
  }
  __syncthreads();

  // 4. tile out
  {
    float2 v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = threadIdx.x + kColThreads * i;
      const int w = idx % kColTile, t = idx / kColTile;
      const int n = t % N, c = t / N;
      v[i] = FH_IN(CK_COL_TILE, (c * kColTile + w) * LS + wpad(n), nT) ? tile[(c * kColTile + w) * LS + wpad(n)]
                                                                        : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = threadIdx.x + kColThreads * i;
      const int w = idx % kColTile, t = idx / kColTile;
      const int n = t % N, c = t / N;
      if (q0 + w < ncols && FH_IN(CK_COL_S, sl0 + (long long)c * g.nhalf + goff(w, n), nS))
        Sl[(size_t)c * g.nhalf + goff(w, n)] = v[i];
    }
  }
}

}  // namespace fh
