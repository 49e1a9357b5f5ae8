// Fused plane pass for 3-D grids in FP32 (n_v = 6): one plane x0 = const of
// one load per cluster of two CTAs.
//
// The four-pass iteration (row pass, axis-1 forward, axis-0 forward + Green +
// inverse, axis-1 inverse) moves every load's spectrum through HBM three
// times besides the strain itself.  This kernel replaces the row pass and both
// axis-1 passes: a plane of a load (N1 x H half-spectrum entries per
// component) stays in shared memory while it goes through
//   1. inverse transforms along axis 1 (warp per column),
//   2. inverse transforms along axis 2 (warp per pair of rows: two real rows
//      as the real and imaginary part of one complex line), the strain update
//      E_new, the Cauchy-residual sums, and E_new written to global memory,
//   3. the constitutive stage tau = (C(y) - C0):(E_new + eps0) of Eq.
//      (pde_coefficients) at every point,
//   4. forward transforms along axis 2, split into half spectra,
//   5. forward transforms along axis 1,
// and leaves for the axis-0 pass (which applies the Green step) in global
// memory.  CTA r of the cluster holds the components 3r .. 3r+2 (199.7 KB for
// a 128 x 65 plane), so the pointwise stage reads the other three components
// of its points from the partner CTA's shared memory (distributed shared
// memory): the points are split between the two CTAs by rows, and each thread
// reads the six strain components of its point and writes the six stress
// components back to the same places, so no point is touched by two threads.
//
// Axis-1 columns are stored in shared memory with their frequencies in the
// register order of the warp FFT (slot l + 32 q holds the frequency that lane
// l, register q holds: plane_slot), so that the column transforms read and
// write conflict-free; the permutation is applied on the row index when the
// plane moves between global and shared memory, where whole rows move
// together and coalescing is unaffected.
#pragma once

#include <cooperative_groups.h>

#include "warprow.cuh"

namespace fh {

namespace pcg = cooperative_groups;

constexpr int kPlaneThreads = 512;
constexpr int kPlaneWarps = kPlaneThreads / 32;

// shared-memory slot of axis-1 frequency f: the inverse of (l, q) -> warp_freq<P>(l, q)
template <int P>
__device__ __forceinline__ int plane_slot(int f) {
  if (P == 1) {
    return bitrev5(f);
  } else {
    const int lo = f % P, hi = f / P;
    const int b = bitrev5(hi);
    const int lane = ((lo & 1) << 4) | (b >> 1);
    const int q = ((lo >> 1) << 1) | (b & 1);
    return lane + 32 * q;
  }
}

// per-warp scratch line (complex entries): two half spectra or one line, padded
__host__ __device__ constexpr int plane_ws(int L) {
  return ((2 * (L / 2 + 1) + (2 * (L / 2 + 1)) / 16 + 2) + 1) & ~1;
}

template <int P1, int P2>
__host__ inline size_t plane_smem() {
  constexpr int N1 = 32 * P1, L = 32 * P2, H = L / 2 + 1;
  return (size_t)(3 * N1 * H + N1 + L + kPlaneWarps * plane_ws(L)) * sizeof(float2);
}

template <int P1, int P2, bool FIRST>
__global__ void __launch_bounds__(kPlaneThreads, 1) plane_pass_warp6(GridInfo g, const float2* __restrict__ tw1g,
                                                                    const float2* __restrict__ tw2g,
                                                                    float* __restrict__ E, float2* __restrict__ S,
                                                                    const uint8_t* __restrict__ phase,
                                                                    const float* __restrict__ dC, Control* ctl,
                                                                    LoadState* st, double* __restrict__ partials,
                                                                    double* __restrict__ hist) {
  constexpr int NV = 6, N1 = 32 * P1, L = 32 * P2, H = L / 2 + 1;
  constexpr int RS = H;                       // complex entries per tile row
  constexpr int RF = 2 * RS;                  // floats per tile row
  constexpr int WS = plane_ws(L);
  constexpr int KI = (H + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);      // [3][N1][RS]
  float* tile_f = reinterpret_cast<float*>(smem_raw);
  float2* tw1 = tile + 3 * N1 * RS;                          // N1
  float2* tw2 = tw1 + N1;                                    // L
  float2* scratch = tw2 + L;                                 // kPlaneWarps * WS
  __shared__ __align__(16) float dcs[16 * NV * NV];
  __shared__ double red[32];
  pcg::cluster_group cluster = pcg::this_cluster();
  const int rank = (int)cluster.block_rank();                // components 3 rank .. 3 rank + 2
  const int N0 = g.dims[0];
  const int pl = blockIdx.x >> 1;
  const int x0 = pl % N0, load = pl / N0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = st[load].done;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) tw1[i] = tw1g[i];
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < 16 * NV * NV; i += blockDim.x) dcs[i] = dC[i];
  float e0[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) e0[c] = (float)ctl->eps0[load][c];
  const size_t m = (size_t)g.m;
  const size_t plane_pts = (size_t)N1 * L;                   // points of the plane per component
  const size_t plane_spec = (size_t)N1 * H;                  // half-spectrum entries per component
  // component c' of this CTA: global component 3 rank + c'
  auto Ecomp = [&](int cl) { return E + ((size_t)load * NV + 3 * rank + cl) * m + (size_t)x0 * plane_pts; };
  auto Scomp = [&](int cl) {
    return S + ((size_t)load * NV + 3 * rank + cl) * (size_t)g.nrows * H + (size_t)x0 * plane_spec;
  };
  ResAcc<float> acc_d, acc_n;
  float2* ws = scratch + warp * WS;
  __syncthreads();
  // a stopped load: both CTAs of the cluster skip the work (and every cluster
  // barrier) alike, and still take part in the block count below
  if (!s_skip) {
  if (!FIRST) {
    // 1. plane of half spectra in, row k1 to slot plane_slot(k1)
    constexpr int U = 8;
    constexpr int TOT = 3 * N1 * H;
    for (int base = threadIdx.x; base < TOT; base += U * kPlaneThreads) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * kPlaneThreads;
        if (idx < TOT) {
          const int cl = idx / (N1 * H), rem = idx - cl * (N1 * H);
          v[u] = Scomp(cl)[rem];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * kPlaneThreads;
        if (idx < TOT) {
          const int cl = idx / (N1 * H), rem = idx - cl * (N1 * H);
          const int k1 = rem / H, k2 = rem - k1 * H;
          tile[(cl * N1 + plane_slot<P1>(k1)) * RS + k2] = v[u];
        }
      }
    }
    __syncthreads();
    // 2. inverse transforms along axis 1, one warp per column (c', k2)
    for (int col = warp; col < 3 * H; col += kPlaneWarps) {
      const int cl = col / H, k2 = col - cl * H;
      float2* cb = tile + cl * N1 * RS + k2;
      float2 v[1][P1];
#pragma unroll
      for (int q = 0; q < P1; ++q) v[0][q] = cb[(lane + 32 * q) * RS];
      warp_fft_inv_any<P1, 1, float>(v, tw1, lane);
#pragma unroll
      for (int j = 0; j < P1; ++j) cb[(lane + 32 * j) * RS] = v[0][j];
    }
    __syncthreads();
    // 3. inverse transforms along axis 2, two rows of one component per warp
    //    line; E_new to global memory and to the tile (as reals), residual sums
    const float scale = (float)g.inv_m;
    const bool incremental = ctl->form == 1;
    for (int pr = warp; pr < 3 * (N1 / 2); pr += kPlaneWarps) {
      const int cl = pr / (N1 / 2), xa = 2 * (pr - cl * (N1 / 2)), xb = xa + 1;
      float* Eg = Ecomp(cl);
      float ea[P2], eb[P2];
#pragma unroll
      for (int j = 0; j < P2; ++j) {
        ea[j] = Eg[(size_t)xa * L + lane + 32 * j];
        eb[j] = Eg[(size_t)xb * L + lane + 32 * j];
      }
      const float2* ra = tile + (cl * N1 + xa) * RS;
      const float2* rb = tile + (cl * N1 + xb) * RS;
#pragma unroll
      for (int i = 0; i < KI; ++i) {
        const int k = lane + 32 * i;
        if (k < H) {
          ws[wpad(k)] = ra[k];
          ws[wpad(H + k)] = rb[k];
        }
      }
      __syncwarp();
      float2 z[1][P2];
#pragma unroll
      for (int q = 0; q < P2; ++q) {
        const int k = warp_freq<P2>(lane, q);
        const bool lo = k <= L / 2;
        const int kk = lo ? k : L - k;
        float2 A = ws[wpad(kk)], B = ws[wpad(H + kk)];
        if (!lo) { A.y = -A.y; B.y = -B.y; }
        z[0][q].x = A.x - B.y;
        z[0][q].y = A.y + B.x;
      }
      __syncwarp();
      warp_fft_inv_any<P2, 1, float>(z, tw2, lane);
      float* fa = tile_f + (cl * N1 + xa) * RF;
      float* fb = tile_f + (cl * N1 + xb) * RF;
      const float e0c = e0[3 * rank + cl];
      float rd = 0.f, rn = 0.f;
#pragma unroll
      for (int j = 0; j < P2; ++j) {
        const int x = lane + 32 * j;
        float na = z[0][j].x * scale, nb = z[0][j].y * scale;
        if (incremental) { na += ea[j]; nb += eb[j]; }
        const float da = na - ea[j], db = nb - eb[j];
        const float sa = na + e0c, sb = nb + e0c;
        rd = fmaf(da, da, fmaf(db, db, rd));
        rn = fmaf(sa, sa, fmaf(sb, sb, rn));
        Eg[(size_t)xa * L + x] = na;
        Eg[(size_t)xb * L + x] = nb;
        fa[x] = na;
        fb[x] = nb;
      }
      acc_d.add(rd);
      acc_n.add(rn);
      __syncwarp();
    }
  } else {
    // start: the strain field itself goes into the tile
    constexpr int TOT = 3 * N1 * L;
    for (int idx = threadIdx.x; idx < TOT; idx += kPlaneThreads) {
      const int cl = idx / (N1 * L), rem = idx - cl * (N1 * L);
      const int x1 = rem / L, x2 = rem - x1 * L;
      tile_f[(cl * N1 + x1) * RF + x2] = Ecomp(cl)[rem];
    }
  }
  cluster.sync();   // both halves of the plane hold E_new

  // 4. constitutive stage: this CTA takes rows [rank N1/2, (rank+1) N1/2) of
  //    both CTAs' tiles; tau replaces E in place
  {
    float* own = tile_f;
    float* other = cluster.map_shared_rank(tile_f, rank ^ 1);
    const int r0 = rank * (N1 / 2);
    const uint8_t* ph = phase + (size_t)x0 * plane_pts;
    for (int idx = threadIdx.x; idx < (N1 / 2) * L; idx += kPlaneThreads) {
      const int x1 = r0 + idx / L, x2 = idx - (idx / L) * L;
      float* p[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        float* t = (c / 3 == rank) ? own : other;
        p[c] = t + ((c % 3) * N1 + x1) * RF + x2;
      }
      float e[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) e[c] = *p[c] + e0[c];
      const float* dc = dcs + ph[(size_t)x1 * L + x2] * NV * NV;
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        float t = 0.f;
#pragma unroll
        for (int b = 0; b < NV; ++b) t = fmaf(dc[a * NV + b], e[b], t);
        *p[a] = t;
      }
    }
  }
  cluster.sync();   // every stress value is in place; no remote access after this

  // 5. forward transforms along axis 2 and the split into half spectra
  for (int pr = warp; pr < 3 * (N1 / 2); pr += kPlaneWarps) {
    const int cl = pr / (N1 / 2), xa = 2 * (pr - cl * (N1 / 2)), xb = xa + 1;
    const float* fa = tile_f + (cl * N1 + xa) * RF;
    const float* fb = tile_f + (cl * N1 + xb) * RF;
    float2 z[1][P2];
#pragma unroll
    for (int j = 0; j < P2; ++j) {
      z[0][j].x = fa[lane + 32 * j];
      z[0][j].y = fb[lane + 32 * j];
    }
    warp_fft_fwd_any<P2, 1, float>(z, tw2, lane);
#pragma unroll
    for (int q = 0; q < P2; ++q) ws[wpad(warp_freq<P2>(lane, q))] = z[0][q];
    __syncwarp();
    float2* ra = tile + (cl * N1 + xa) * RS;
    float2* rb = tile + (cl * N1 + xb) * RS;
#pragma unroll
    for (int i = 0; i < KI; ++i) {
      const int k = lane + 32 * i;
      if (k < H) {
        const float2 zk = ws[wpad(k)];
        const float2 zm = ws[wpad(k == 0 ? 0 : L - k)];
        float2 A, B;
        A.x = 0.5f * (zk.x + zm.x);
        A.y = 0.5f * (zk.y - zm.y);
        B.x = 0.5f * (zk.y + zm.y);
        B.y = -0.5f * (zk.x - zm.x);
        ra[k] = A;
        rb[k] = B;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // 6. forward transforms along axis 1: natural rows in, frequency slots out
  for (int col = warp; col < 3 * H; col += kPlaneWarps) {
    const int cl = col / H, k2 = col - cl * H;
    float2* cb = tile + cl * N1 * RS + k2;
    float2 v[1][P1];
#pragma unroll
    for (int j = 0; j < P1; ++j) v[0][j] = cb[(lane + 32 * j) * RS];
    warp_fft_fwd_any<P1, 1, float>(v, tw1, lane);
#pragma unroll
    for (int q = 0; q < P1; ++q) cb[(lane + 32 * q) * RS] = v[0][q];
  }
  __syncthreads();
  // 7. plane of half spectra out, slot plane_slot(k1) to row k1
  {
    constexpr int U = 8;
    constexpr int TOT = 3 * N1 * H;
    for (int base = threadIdx.x; base < TOT; base += U * kPlaneThreads) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * kPlaneThreads;
        if (idx < TOT) {
          const int cl = idx / (N1 * H), rem = idx - cl * (N1 * H);
          const int k1 = rem / H, k2 = rem - k1 * H;
          v[u] = tile[(cl * N1 + plane_slot<P1>(k1)) * RS + k2];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * kPlaneThreads;
        if (idx < TOT) {
          const int cl = idx / (N1 * H), rem = idx - cl * (N1 * H);
          Scomp(cl)[rem] = v[u];
        }
      }
    }
  }
  }  // !s_skip
  if (FIRST) return;
  // 8. residual partials; the last block reduces per load in a fixed order and
  //    advances the per-load states (as the row passes do)
  const double d2 = block_sum_acc(acc_d, red);
  const double n2 = block_sum_acc(acc_n, red);
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
  const int bpl = 2 * N0;
  for (int load2 = 0; load2 < ctl->nload; ++load2) {
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < bpl; q += blockDim.x) {
      const size_t blk = (size_t)load2 * bpl + q;
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
