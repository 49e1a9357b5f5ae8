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
//      as the real and imaginary part of one complex line), then a streaming
//      loop over the plane: the strain update E_new, the Cauchy-residual sums,
//      E_new written to global memory,
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
// together and coalescing is unaffected.  Every warp transforms the three
// components of one column (axis 1) or one row pair (axis 2) together, for
// instruction-level parallelism with a single CTA per SM; the plane comes in
// through asynchronous 8-byte copies, and the forward row transform stages
// its spectrum in the two tile rows it will overwrite (no scratch memory).
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

template <int P1, int P2>
__host__ inline size_t plane_smem() {
  constexpr int N1 = 32 * P1, L = 32 * P2, H = L / 2 + 1;
  return (size_t)(3 * N1 * H + N1 + L) * sizeof(float2);
}

// 8-byte asynchronous global -> shared copy (both addresses 8-byte aligned)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// complex slot f (0 <= f < 2 H) of the two tile rows a, b read as one line:
// row a holds slots 0 .. H-1, row b the rest (used as the forward split's
// staging line: L <= 2 H - 2 entries)
__device__ __forceinline__ float2* pair_slot(float2* ra, float2* rb, int f, int H) { return f < H ? ra + f : rb + (f - H); }

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
  constexpr int KI = (H + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);      // [3][N1][RS]
  float* tile_f = reinterpret_cast<float*>(smem_raw);
  float2* tw1 = tile + 3 * N1 * RS;                          // N1
  float2* tw2 = tw1 + N1;                                    // L
  __shared__ __align__(16) float dcs[16 * NV * NV];
  __shared__ double red[32];
  __shared__ int s_skip;
  pcg::cluster_group cluster = pcg::this_cluster();
  const int rank = (int)cluster.block_rank();                // components 3 rank .. 3 rank + 2
  const int N0 = g.dims[0];
  const int pl = blockIdx.x >> 1;
  const int x0 = pl % N0, load = pl / N0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_skip = st[load].done;
  for (int i = threadIdx.x; i < N1; i += blockDim.x) tw1[i] = tw1g[i];
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < 16 * NV * NV; i += blockDim.x) dcs[i] = dC[i];
  float e0[NV], e0own[3];
#pragma unroll
  for (int c = 0; c < NV; ++c) e0[c] = (float)ctl->eps0[load][c];
#pragma unroll
  for (int cl = 0; cl < 3; ++cl) e0own[cl] = rank ? e0[3 + cl] : e0[cl];
  const size_t m = (size_t)g.m;
  const size_t plane_pts = (size_t)N1 * L;                   // points of the plane per component
  const size_t plane_spec = (size_t)N1 * H;                  // half-spectrum entries per component
  // component c' of this CTA: global component 3 rank + c'
  auto Ecomp = [&](int cl) { return E + ((size_t)load * NV + 3 * rank + cl) * m + (size_t)x0 * plane_pts; };
  auto Scomp = [&](int cl) {
    return S + ((size_t)load * NV + 3 * rank + cl) * (size_t)g.nrows * H + (size_t)x0 * plane_spec;
  };
  ResAcc<float> acc_d, acc_n;
  __syncthreads();
  // a stopped load: both CTAs of the cluster skip the work (and every cluster
  // barrier) alike, and still take part in the block count below
  if (!s_skip) {
    if (!FIRST) {
      // 1. plane of half spectra in (asynchronous copies), row k1 to slot plane_slot(k1)
      for (int idx = threadIdx.x; idx < 3 * N1 * H; idx += kPlaneThreads) {
        const int cl = idx / (N1 * H), rem = idx - cl * (N1 * H);
        const int k1 = rem / H, k2 = rem - k1 * H;
        cp_async8(tile + (cl * N1 + plane_slot<P1>(k1)) * RS + k2, Scomp(cl) + rem);
      }
      cp_async_wait_all();
      __syncthreads();
      // 2. inverse transforms along axis 1: warp per k2, the three components together
      for (int k2 = warp; k2 < H; k2 += kPlaneWarps) {
        float2 v[3][P1];
#pragma unroll
        for (int cl = 0; cl < 3; ++cl)
#pragma unroll
          for (int q = 0; q < P1; ++q) v[cl][q] = tile[(cl * N1 + lane + 32 * q) * RS + k2];
        warp_fft_inv_any<P1, 3, float>(v, tw1, lane);
#pragma unroll
        for (int cl = 0; cl < 3; ++cl)
#pragma unroll
          for (int j = 0; j < P1; ++j) tile[(cl * N1 + lane + 32 * j) * RS + k2] = v[cl][j];
      }
      __syncthreads();
      // 3a. inverse transforms along axis 2: warp per row pair, three components
      //     (two real rows as one complex line each); E_new to the tile as reals
      const float scale = (float)g.inv_m;
      for (int pr = warp; pr < N1 / 2; pr += kPlaneWarps) {
        const int xa = 2 * pr, xb = xa + 1;
        float2 z[3][P2];
#pragma unroll
        for (int cl = 0; cl < 3; ++cl) {
          const float2* ra = tile + (cl * N1 + xa) * RS;
          const float2* rb = tile + (cl * N1 + xb) * RS;
#pragma unroll
          for (int q = 0; q < P2; ++q) {
            const int k = warp_freq<P2>(lane, q);
            const bool lo = k <= L / 2;
            const int kk = lo ? k : L - k;
            float2 A = ra[kk], B = rb[kk];
            if (!lo) { A.y = -A.y; B.y = -B.y; }
            z[cl][q].x = A.x - B.y;
            z[cl][q].y = A.y + B.x;
          }
        }
        __syncwarp();
        warp_fft_inv_any<P2, 3, float>(z, tw2, lane);
#pragma unroll
        for (int cl = 0; cl < 3; ++cl) {
          float* fa = tile_f + (cl * N1 + xa) * RF;
          float* fb = tile_f + (cl * N1 + xb) * RF;
#pragma unroll
          for (int j = 0; j < P2; ++j) {
            fa[lane + 32 * j] = z[cl][j].x * scale;
            fb[lane + 32 * j] = z[cl][j].y * scale;
          }
        }
        __syncwarp();
      }
      __syncthreads();
      // 3b. E_new against E_old (global): residual sums, E_new to global memory;
      //     the variational form adds the update to E_old
      const bool incremental = ctl->form == 1;
      constexpr int U = 4;
      constexpr int TOT = 3 * N1 * L;
      for (int base = threadIdx.x; base < TOT; base += U * kPlaneThreads) {
        float eo[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base + u * kPlaneThreads;
          eo[u] = 0.f;
          if (idx < TOT) {
            const int cl = idx / (N1 * L), rem = idx - cl * (N1 * L);
            eo[u] = Ecomp(cl)[rem];
          }
        }
        float rd = 0.f, rn = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = base + u * kPlaneThreads;
          if (idx < TOT) {
            const int cl = idx / (N1 * L), rem = idx - cl * (N1 * L);
            const int x1 = rem / L, x2 = rem - x1 * L;
            float* tp = tile_f + (cl * N1 + x1) * RF + x2;
            float en = *tp;
            if (incremental) {
              en += eo[u];
              *tp = en;
            }
            const float dd = en - eo[u], nn = en + (cl == 0 ? e0own[0] : cl == 1 ? e0own[1] : e0own[2]);
            rd = fmaf(dd, dd, rd);
            rn = fmaf(nn, nn, rn);
            Ecomp(cl)[rem] = en;
          }
        }
        acc_d.add(rd);
        acc_n.add(rn);
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
    //    both CTAs' tiles, two points per thread at a time, every load before
    //    any store; tau replaces E in place
    {
      float* own = tile_f;
      float* other = cluster.map_shared_rank(tile_f, rank ^ 1);
      float* base[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) base[c] = ((c / 3 == rank) ? own : other) + (c % 3) * N1 * RF;
      const int r0 = rank * (N1 / 2);
      const uint8_t* ph = phase + (size_t)x0 * plane_pts;
      constexpr int NPT = (N1 / 2) * L;
      constexpr int V = 2;
      for (int i0 = threadIdx.x; i0 < NPT; i0 += V * kPlaneThreads) {
        float e[V][NV];
        int off[V], pid[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int idx = i0 + v * kPlaneThreads;
          const int x1 = r0 + idx / L, x2 = idx - (idx / L) * L;
          off[v] = x1 * RF + x2;
          pid[v] = idx < NPT ? ph[(size_t)x1 * L + x2] : 0;
#pragma unroll
          for (int c = 0; c < NV; ++c) e[v][c] = idx < NPT ? base[c][off[v]] + e0[c] : 0.f;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (i0 + v * kPlaneThreads >= NPT) continue;
          const float* dc = dcs + pid[v] * NV * NV;
#pragma unroll
          for (int a = 0; a < NV; ++a) {
            float t = 0.f;
#pragma unroll
            for (int b = 0; b < NV; ++b) t = fmaf(dc[a * NV + b], e[v][b], t);
            base[a][off[v]] = t;
          }
        }
      }
    }
    cluster.sync();   // every stress value is in place; no remote access after this

    // 5. forward transforms along axis 2 (warp per row pair, three components),
    //    the spectrum staged in the pair's own two tile rows, then split into
    //    the two half spectra
    for (int pr = warp; pr < N1 / 2; pr += kPlaneWarps) {
      const int xa = 2 * pr, xb = xa + 1;
      float2 z[3][P2];
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) {
        const float* fa = tile_f + (cl * N1 + xa) * RF;
        const float* fb = tile_f + (cl * N1 + xb) * RF;
#pragma unroll
        for (int j = 0; j < P2; ++j) {
          z[cl][j].x = fa[lane + 32 * j];
          z[cl][j].y = fb[lane + 32 * j];
        }
      }
      warp_fft_fwd_any<P2, 3, float>(z, tw2, lane);
      __syncwarp();   // every lane has read its reals before the rows are overwritten
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) {
        float2* ra = tile + (cl * N1 + xa) * RS;
        float2* rb = tile + (cl * N1 + xb) * RS;
#pragma unroll
        for (int q = 0; q < P2; ++q) *pair_slot(ra, rb, warp_freq<P2>(lane, q), H) = z[cl][q];
      }
      __syncwarp();
      float2 zk[3][KI], zm[3][KI];
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) {
        float2* ra = tile + (cl * N1 + xa) * RS;
        float2* rb = tile + (cl * N1 + xb) * RS;
#pragma unroll
        for (int i = 0; i < KI; ++i) {
          const int k = lane + 32 * i;
          if (k < H) {
            zk[cl][i] = *pair_slot(ra, rb, k, H);
            zm[cl][i] = *pair_slot(ra, rb, k == 0 ? 0 : L - k, H);
          }
        }
      }
      __syncwarp();   // the staged spectrum is read before the half spectra replace it
#pragma unroll
      for (int cl = 0; cl < 3; ++cl) {
        float2* ra = tile + (cl * N1 + xa) * RS;
        float2* rb = tile + (cl * N1 + xb) * RS;
#pragma unroll
        for (int i = 0; i < KI; ++i) {
          const int k = lane + 32 * i;
          if (k < H) {
            float2 A, B;
            A.x = 0.5f * (zk[cl][i].x + zm[cl][i].x);
            A.y = 0.5f * (zk[cl][i].y - zm[cl][i].y);
            B.x = 0.5f * (zk[cl][i].y + zm[cl][i].y);
            B.y = -0.5f * (zk[cl][i].x - zm[cl][i].x);
            ra[k] = A;
            rb[k] = B;
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
    // 6. forward transforms along axis 1: natural rows in, frequency slots out
    for (int k2 = warp; k2 < H; k2 += kPlaneWarps) {
      float2 v[3][P1];
#pragma unroll
      for (int cl = 0; cl < 3; ++cl)
#pragma unroll
        for (int j = 0; j < P1; ++j) v[cl][j] = tile[(cl * N1 + lane + 32 * j) * RS + k2];
      warp_fft_fwd_any<P1, 3, float>(v, tw1, lane);
#pragma unroll
      for (int cl = 0; cl < 3; ++cl)
#pragma unroll
        for (int q = 0; q < P1; ++q) tile[(cl * N1 + lane + 32 * q) * RS + k2] = v[cl][q];
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
