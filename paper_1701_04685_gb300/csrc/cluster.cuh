// Cluster-resident Basic-Scheme solver for 2-axis Smith grids.
//
// One thread-block cluster owns one load case for the whole solve (a task;
// the kernel's clusters take tasks from a queue until it is empty).  The
// strain E, the half spectrum and the cluster's slice of the Gamma^p table
// stay in the distributed shared memory of the cluster; only the final strain
// goes back to global memory.  Each iteration of the paper's fixed point
// (Eq. (pde_coefficients), Sec. 4) is:
//
//   column phase  CTA c gathers its half-spectrum columns [c0, c1) of every row
//                 from the owning CTAs (DSMEM loads), FFT along axis 0, Green
//                 step E^ = -Gamma^p tau^ (E^_0 = 0), inverse FFT, scatters
//                 the columns back (DSMEM stores); meanwhile the control warp
//                 of every CTA takes the stop decision of the previous
//                 iteration (the CS partial sums in a fixed order, so every
//                 CTA takes the same decision; rank 0 records r_n)
//   cluster barrier (the decision is read; a stopped load leaves the loop)
//   row phase     CTA c, for its rows [r0, r1): inverse FFT along the
//                 contiguous axis, E_new, FP64 residual partial sums (pushed
//                 to every CTA), tau = (C - C0):(E_new + eps0), forward FFT
//   cluster barrier
//
// Cluster barriers are hardware barriers (no spin loops); the iteration count
// is bounded by max_iter.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"
#include "warprow.cuh"

namespace fh {

namespace cg = cooperative_groups;

struct ClusterLayout {
  // per-CTA shared-memory layout (byte offsets), identical in every CTA
  int rows_max;   // max rows owned by one CTA
  int cols_max;   // max half-spectrum columns owned by one CTA
  int npair_max;  // complex lines of the row phase
  size_t off_E, off_S, off_G, off_ph, off_tw0, off_tw1, off_dc, off_own, off_loc, off_work, off_part, total;
};

__host__ __device__ inline int split_lo(int n, int parts, int c) { return (int)(((long long)n * c) / parts); }

// shift of the row-line padding: one spare slot per 128-byte wavefront
template <typename T> struct RowPad { static constexpr int SH = sizeof(T) == 4 ? 4 : 3; };

// g_smem = false keeps the Gamma^p slice in global memory (L2) instead of
// shared memory, for grids whose fields fill the cluster otherwise.
template <typename T>
__host__ __device__ inline ClusterLayout cluster_layout(int N0, int L, int nv, int CS, bool g_smem = true) {
  ClusterLayout c{};
  const int H = L / 2 + 1;
  c.rows_max = 0;
  c.cols_max = 0;
  for (int q = 0; q < CS; ++q) {
    c.rows_max = max(c.rows_max, split_lo(N0, CS, q + 1) - split_lo(N0, CS, q));
    c.cols_max = max(c.cols_max, split_lo(H, CS, q + 1) - split_lo(H, CS, q));
  }
  c.npair_max = (c.rows_max * nv + 1) / 2;
  const size_t ntri = (size_t)nv * (nv + 1) / 2;
  const size_t cs = sizeof(T) * 2;
  auto align = [](size_t x) { return (x + 127) & ~(size_t)127; };
  size_t o = 0;
  c.off_E = o;    o = align(o + (size_t)c.rows_max * nv * L * sizeof(T));
  c.off_S = o;    o = align(o + (size_t)c.rows_max * nv * H * cs);
  c.off_G = o;    o = align(o + (g_smem ? ntri * (size_t)N0 * c.cols_max * sizeof(T) : 0));
  c.off_ph = o;   o = align(o + (size_t)c.rows_max * L);
  c.off_tw0 = o;  o = align(o + (size_t)N0 * cs);
  c.off_tw1 = o;  o = align(o + (size_t)L * cs);
  c.off_dc = o;   o = align(o + (size_t)16 * nv * nv * sizeof(T));
  c.off_own = o;  o = align(o + (size_t)N0);
  c.off_loc = o;  o = align(o + (size_t)N0 * sizeof(short));
  c.off_part = o; o = align(o + (size_t)CS * 2 * sizeof(double));
  const size_t row_work = (size_t)2 * c.npair_max * padded_len<RowPad<T>::SH>(L) * cs;
  const size_t col_work = (size_t)2 * nv * c.cols_max * (N0 + 1) * cs;
  c.off_work = o; o = align(o + (row_work > col_work ? row_work : col_work));
  c.total = o;
  return c;
}

// threads per CTA: 8 warps for general radix plans (with the 11- and
// 13-point stages compiled in, 16 warps would cap registers at 128 and
// spill) and in FP64; 16 warps for FP32 plans of radices 2, 4, 8 only
template <typename T, bool POW2> struct ClusterThreads { static constexpr int value = (POW2 && sizeof(T) == 4) ? 512 : 256; };

// The whole solve of load `load` by the cluster this CTA belongs to.  Ends
// with a cluster barrier, after which the cluster may start another solve.
template <typename T, int NV, int CS, bool POW2>
__device__ __forceinline__ void cluster_solve_body(const GridInfo& g, const DevPlan& plan0, const DevPlan& plan1,
                                                   const cplx<T>* __restrict__ tw0g, const cplx<T>* __restrict__ tw1g,
                                                   T* __restrict__ Eg, const uint8_t* __restrict__ phase,
                                                   const T* __restrict__ dC, int nphase, const T* __restrict__ Gt,
                                                   Control* ctl, LoadState* st, double* __restrict__ hist, int g_smem,
                                                   int load) {
  constexpr int NTRI = NV * (NV + 1) / 2;
  extern __shared__ __align__(128) unsigned char sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int N0 = g.dims[0], L = g.L, H = g.H;
  const int m = (int)g.m;
  const ClusterLayout lay = cluster_layout<T>(N0, L, NV, CS, g_smem != 0);
  const int r0 = split_lo(N0, CS, rank), r1 = split_lo(N0, CS, rank + 1);
  const int c0 = split_lo(H, CS, rank), c1 = split_lo(H, CS, rank + 1);
  const int nrow = r1 - r0, ncol = c1 - c0;
  T* El = reinterpret_cast<T*>(sm + lay.off_E);                  // [row*NV + comp][L]
  cplx<T>* Sl = reinterpret_cast<cplx<T>*>(sm + lay.off_S);       // [row*NV + comp][H]
  T* Gl = reinterpret_cast<T*>(sm + lay.off_G);                  // [tri][N0][ncol]
  uint8_t* phl = sm + lay.off_ph;                                // [row][L]
  cplx<T>* tw0 = reinterpret_cast<cplx<T>*>(sm + lay.off_tw0);
  cplx<T>* tw1 = reinterpret_cast<cplx<T>*>(sm + lay.off_tw1);
  T* dcs = reinterpret_cast<T*>(sm + lay.off_dc);
  uint8_t* own = sm + lay.off_own;                                // owner rank of row n
  short* loc = reinterpret_cast<short*>(sm + lay.off_loc);        // local row index in the owner
  double* part = reinterpret_cast<double*>(sm + lay.off_part);    // [CS][2], used in rank 0
  constexpr int PS = RowPad<T>::SH;
  const int Lp = padded_len<PS>(L);      // padded row-line stride
  const int N0p = N0 + 1;                // odd column-line stride
  cplx<T>* W0 = reinterpret_cast<cplx<T>*>(sm + lay.off_work);
  cplx<T>* W1 = reinterpret_cast<cplx<T>*>(sm + lay.off_work) + (size_t)lay.npair_max * Lp;
  cplx<T>* X0 = W0;
  cplx<T>* X1 = W0 + (size_t)NV * lay.cols_max * N0p;
  const size_t Ebase = (size_t)load * NV * g.m;
  const FDiv fL = make_fdiv(L), fH = make_fdiv(H), fN0 = make_fdiv(N0), fnc = make_fdiv(ncol > 0 ? ncol : 1);

  // ---- stage everything this CTA keeps for the whole solve
  for (int i = threadIdx.x; i < N0; i += blockDim.x) tw0[i] = tw0g[i];
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw1[i] = tw1g[i];
  for (int i = threadIdx.x; i < nphase * NV * NV; i += blockDim.x) dcs[i] = dC[i];
  for (int q = 0; q < CS; ++q) {
    const int a = split_lo(N0, CS, q), b = split_lo(N0, CS, q + 1);
    for (int n = a + (int)threadIdx.x; n < b; n += blockDim.x) {
      own[n] = (uint8_t)q;
      loc[n] = (short)(n - a);
    }
  }
  for (int i = threadIdx.x; i < nrow * L; i += blockDim.x) {
    const int r = fdiv(i, fL), x = i - r * L;
    const int gi = (r0 + r) * L + x;
    if (!FH_IN(CK_CLUSTER, gi, m)) continue;
    phl[i] = phase[gi];
    if (!FH_IN(CK_CLUSTER, phl[i], nphase)) phl[i] = 0;
#pragma unroll
    for (int c = 0; c < NV; ++c) El[(r * NV + c) * L + x] = Eg[Ebase + (size_t)c * m + gi];
  }
  for (int i = threadIdx.x; g_smem && i < NTRI * N0 * ncol; i += blockDim.x) {
    const int t2 = fdiv(i, fnc);
    const int j = i - t2 * ncol;
    const int t = fdiv(t2, fN0);
    const int n = t2 - t * N0;
    if (!FH_IN(CK_CLUSTER, (long long)t * g.nhalf + (long long)n * H + c0 + j, (long long)NTRI * g.nhalf)) continue;
    Gl[i] = Gt[(size_t)t * g.nhalf + (size_t)n * H + c0 + j];
  }
  T e0[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) e0[c] = (T)ctl->eps0[load][c];
  LoadState s = st[load];
  const double tol = ctl->tol;
  const int max_iter = ctl->max_iter;
  const int stall_window = ctl->stall_window;
  const bool incremental = ctl->form == 1;
  const T scale = (T)g.inv_m;
  __syncthreads();

  // ---- row phase: (optional inverse FFT + E update + residual) + stress + forward FFT
  auto row_phase = [&](bool with_inverse, ResAcc<T>& acc_d, ResAcc<T>& acc_n) {
    const int nreal = nrow * NV;
    const int npair = (nreal + 1) >> 1;
    cplx<T>* Z = W0;
    cplx<T>* Zo = W1;
    if (with_inverse) {
      // rebuild Z = A + i B per line pair in natural order (conflict-free
      // reads of the unpadded half spectra), then the inverse transform
      for (int idx = threadIdx.x; idx < npair * L; idx += blockDim.x) {
        const int p = fdiv(idx, fL), k = idx - p * L;
        const int fa = 2 * p, fb = 2 * p + 1;
        const bool lo = k <= (L >> 1);
        const int kk = lo ? k : L - k;
        cplx<T> A = Sl[fa * H + kk];
        cplx<T> B;
        B.x = T(0); B.y = T(0);
        if (fb < nreal) B = Sl[fb * H + kk];
        if (!lo) { A.y = -A.y; B.y = -B.y; }
        cplx<T> z;
        z.x = A.x - B.y;
        z.y = A.y + B.x;
        W0[p * Lp + padi<PS>(k)] = z;
      }
      __syncthreads();
      bool warp_done = false;   // FP32, power-of-two rows of 32..512 points: one warp per line, in place
      if constexpr (POW2 && sizeof(T) == 4) warp_done = warp_lines_any<+1, PS, T>(W0, npair, Lp, L, tw1, threadIdx.x, blockDim.x);
      Z = warp_done ? W0 : fft_lines_pp<+1, T, PS, POW2>(W0, W1, npair, Lp, plan1, tw1);
      Zo = (Z == W0) ? W1 : W0;
    }
    // E update, residual sums and stress, two points per thread at a time
    // with every shared-memory load of both issued before any store
    for (int base = threadIdx.x; base < nrow * L; base += 2 * blockDim.x) {
      T en[2][NV], eo[2][NV];
      int ph[2], rr[2], xx[2];
      bool ok[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int idx = base + u * blockDim.x;
        ok[u] = idx < nrow * L;
        const int id = ok[u] ? idx : 0;
        rr[u] = fdiv(id, fL);
        xx[u] = id - rr[u] * L;
        ph[u] = phl[id];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const int f = rr[u] * NV + c;
          eo[u][c] = El[f * L + xx[u]];
          if (with_inverse) {
            const cplx<T> zz = Z[(f >> 1) * Lp + padi<PS>(xx[u])];
            en[u][c] = ((f & 1) ? zz.y : zz.x) * scale;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!ok[u]) continue;
        const int r = rr[u], x = xx[u];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          if (with_inverse) {
            if (incremental) en[u][c] += eo[u][c];
            acc_d.add_sq(en[u][c] - eo[u][c]);
            acc_n.add_sq(en[u][c] + e0[c]);
            El[(r * NV + c) * L + x] = en[u][c];
          } else {
            en[u][c] = eo[u][c];
          }
        }
        const T* dc = dcs + ph[u] * NV * NV;
#pragma unroll
        for (int a = 0; a < NV; ++a) {
          T t = T(0);
#pragma unroll
          for (int b = 0; b < NV; ++b) t += dc[a * NV + b] * (en[u][b] + e0[b]);
          const int f = r * NV + a;
          if (f & 1) Z[(f >> 1) * Lp + padi<PS>(x)].y = t;
          else Z[(f >> 1) * Lp + padi<PS>(x)].x = t;
        }
      }
    }
    if (nreal & 1)
      for (int x = threadIdx.x; x < L; x += blockDim.x) Z[(npair - 1) * Lp + padi<PS>(x)].y = T(0);
    __syncthreads();
    // FP32 power-of-two rows: forward transform and split by the owning warp
    bool fused = false;
    if constexpr (POW2 && sizeof(T) == 4)
      fused = warp_rows_fwd_split_any<PS, T>(Z, npair, Lp, L, Sl, H, nreal, tw1, threadIdx.x, blockDim.x);
    if (!fused) {
      cplx<T>* Zf = fft_lines_pp<-1, T, PS, POW2>(Z, Zo, npair, Lp, plan1, tw1);
      for (int idx = threadIdx.x; idx < npair * H; idx += blockDim.x) {
        const int p = fdiv(idx, fH), k = idx - p * H;
        const cplx<T> zk = Zf[p * Lp + padi<PS>(k)];
        const cplx<T> zm = Zf[p * Lp + padi<PS>(k == 0 ? 0 : L - k)];
        cplx<T> A, B;
        A.x = T(0.5) * (zk.x + zm.x);
        A.y = T(0.5) * (zk.y - zm.y);
        B.x = T(0.5) * (zk.y + zm.y);
        B.y = T(-0.5) * (zk.x - zm.x);
        Sl[(2 * p) * H + k] = A;
        if (2 * p + 1 < nreal) Sl[(2 * p + 1) * H + k] = B;
      }
    }
  };

  // ---- column phase: gather columns over DSMEM, FFT, Green, inverse FFT,
  // scatter; run by the worker threads 0 .. nwork-1 only (the last warp is
  // the control warp, see the iteration loop), synchronised on a named barrier
  const int nwork = (int)blockDim.x - 32;
  const int tid = (int)threadIdx.x;
  auto col_phase = [&]() {
    const int nl = NV * ncol;
    for (int idx = tid; idx < NV * N0 * ncol; idx += nwork) {
      const int t = fdiv(idx, fnc);
      const int j = idx - t * ncol;
      const int c = fdiv(t, fN0);
      const int n = t - c * N0;
      const cplx<T>* rem = cluster.map_shared_rank(Sl, (int)own[n]);
      X0[(c * ncol + j) * N0p + n] = rem[((int)loc[n] * NV + c) * H + c0 + j];
    }
    team_sync(nwork);
    bool warp_done = false;   // FP32, power-of-two columns of 32..512 points: one warp per line, in place
    if constexpr (POW2 && sizeof(T) == 4) warp_done = warp_lines_any<-1, 0, T>(X0, nl, N0p, N0, tw0, tid, nwork);
    cplx<T>* Xf = warp_done ? X0 : fft_lines_pp<-1, T, 0, POW2>(X0, X1, nl, N0p, plan0, tw0, tid, nwork);
    for (int idx = tid; idx < N0 * ncol; idx += nwork) {
      const int n = fdiv(idx, fnc);
      const int j = idx - n * ncol;
      cplx<T> tv[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) tv[c] = Xf[(c * ncol + j) * N0p + n];
      const bool zero = (n == 0 && c0 + j == 0);
      T gm[NTRI];
#pragma unroll
      for (int t = 0; t < NTRI; ++t)
        gm[t] = g_smem ? Gl[(t * N0 + n) * ncol + j] : Gt[(size_t)t * g.nhalf + (size_t)n * H + c0 + j];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        T re = T(0), im = T(0);
#pragma unroll
        for (int b = 0; b < NV; ++b) {
          const int lo = a < b ? a : b, hi = a < b ? b : a;
          const T gv = gm[lo * NV - (lo * (lo - 1)) / 2 + (hi - lo)];
          re -= gv * tv[b].x;
          im -= gv * tv[b].y;
        }
        cplx<T> e;
        e.x = zero ? T(0) : re;
        e.y = zero ? T(0) : im;
        Xf[(a * ncol + j) * N0p + n] = e;
      }
    }
    team_sync(nwork);
    if constexpr (POW2 && sizeof(T) == 4) warp_done = warp_lines_any<+1, 0, T>(Xf, nl, N0p, N0, tw0, tid, nwork);
    cplx<T>* Xi = warp_done ? Xf : fft_lines_pp<+1, T, 0, POW2>(Xf, Xf == X0 ? X1 : X0, nl, N0p, plan0, tw0, tid, nwork);
    for (int idx = tid; idx < NV * N0 * ncol; idx += nwork) {
      const int t = fdiv(idx, fnc);
      const int j = idx - t * ncol;
      const int c = fdiv(t, fN0);
      const int n = t - c * N0;
      cplx<T>* rem = cluster.map_shared_rank(Sl, (int)own[n]);
      rem[((int)loc[n] * NV + c) * H + c0 + j] = Xi[(c * ncol + j) * N0p + n];
    }
  };

  // ---- initial stress and forward transform of the rows
  {
    ResAcc<T> a, b;
    row_phase(false, a, b);
  }
  cluster.sync();
  // Iteration n: the workers run the column phase of n while the control
  // warp (the last warp) sums the residual partials of n - 1 and takes the
  // stop decision; the first cluster barrier publishes the decision before E
  // is touched.  The column phase only rewrites the half spectra (scratch
  // rebuilt from E at the start of every solve), so the one that follows the
  // last iteration is harmless.
  __shared__ int s_done;
  __shared__ double2 red2[32];
  const int hist_cap = ctl->hist_cap;
  const bool control = tid >= nwork;
  if (tid == 0) s_done = (s.done || max_iter <= 0) ? 1 : 0;
  __syncthreads();
  for (int it = 0;; ++it) {
    if (!control) {
      col_phase();
    } else if (it > 0) {
      // every CTA sums the CS partials of iteration it - 1 in the same fixed
      // order and takes the same decision
      const int lane = tid - nwork;
      double a = lane < CS ? part[2 * lane] : 0.0, b = lane < CS ? part[2 * lane + 1] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        update_state(s, a, b, tol, max_iter, stall_window);
        if (rank == 0 && s.iter <= hist_cap) hist[(size_t)load * hist_cap + (s.iter - 1)] = s.r;
        s_done = s.done;
      }
    }
    cluster.sync();
    if (s_done) break;
    ResAcc<T> acc_d, acc_n;
    row_phase(true, acc_d, acc_n);
    // this CTA's partial sums, pushed into every CTA's `part` (lane q of
    // warp 0 stores into CTA q), so that after the barrier all reads are local
    double d2 = 0.0, n2 = 0.0;
    block_sum_pair(acc_d, acc_n, red2, d2, n2);
    if (tid < CS) {
      double* dst = cluster.map_shared_rank(part, tid);
      dst[2 * rank] = d2;
      dst[2 * rank + 1] = n2;
    }
    cluster.sync();
  }
  // ---- results
  for (int i = threadIdx.x; i < nrow * L; i += blockDim.x) {
    const int r = fdiv(i, fL), x = i - r * L;
    if (!FH_IN(CK_CLUSTER, (r0 + r) * L + x, m)) continue;
#pragma unroll
    for (int c = 0; c < NV; ++c) Eg[Ebase + (size_t)c * m + (r0 + r) * L + x] = El[(r * NV + c) * L + x];
  }
  if (rank == 0 && tid == nwork) st[load] = s;   // the control lane holds the full state
  cluster.sync();  // keep every CTA's shared memory alive until remote accesses are done
}

// One solve of one load of one solver: the unit of work of the cluster kernel.
struct ClusterTask {
  GridInfo g;
  DevPlan plan0, plan1;
  const void* tw0;
  const void* tw1;
  void* E;
  const uint8_t* phase;
  const void* dC;
  const void* Gt;
  Control* ctl;
  LoadState* st;
  double* hist;
  int nphase;
  int g_smem;
  int load;
  int pad_;
};

// The cluster kernel: resident clusters take tasks from `tasks` until none is
// left.  A single solve queues its own loads (one cluster each); a batched
// solve queues every load of every solver of the batch, largest pattern first,
// on as many clusters as fit.  Rank 0 of a cluster draws the next index with
// one atomic and the other CTAs read it from rank 0's shared memory; clusters
// never wait on one another.  The task is staged in shared memory.
template <typename T, int NV, int CS, bool POW2>
__global__ void __launch_bounds__(ClusterThreads<T, POW2>::value, 1)
cluster_solve_2d(const ClusterTask* __restrict__ tasks, int ntasks, unsigned int* next) {
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ int s_task;
  __shared__ __align__(16) ClusterTask t;
  for (;;) {
    if (cluster.block_rank() == 0 && threadIdx.x == 0) s_task = (int)atomicAdd(next, 1u);
    cluster.sync();
    const int task = *cluster.map_shared_rank(&s_task, 0);
    if (task < ntasks) {
      const int* src = reinterpret_cast<const int*>(tasks + task);
      int* dst = reinterpret_cast<int*>(&t);
      for (int i = threadIdx.x; i < (int)(sizeof(ClusterTask) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    cluster.sync();   // every CTA holds the index (and the task) before rank 0 draws the next one
    if (task >= ntasks) return;
    cluster_solve_body<T, NV, CS, POW2>(t.g, t.plan0, t.plan1, static_cast<const cplx<T>*>(t.tw0),
                                        static_cast<const cplx<T>*>(t.tw1), static_cast<T*>(t.E), t.phase,
                                        static_cast<const T*>(t.dC), t.nphase, static_cast<const T*>(t.Gt), t.ctl,
                                        t.st, t.hist, t.g_smem, t.load);
  }
}

}  // namespace fh
