// Fourier-neural-operator start predictor: forward, backward and Adam kernels.
//
// The network (not part of the paper; it supplies the starting strain of the
// paper's fixed point) maps input channels x on an N^3 grid to the strain
// fluctuation y:
//   v_0 = P x + p;  u_l = W_l v_l + w_l + K_l v_l,  v_{l+1} = gelu(u_l);  y = Q v_L + q,
// with the spectral convolution restricted to kx, ky in {-m..m-1}, kz in {0..m-1}:
//   v^(k) = sum_x v(x) e^{-2 pi i k.x/N},  c = R_l(k) v^(k),
//   (K v)(x) = N^-3 Re sum_k w(kz) c(k) e^{+2 pi i k.x/N},  w(0) = 1, w(kz>0) = 2.
// Only 4 m^3 of the N^3 modes are kept, so each transform is a small dense
// DFT contraction along one axis at a time (z, then y, then x), with the
// twiddles in shared memory.  R and W are used in BF16 (stored from FP32
// master weights), every product is accumulated in FP32.
//
// Layouts: activations [B][C][N^3] (z fastest); spectral coefficients
// [B][C][mode], mode = (ax * 2m + ay) * m + kz; R [layer][mode][out][in].

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.hpp"
#include "fno_tc.cuh"

namespace {

constexpr int kT = 256;

struct FnoDims {
  int N, cin, cout, W, m, L;
  int N3;      // N^3
  int NM;      // (2m)^2 m modes
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// twiddle e^{sign 2 pi i t / N}, t = 0..N-1, from the FP32 table of e^{-2 pi i t/N}
__device__ __forceinline__ float2 twd(const float2* tw, int t, int sign) {
  float2 w = tw[t];
  if (sign > 0) w.y = -w.y;
  return w;
}

__device__ __forceinline__ int kx_of(int a, int m, int N) { return a < m ? a : N - 2 * m + a; }  // index mod N

// ---------------------------------------------------------------- transforms
// truncated forward DFT along z (real -> kz < m) and y (-> 2m rows), one block per (b, c, x)
__global__ void __launch_bounds__(kT) k_dft_zy(FnoDims d, const float* __restrict__ v, float2* __restrict__ Yy,
                                                const float2* __restrict__ twg, int C) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = d.N, m = d.m;
  float* slab = reinterpret_cast<float*>(sm);                // N*N
  float2* tw = reinterpret_cast<float2*>(slab + N * N);      // N
  float2* Yz = tw + N;                                       // N*m  [y][kz]
  const long long bcx = blockIdx.x;                          // (b*C + c)*N + x
  const float* src = v + bcx * N * N;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) slab[i] = src[i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * m; idx += blockDim.x) {
    const int y = idx / m, kz = idx - y * m;
    float2 acc = make_float2(0.f, 0.f);
    int t = 0;
    for (int z = 0; z < N; ++z) {
      const float s = slab[y * N + z];
      const float2 w = tw[t];
      acc.x += s * w.x;
      acc.y += s * w.y;
      t += kz;
      if (t >= N) t -= N;
    }
    Yz[idx] = acc;
  }
  __syncthreads();
  float2* dst = Yy + bcx * (2 * m * m);
  for (int idx = threadIdx.x; idx < 2 * m * m; idx += blockDim.x) {
    const int a = idx / m, kz = idx - a * m;
    const int ky = kx_of(a, m, N);
    float2 acc = make_float2(0.f, 0.f);
    int t = 0;
    for (int y = 0; y < N; ++y) {
      const float2 p = cmulf(Yz[y * m + kz], tw[t]);
      acc.x += p.x;
      acc.y += p.y;
      t += ky;
      if (t >= N) t -= N;
    }
    dst[idx] = acc;
  }
}

// truncated forward DFT along x, one block per (b, c, a); out[b][c][mode] scaled by
// `scale` and, when `wz` is set, by w(kz)
__global__ void __launch_bounds__(kT) k_dft_x(FnoDims d, const float2* __restrict__ Yy, float2* __restrict__ out,
                                               const float2* __restrict__ twg, int C, float scale, int wz) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = d.N, m = d.m, m2 = 2 * m;
  float2* tw = reinterpret_cast<float2*>(sm);
  float2* Yx = tw + N;                       // [x][kz]
  const int a = blockIdx.x % m2;
  const long long bc = blockIdx.x / m2;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < N * m; i += blockDim.x) {
    const int x = i / m, kz = i - x * m;
    Yx[i] = Yy[((bc * N + x) * m2 + a) * m + kz];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m2 * m; idx += blockDim.x) {
    const int ax = idx / m, kz = idx - ax * m;
    const int kx = kx_of(ax, m, N);
    float2 acc = make_float2(0.f, 0.f);
    int t = 0;
    for (int x = 0; x < N; ++x) {
      const float2 p = cmulf(Yx[x * m + kz], tw[t]);
      acc.x += p.x;
      acc.y += p.y;
      t += kx;
      if (t >= N) t -= N;
    }
    const float s = scale * ((wz && kz > 0) ? 2.f : 1.f);
    out[bc * d.NM + (ax * m2 + a) * m + kz] = make_float2(acc.x * s, acc.y * s);
  }
}

// truncated inverse DFT along x, one block per (b, c, a): Ix[b][c][x][a][kz]
__global__ void __launch_bounds__(kT) k_idft_x(FnoDims d, const float2* __restrict__ cf, float2* __restrict__ Ix,
                                                const float2* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = d.N, m = d.m, m2 = 2 * m;
  float2* tw = reinterpret_cast<float2*>(sm);
  float2* cx = tw + N;                        // [ax][kz]
  const int a = blockIdx.x % m2;
  const long long bc = blockIdx.x / m2;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < m2 * m; i += blockDim.x) {
    const int ax = i / m, kz = i - ax * m;
    cx[i] = cf[bc * d.NM + (ax * m2 + a) * m + kz];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * m; idx += blockDim.x) {
    const int x = idx / m, kz = idx - x * m;
    float2 acc = make_float2(0.f, 0.f);
    for (int ax = 0; ax < m2; ++ax) {
      const int kx = kx_of(ax, m, N);
      const float2 p = cmulf(cx[ax * m + kz], twd(tw, (kx * x) % N, +1));
      acc.x += p.x;
      acc.y += p.y;
    }
    Ix[((bc * N + x) * m2 + a) * m + kz] = acc;
  }
}

// truncated inverse DFT along y and z, one block per (b, c, x):
// out(x,y,z) (+)= scale * sum_kz wk(kz) Re( sum_a Ix[a][kz] e^{+i ky y} e^{+i kz z} )
__global__ void __launch_bounds__(kT) k_idft_yz(FnoDims d, const float2* __restrict__ Ix, float* __restrict__ out,
                                                 const float2* __restrict__ twg, float scale, int wz, int accumulate) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = d.N, m = d.m, m2 = 2 * m;
  float2* tw = reinterpret_cast<float2*>(sm);
  float2* Ia = tw + N;            // [a][kz]
  float2* Iy = Ia + m2 * m;       // [y][kz]
  const long long bcx = blockIdx.x;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < m2 * m; i += blockDim.x) Ia[i] = Ix[bcx * m2 * m + i];
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * m; idx += blockDim.x) {
    const int y = idx / m, kz = idx - y * m;
    float2 acc = make_float2(0.f, 0.f);
    for (int a = 0; a < m2; ++a) {
      const int ky = kx_of(a, m, N);
      const float2 p = cmulf(Ia[a * m + kz], twd(tw, (ky * y) % N, +1));
      acc.x += p.x;
      acc.y += p.y;
    }
    const float s = scale * ((wz && kz > 0) ? 2.f : 1.f);
    Iy[idx] = make_float2(acc.x * s, acc.y * s);
  }
  __syncthreads();
  float* dst = out + bcx * N * N;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int y = idx / N, z = idx - y * N;
    float acc = 0.f;
    int t = 0;
    for (int kz = 0; kz < m; ++kz) {
      // Re(c e^{+i theta}) = c.x cos - c.y sin, with tw = (cos, -sin)
      const float2 w = tw[t];
      const float2 c = Iy[y * m + kz];
      acc += c.x * w.x + c.y * w.y;
      t += z;
      if (t >= N) t -= N;
    }
    dst[idx] = accumulate ? dst[idx] + acc : acc;
  }
}

// ---------------------------------------------------------------- channel mixing
// out[b][o][k] = sum_i R[k][o][i] in[b][i][k]; blocks of KC modes, all batch items
constexpr int KC = 8;
__global__ void __launch_bounds__(kT) k_mix(FnoDims d, int B, const __nv_bfloat162* __restrict__ R,
                                             const float2* __restrict__ in, float2* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int W = d.W, NM = d.NM;
  const int k0 = blockIdx.x * KC;
  const int nk = min(KC, NM - k0);
  float2* Rs = reinterpret_cast<float2*>(sm);         // [kc][o][i]
  float2* xs = Rs + KC * W * W;                        // [kc][i]
  for (int i = threadIdx.x; i < nk * W * W; i += blockDim.x) {
    const __nv_bfloat162 r = R[(size_t)k0 * W * W + i];
    Rs[i] = make_float2(__bfloat162float(r.x), __bfloat162float(r.y));
  }
  for (int b = 0; b < B; ++b) {
    __syncthreads();
    for (int i = threadIdx.x; i < nk * W; i += blockDim.x) {
      const int kc = i / W, c = i - kc * W;
      xs[i] = in[((size_t)b * W + c) * NM + k0 + kc];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nk * W; idx += blockDim.x) {
      const int kc = idx / W, o = idx - kc * W;
      float2 acc = make_float2(0.f, 0.f);
      const float2* r = Rs + ((size_t)kc * W + o) * W;
      const float2* x = xs + kc * W;
      for (int i = 0; i < W; ++i) {
        const float2 p = cmulf(r[i], x[i]);
        acc.x += p.x;
        acc.y += p.y;
      }
      out[((size_t)b * W + o) * NM + k0 + kc] = acc;
    }
  }
}

// backward of the mixing: gin[b][i][k] = sum_o conj(R[k][o][i]) g[b][o][k];
// gR[k][o][i] += sum_b g[b][o][k] conj(x[b][i][k])
__global__ void __launch_bounds__(kT) k_mix_back(FnoDims d, int B, const __nv_bfloat162* __restrict__ R,
                                                  const float2* __restrict__ x, const float2* __restrict__ g,
                                                  float2* __restrict__ gin, float2* __restrict__ gR) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int W = d.W, NM = d.NM;
  const int k0 = blockIdx.x * KC;
  const int nk = min(KC, NM - k0);
  float2* Rs = reinterpret_cast<float2*>(sm);          // [kc][o][i]
  float2* xs = Rs + KC * W * W;                         // [b][kc][i]
  float2* gs = xs + (size_t)B * KC * W;                 // [b][kc][o]
  for (int i = threadIdx.x; i < nk * W * W; i += blockDim.x) {
    const __nv_bfloat162 r = R[(size_t)k0 * W * W + i];
    Rs[i] = make_float2(__bfloat162float(r.x), __bfloat162float(r.y));
  }
  for (int i = threadIdx.x; i < B * nk * W; i += blockDim.x) {
    const int b = i / (nk * W), rem = i - b * nk * W, kc = rem / W, c = rem - kc * W;
    xs[(b * KC + kc) * W + c] = x[((size_t)b * W + c) * NM + k0 + kc];
    gs[(b * KC + kc) * W + c] = g[((size_t)b * W + c) * NM + k0 + kc];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < B * nk * W; idx += blockDim.x) {
    const int b = idx / (nk * W), rem = idx - b * nk * W, kc = rem / W, i = rem - kc * W;
    float2 acc = make_float2(0.f, 0.f);
    for (int o = 0; o < W; ++o) {
      const float2 r = Rs[((size_t)kc * W + o) * W + i];
      const float2 gg = gs[(b * KC + kc) * W + o];
      acc.x += r.x * gg.x + r.y * gg.y;   // conj(r) * g
      acc.y += r.x * gg.y - r.y * gg.x;
    }
    gin[((size_t)b * W + i) * NM + k0 + kc] = acc;
  }
  for (int idx = threadIdx.x; idx < nk * W * W; idx += blockDim.x) {
    const int kc = idx / (W * W), rem = idx - kc * W * W, o = rem / W, i = rem - o * W;
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < B; ++b) {
      const float2 gg = gs[(b * KC + kc) * W + o];
      const float2 xx = xs[(b * KC + kc) * W + i];
      acc.x += gg.x * xx.x + gg.y * xx.y;  // g * conj(x)
      acc.y += gg.y * xx.x - gg.x * xx.y;
    }
    float2* t = gR + (size_t)(k0 + kc) * W * W + o * W + i;
    t->x += acc.x;
    t->y += acc.y;
  }
}

// ---------------------------------------------------------------- pointwise layers
__device__ __forceinline__ float gelu_f(float u) { return 0.5f * u * (1.f + erff(u * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float u) {
  return 0.5f * (1.f + erff(u * 0.70710678118654752f)) + u * 0.39894228040143268f * expf(-0.5f * u * u);
}

// y[b][o][p] = sum_c A[o][c] x[b][c][p] + bias[o] (+ add[b][o][p]); optional gelu; optional store of u
template <bool BF16>
__global__ void __launch_bounds__(kT) k_pointwise(int B, int N3, int Cin, int Cout, const void* __restrict__ A,
                                                   const float* __restrict__ bias, const float* __restrict__ x,
                                                   const float* __restrict__ add, float* __restrict__ u_out,
                                                   float* __restrict__ y, int act) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* As = reinterpret_cast<float*>(sm);   // [o][c]
  for (int i = threadIdx.x; i < Cout * Cin; i += blockDim.x)
    As[i] = BF16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(A)[i]) : reinterpret_cast<const float*>(A)[i];
  __syncthreads();
  const long long total = (long long)B * N3;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / N3);
    const int p = (int)(t - (long long)b * N3);
    float xin[64];
    for (int c = 0; c < Cin; ++c) xin[c] = x[((size_t)b * Cin + c) * N3 + p];
    for (int o = 0; o < Cout; ++o) {
      float acc = bias[o];
      const float* a = As + o * Cin;
      for (int c = 0; c < Cin; ++c) acc += a[c] * xin[c];
      const size_t oi = ((size_t)b * Cout + o) * N3 + p;
      if (add) acc += add[oi];
      if (u_out) u_out[oi] = acc;
      y[oi] = act ? gelu_f(acc) : acc;
    }
  }
}

// gx[b][c][p] = sum_o A[o][c] gy[b][o][p] (gy optionally times gelu'(u) first, stored in gu)
template <bool BF16>
__global__ void __launch_bounds__(kT) k_pointwise_back(int B, int N3, int Cin, int Cout, const void* __restrict__ A,
                                                        const float* __restrict__ gy, const float* __restrict__ u,
                                                        float* __restrict__ gu, float* __restrict__ gx) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* As = reinterpret_cast<float*>(sm);
  for (int i = threadIdx.x; i < Cout * Cin; i += blockDim.x)
    As[i] = BF16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(A)[i]) : reinterpret_cast<const float*>(A)[i];
  __syncthreads();
  const long long total = (long long)B * N3;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / N3);
    const int p = (int)(t - (long long)b * N3);
    float g[64];
    for (int o = 0; o < Cout; ++o) {
      const size_t oi = ((size_t)b * Cout + o) * N3 + p;
      float v = gy[oi];
      if (u) {
        v *= gelu_d(u[oi]);
        gu[oi] = v;
      }
      g[o] = v;
    }
    if (!gx) continue;
    for (int c = 0; c < Cin; ++c) {
      float acc = 0.f;
      for (int o = 0; o < Cout; ++o) acc += As[o * Cin + c] * g[o];
      gx[((size_t)b * Cin + c) * N3 + p] = acc;
    }
  }
}

// gA[o][c] += sum_{b,p} g[b][o][p] x[b][c][p];  gbias[o] += sum g[b][o][p]   (tile of 256 voxels per block)
__global__ void __launch_bounds__(kT) k_weight_grad(int B, int N3, int Cin, int Cout, const float* __restrict__ g,
                                                     const float* __restrict__ x, float* __restrict__ gA,
                                                     float* __restrict__ gbias) {
  extern __shared__ __align__(16) unsigned char sm[];
  constexpr int TP = 128, TS = TP + 1;        // odd row stride: no bank conflicts
  float* gs = reinterpret_cast<float*>(sm);   // [o][TS]
  float* xs = gs + Cout * TS;                  // [c][TS]
  const long long total = (long long)B * N3;
  const long long t0 = (long long)blockIdx.x * TP;
  for (int i = threadIdx.x; i < Cout * TP; i += blockDim.x) {
    const int o = i / TP, q = i - o * TP;
    const long long t = t0 + q;
    float v = 0.f;
    if (t < total) {
      const int b = (int)(t / N3), p = (int)(t - (long long)b * N3);
      v = g[((size_t)b * Cout + o) * N3 + p];
    }
    gs[o * TS + q] = v;
  }
  for (int i = threadIdx.x; i < Cin * TP; i += blockDim.x) {
    const int c = i / TP, q = i - c * TP;
    const long long t = t0 + q;
    float v = 0.f;
    if (t < total) {
      const int b = (int)(t / N3), p = (int)(t - (long long)b * N3);
      v = x[((size_t)b * Cin + c) * N3 + p];
    }
    xs[c * TS + q] = v;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < Cout * Cin; idx += blockDim.x) {
    const int o = idx / Cin, c = idx - o * Cin;
    float acc = 0.f;
    for (int q = 0; q < TP; ++q) acc += gs[o * TS + q] * xs[c * TS + q];
    atomicAdd(&gA[idx], acc);
  }
  for (int o = threadIdx.x; o < Cout; o += blockDim.x) {
    float acc = 0.f;
    for (int q = 0; q < TP; ++q) acc += gs[o * TS + q];
    atomicAdd(&gbias[o], acc);
  }
}

// mean-squared-error gradient: g = 2 (y - t) / count; per-block partial sums of (y - t)^2
__global__ void __launch_bounds__(kT) k_mse(long long n, const float* __restrict__ y, const float* __restrict__ t,
                                            float* __restrict__ g, double* __restrict__ partial, float inv_count) {
  __shared__ double red[kT / 32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float e = y[i] - t[i];
    acc += (double)e * e;
    g[i] = 2.f * e * inv_count;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kT / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_adam(long long n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

struct FeatParams {
  float logE[16];
  float e0[6];
};

__global__ void k_features(int N3, FeatParams P, const uint8_t* __restrict__ phase, float* __restrict__ x,
                           int with_strain) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N3; i += gridDim.x * blockDim.x) {
    x[i] = P.logE[phase[i] & 15];
    if (with_strain)
      for (int c = 0; c < 6; ++c) x[(size_t)(c + 1) * N3 + i] = P.e0[c];
  }
}

__global__ void k_to_bf16(long long n, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

}  // namespace

// ---------------------------------------------------------------- host object
struct fh_fno {
  FnoDims d{};
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  // parameters (FP32 master): P [W][cin], p [W], Wl [L][W][W], wl [L][W], R [L][NM][W][W] complex, Q [cout][W], q [cout]
  long long off_P, off_p, off_W, off_w, off_R, off_Q, off_q, nparam;
  float* prm = nullptr;
  float* grd = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  __nv_bfloat16* Wbf = nullptr;   // [L][W][W]
  __nv_bfloat16* Rbf = nullptr;   // [L][NM][W][W][2]
  float2* tw = nullptr;           // e^{-2 pi i t/N}
  // activations
  float* v = nullptr;       // [L+1][B][W][N3]
  float* u = nullptr;       // [L][B][W][N3]
  float2* vh = nullptr;     // [L][B][W][NM]
  float* spec = nullptr;    // [B][W][N3]
  float2* Yy = nullptr;     // [B][W][N][2m][m]
  float2* cf = nullptr;     // [B][W][NM]
  float2* gin = nullptr;    // [B][W][NM]
  float* y = nullptr;       // [B][cout][N3]
  float* gy = nullptr;      // [B][cout][N3]
  float* ga = nullptr;      // [B][W][N3]  gradient wrt an activation
  float* gb = nullptr;      // [B][W][N3]
  double* part = nullptr;
  int nparts = 0;
  // hidden 1 x 1 layers on the tensor cores (fno_tc.cuh) where the width is
  // 16, 32 or 64 and N^3 is a multiple of 128; tc_err is set by a kernel whose
  // bounded wait gave up
  bool tensor_cores = true;
  int* tc_err = nullptr;
};

namespace {

#define FCK(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      fh::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));     \
      return FH_ERR_CUDA;                                                    \
    }                                                                        \
  } while (0)

int grid_for(long long n) { return (int)std::min<long long>((n + kT - 1) / kT, 152 * 16); }

// K v for the activations a ([B][W][N3]) with the layer's R; result into out (or added)
fh_status spectral_forward(fh_fno* f, int B, int l, const float* a, float2* coef_store, float* out) {
  const FnoDims& d = f->d;
  const int m2 = 2 * d.m;
  const size_t sm_zy = (size_t)d.N * d.N * 4 + (size_t)d.N * 8 + (size_t)d.N * d.m * 8;
  k_dft_zy<<<B * d.W * d.N, kT, sm_zy, f->stream>>>(d, a, f->Yy, f->tw, d.W);
  const size_t sm_x = (size_t)d.N * 8 + (size_t)d.N * d.m * 8;
  k_dft_x<<<B * d.W * m2, kT, sm_x, f->stream>>>(d, f->Yy, coef_store, f->tw, d.W, 1.f, 0);
  const size_t sm_mix = (size_t)KC * d.W * d.W * 8 + (size_t)KC * d.W * 8;
  k_mix<<<(d.NM + KC - 1) / KC, kT, sm_mix, f->stream>>>(d, B, reinterpret_cast<const __nv_bfloat162*>(f->Rbf) + (size_t)l * d.NM * d.W * d.W,
                                                        coef_store, f->cf);
  const size_t sm_ix = (size_t)d.N * 8 + (size_t)m2 * d.m * 8;
  k_idft_x<<<B * d.W * m2, kT, sm_ix, f->stream>>>(d, f->cf, f->Yy, f->tw);
  const size_t sm_iyz = (size_t)d.N * 8 + (size_t)m2 * d.m * 8 + (size_t)d.N * d.m * 8;
  k_idft_yz<<<B * d.W * d.N, kT, sm_iyz, f->stream>>>(d, f->Yy, out, f->tw, 1.f / (float)d.N3, 1, 0);
  FCK(cudaGetLastError());
  return FH_OK;
}

// a tensor-core layer whose bounded wait gave up leaves an error word
fh_status tc_status(fh_fno* f) {
  int h = 0;
  FCK(cudaMemcpy(&h, f->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    FCK(cudaMemset(f->tc_err, 0, sizeof(int)));
    fh::set_error("a tensor-core layer's wait for its MMAs gave up");
    return FH_ERR_TIMEOUT;
  }
  return FH_OK;
}

bool use_tc(const fh_fno* f) {
  const FnoDims& d = f->d;
  return f->tensor_cores && (d.W == 16 || d.W == 32 || d.W == 64) && d.N3 % fhtc::kTcTile == 0;
}

fh_status forward_all(fh_fno* f, int B, const float* x) {
  const FnoDims& d = f->d;
  const size_t act = (size_t)B * d.W * d.N3;
  const long long tot = (long long)B * d.N3;
  k_pointwise<false><<<grid_for(tot), kT, (size_t)d.W * d.cin * 4, f->stream>>>(
      B, d.N3, d.cin, d.W, f->prm + f->off_P, f->prm + f->off_p, x, nullptr, nullptr, f->v, 0);
  for (int l = 0; l < d.L; ++l) {
    const float* vl = f->v + (size_t)l * act;
    fh_status rc = spectral_forward(f, B, l, vl, f->vh + (size_t)l * B * d.W * d.NM, f->spec);
    if (rc != FH_OK) return rc;
    if (use_tc(f)) {
      const int ntiles = B * (d.N3 / fhtc::kTcTile);
      const int grid = std::min(ntiles, 152 * 4);
      const __nv_bfloat16* Wl = f->Wbf + (size_t)l * d.W * d.W;
      const float* wl = f->prm + f->off_w + (size_t)l * d.W;
      float* ul = f->u + (size_t)l * act;
      float* vn = f->v + (size_t)(l + 1) * act;
      if (d.W == 16)
        fhtc::k_pointwise_tc<16><<<grid, fhtc::kTcThreads, 0, f->stream>>>(B, d.N3, Wl, wl, vl, f->spec, ul, vn, 1, f->tc_err);
      else if (d.W == 32)
        fhtc::k_pointwise_tc<32><<<grid, fhtc::kTcThreads, 0, f->stream>>>(B, d.N3, Wl, wl, vl, f->spec, ul, vn, 1, f->tc_err);
      else
        fhtc::k_pointwise_tc<64><<<grid, fhtc::kTcThreads, 0, f->stream>>>(B, d.N3, Wl, wl, vl, f->spec, ul, vn, 1, f->tc_err);
    } else {
      k_pointwise<true><<<grid_for(tot), kT, (size_t)d.W * d.W * 4, f->stream>>>(
          B, d.N3, d.W, d.W, f->Wbf + (size_t)l * d.W * d.W, f->prm + f->off_w + (size_t)l * d.W, vl, f->spec,
          f->u + (size_t)l * act, f->v + (size_t)(l + 1) * act, 1);
    }
  }
  k_pointwise<false><<<grid_for(tot), kT, (size_t)d.cout * d.W * 4, f->stream>>>(
      B, d.N3, d.W, d.cout, f->prm + f->off_Q, f->prm + f->off_q, f->v + (size_t)d.L * act, nullptr, nullptr, f->y, 0);
  FCK(cudaGetLastError());
  return FH_OK;
}

fh_status refresh_bf16(fh_fno* f) {
  const FnoDims& d = f->d;
  const long long nW = (long long)d.L * d.W * d.W, nR = (long long)d.L * d.NM * d.W * d.W * 2;
  k_to_bf16<<<grid_for(nW), kT, 0, f->stream>>>(nW, f->prm + f->off_W, f->Wbf);
  k_to_bf16<<<grid_for(nR), kT, 0, f->stream>>>(nR, f->prm + f->off_R, f->Rbf);
  FCK(cudaGetLastError());
  return FH_OK;
}

}  // namespace

extern "C" {

fh_status fh_fno_create(int n, int cin, int cout, int width, int modes, int layers, int max_batch, void* stream,
                        fh_fno** out) {
  if (!out) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (n < 4 || n > 128 || cin < 1 || cin > 64 || cout < 1 || cout > 64 || width < 1 || width > 64 || modes < 1 ||
      2 * modes > n || layers < 1 || layers > 8 || max_batch < 1 || max_batch > 64) {
    fh::set_error("FNO sizes out of range (n<=128, channels<=64, 2*modes<=n, layers<=8, batch<=64)");
    return FH_ERR_ARG;
  }
  fh_fno* f = new fh_fno();
  FnoDims& d = f->d;
  d.N = n; d.cin = cin; d.cout = cout; d.W = width; d.m = modes; d.L = layers;
  d.N3 = n * n * n;
  d.NM = 4 * modes * modes * modes;
  f->max_batch = max_batch;
  f->stream = reinterpret_cast<cudaStream_t>(stream);
  long long o = 0;
  f->off_P = o; o += (long long)width * cin;
  f->off_p = o; o += width;
  f->off_W = o; o += (long long)layers * width * width;
  f->off_w = o; o += (long long)layers * width;
  f->off_R = o; o += (long long)layers * d.NM * width * width * 2;
  f->off_Q = o; o += (long long)cout * width;
  f->off_q = o; o += cout;
  f->nparam = o;
  auto fail = [&](cudaError_t e) {
    fh::set_error(std::string("FNO allocation: ") + cudaGetErrorString(e));
    fh_fno_destroy(f);
    return FH_ERR_CUDA;
  };
  cudaError_t e;
  const size_t act = (size_t)max_batch * width * d.N3;
  if ((e = cudaMalloc(&f->prm, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->grd, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->m1, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->m2, o * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->Wbf, (size_t)layers * width * width * 2)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->Rbf, (size_t)layers * d.NM * width * width * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->tw, (size_t)n * 8)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->v, (layers + 1) * act * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->u, layers * act * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->vh, (size_t)layers * max_batch * width * d.NM * 8)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->spec, act * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->Yy, (size_t)max_batch * width * n * 2 * modes * modes * 8)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->cf, (size_t)max_batch * width * d.NM * 8)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->gin, (size_t)max_batch * width * d.NM * 8)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->y, (size_t)max_batch * cout * d.N3 * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->gy, (size_t)max_batch * cout * d.N3 * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->ga, act * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->gb, act * 4)) != cudaSuccess) return fail(e);
  f->nparts = 152 * 16;
  if ((e = cudaMalloc(&f->part, f->nparts * sizeof(double))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&f->tc_err, sizeof(int))) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(f->tc_err, 0, sizeof(int))) != cudaSuccess) return fail(e);
  cudaMemset(f->prm, 0, o * 4);
  cudaMemset(f->grd, 0, o * 4);
  cudaMemset(f->m1, 0, o * 4);
  cudaMemset(f->m2, 0, o * 4);
  // shared memory of the mixing kernels grows with width^2 (and the batch)
  const size_t sm_mix = (size_t)KC * width * width * 8 + (size_t)KC * width * 8;
  const size_t sm_mb = (size_t)KC * width * width * 8 + (size_t)2 * max_batch * KC * width * 8;
  const size_t sm_zy = (size_t)n * n * 4 + (size_t)n * 8 + (size_t)n * modes * 8;
  if (sm_mb > 227 * 1024 || sm_zy > 227 * 1024) {
    fh::set_error("FNO width/batch/grid too large for the shared-memory tiles");
    fh_fno_destroy(f);
    return FH_ERR_UNSUPPORTED;
  }
  if ((e = cudaFuncSetAttribute(k_mix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_mix)) != cudaSuccess) return fail(e);
  if ((e = cudaFuncSetAttribute(k_mix_back, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_mb)) != cudaSuccess) return fail(e);
  if ((e = cudaFuncSetAttribute(k_dft_zy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_zy)) != cudaSuccess) return fail(e);
  std::vector<float2> tw(n);
  for (int t = 0; t < n; ++t) {
    const long double a = 2.0L * 3.141592653589793238462643383279502884L * t / n;
    tw[t] = make_float2((float)cosl(a), (float)(-sinl(a)));
  }
  if ((e = cudaMemcpy(f->tw, tw.data(), n * 8, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  *out = f;
  return FH_OK;
}

void fh_fno_destroy(fh_fno* f) {
  if (!f) return;
  void* ptrs[] = {f->prm, f->grd, f->m1, f->m2, f->Wbf, f->Rbf, f->tw, f->v, f->u, f->vh, f->spec,
                  f->Yy, f->cf, f->gin, f->y, f->gy, f->ga, f->gb, f->part, f->tc_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete f;
}

fh_status fh_fno_param_count(const fh_fno* f, long long* count) {
  if (!f || !count) { fh::set_error("null argument"); return FH_ERR_ARG; }
  *count = f->nparam;
  return FH_OK;
}

}  // extern "C"

namespace {
// The public parameter vector stores R as all real parts then all imaginary
// parts; the device keeps each complex weight interleaved.
void flat_to_device(const fh_fno* f, const float* flat, std::vector<float>& dev) {
  dev.assign(flat, flat + f->nparam);
  const long long nR = (f->off_Q - f->off_R) / 2;
  for (long long i = 0; i < nR; ++i) {
    dev[f->off_R + 2 * i] = flat[f->off_R + i];
    dev[f->off_R + 2 * i + 1] = flat[f->off_R + nR + i];
  }
}
void device_to_flat(const fh_fno* f, const std::vector<float>& dev, float* flat) {
  std::memcpy(flat, dev.data(), f->nparam * 4);
  const long long nR = (f->off_Q - f->off_R) / 2;
  for (long long i = 0; i < nR; ++i) {
    flat[f->off_R + i] = dev[f->off_R + 2 * i];
    flat[f->off_R + nR + i] = dev[f->off_R + 2 * i + 1];
  }
}
fh_status copy_out(const fh_fno* f, const float* src, float* flat) {
  std::vector<float> dev(f->nparam);
  FCK(cudaMemcpyAsync(dev.data(), src, f->nparam * 4, cudaMemcpyDeviceToHost, f->stream));
  FCK(cudaStreamSynchronize(f->stream));
  device_to_flat(f, dev, flat);
  return FH_OK;
}
}  // namespace

extern "C" {

fh_status fh_fno_set_params(fh_fno* f, const float* flat) {
  if (!f || !flat) { fh::set_error("null argument"); return FH_ERR_ARG; }
  std::vector<float> dev;
  flat_to_device(f, flat, dev);
  FCK(cudaMemcpyAsync(f->prm, dev.data(), f->nparam * 4, cudaMemcpyHostToDevice, f->stream));
  fh_status rc = refresh_bf16(f);
  if (rc != FH_OK) return rc;
  FCK(cudaStreamSynchronize(f->stream));
  return FH_OK;
}

fh_status fh_fno_get_params(const fh_fno* f, float* flat) {
  if (!f || !flat) { fh::set_error("null argument"); return FH_ERR_ARG; }
  return copy_out(f, f->prm, flat);
}

fh_status fh_fno_get_grads(const fh_fno* f, float* flat) {
  if (!f || !flat) { fh::set_error("null argument"); return FH_ERR_ARG; }
  return copy_out(f, f->grd, flat);
}

// input channels of one sample: [log10 E(x) / 2, eps0 (n_v constant channels)]
fh_status fh_fno_make_input(const fh_fno* f, const uint8_t* phase, int nphase, const double* phase_logE,
                            const double* eps0, float* x) {
  if (!f || !phase || !phase_logE || !eps0 || !x) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (nphase < 1 || nphase > 16) { fh::set_error("nphase must be 1..16"); return FH_ERR_ARG; }
  if (f->d.cin != 7 && f->d.cin != 1) {
    fh::set_error("make_input builds 1 channel (log10 E) or 7 (log10 E, 6 strains)");
    return FH_ERR_ARG;
  }
  FeatParams P{};
  for (int q = 0; q < nphase; ++q) P.logE[q] = (float)(0.5 * phase_logE[q]);
  for (int c = 0; c < 6; ++c) P.e0[c] = (float)eps0[c];
  k_features<<<grid_for(f->d.N3), kT, 0, f->stream>>>(f->d.N3, P, phase, x, f->d.cin == 7);
  FCK(cudaGetLastError());
  FCK(cudaStreamSynchronize(f->stream));
  return FH_OK;
}

fh_status fh_fno_zero_grad(fh_fno* f) {
  if (!f) { fh::set_error("null argument"); return FH_ERR_ARG; }
  FCK(cudaMemsetAsync(f->grd, 0, f->nparam * 4, f->stream));
  return FH_OK;
}

fh_status fh_fno_forward(fh_fno* f, int batch, const float* x, float* y) {
  if (!f || !x || !y) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (batch < 1 || batch > f->max_batch) { fh::set_error("batch out of range"); return FH_ERR_ARG; }
  fh_status rc = forward_all(f, batch, x);
  if (rc != FH_OK) return rc;
  FCK(cudaMemcpyAsync(y, f->y, (size_t)batch * f->d.cout * f->d.N3 * 4, cudaMemcpyDefault, f->stream));
  FCK(cudaStreamSynchronize(f->stream));
  return tc_status(f);
}

fh_status fh_fno_set_tensor_cores(fh_fno* f, int enable) {
  if (!f || (enable != 0 && enable != 1)) { fh::set_error("null network or enable not 0/1"); return FH_ERR_ARG; }
  f->tensor_cores = enable != 0;
  return FH_OK;
}

fh_status fh_fno_loss_grad(fh_fno* f, int batch, const float* x, const float* target, double* loss) {
  if (!f || !x || !target) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (batch < 1 || batch > f->max_batch) { fh::set_error("batch out of range"); return FH_ERR_ARG; }
  const FnoDims& d = f->d;
  fh_status rc = forward_all(f, batch, x);
  if (rc != FH_OK) return rc;
  const long long ny = (long long)batch * d.cout * d.N3;
  const int gb = std::min(f->nparts, grid_for(ny));
  k_mse<<<gb, kT, 0, f->stream>>>(ny, f->y, target, f->gy, f->part, 1.f / (float)ny);
  const size_t act = (size_t)batch * d.W * d.N3;
  const long long tot = (long long)batch * d.N3;
  const int m2 = 2 * d.m;
  // projection
  const int tiles = (int)((tot + 127) / 128);
  k_weight_grad<<<tiles, kT, (size_t)(d.cout + d.W) * 129 * 4, f->stream>>>(
      batch, d.N3, d.W, d.cout, f->gy, f->v + (size_t)d.L * act, f->grd + f->off_Q, f->grd + f->off_q);
  k_pointwise_back<false><<<grid_for(tot), kT, (size_t)d.cout * d.W * 4, f->stream>>>(
      batch, d.N3, d.W, d.cout, f->prm + f->off_Q, f->gy, nullptr, nullptr, f->ga);
  for (int l = d.L - 1; l >= 0; --l) {
    const float* vl = f->v + (size_t)l * act;
    // gu = ga * gelu'(u_l) -> gb ; ga <- W^T gu
    k_pointwise_back<true><<<grid_for(tot), kT, (size_t)d.W * d.W * 4, f->stream>>>(
        batch, d.N3, d.W, d.W, f->Wbf + (size_t)l * d.W * d.W, f->ga, f->u + (size_t)l * act, f->gb, f->ga);
    k_weight_grad<<<tiles, kT, (size_t)(2 * d.W) * 129 * 4, f->stream>>>(
        batch, d.N3, d.W, d.W, f->gb, vl, f->grd + f->off_W + (size_t)l * d.W * d.W, f->grd + f->off_w + (size_t)l * d.W);
    // spectral adjoint: G_c = (w/N^3) DFT_trunc(gu); mixing backward; ga += Re sum G_v e^{+ikx}
    const size_t sm_zy = (size_t)d.N * d.N * 4 + (size_t)d.N * 8 + (size_t)d.N * d.m * 8;
    k_dft_zy<<<batch * d.W * d.N, kT, sm_zy, f->stream>>>(d, f->gb, f->Yy, f->tw, d.W);
    const size_t sm_x = (size_t)d.N * 8 + (size_t)d.N * d.m * 8;
    k_dft_x<<<batch * d.W * m2, kT, sm_x, f->stream>>>(d, f->Yy, f->cf, f->tw, d.W, 1.f / (float)d.N3, 1);
    const size_t sm_mb = (size_t)KC * d.W * d.W * 8 + (size_t)2 * batch * KC * d.W * 8;
    float2* gin = f->gin;
    k_mix_back<<<(d.NM + KC - 1) / KC, kT, sm_mb, f->stream>>>(
        d, batch, reinterpret_cast<const __nv_bfloat162*>(f->Rbf) + (size_t)l * d.NM * d.W * d.W,
        f->vh + (size_t)l * batch * d.W * d.NM, f->cf, gin,
        reinterpret_cast<float2*>(f->grd + f->off_R) + (size_t)l * d.NM * d.W * d.W);
    const size_t sm_ix = (size_t)d.N * 8 + (size_t)m2 * d.m * 8;
    k_idft_x<<<batch * d.W * m2, kT, sm_ix, f->stream>>>(d, gin, f->Yy, f->tw);
    const size_t sm_iyz = (size_t)d.N * 8 + (size_t)m2 * d.m * 8 + (size_t)d.N * d.m * 8;
    k_idft_yz<<<batch * d.W * d.N, kT, sm_iyz, f->stream>>>(d, f->Yy, f->ga, f->tw, 1.f, 0, 1);
  }
  // lift
  k_weight_grad<<<tiles, kT, (size_t)(d.W + d.cin) * 129 * 4, f->stream>>>(batch, d.N3, d.cin, d.W, f->ga, x,
                                                                           f->grd + f->off_P, f->grd + f->off_p);
  FCK(cudaGetLastError());
  std::vector<double> parts(gb);
  FCK(cudaMemcpyAsync(parts.data(), f->part, gb * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
  FCK(cudaStreamSynchronize(f->stream));
  if (loss) {
    double s = 0.0;
    for (double p : parts) s += p;
    *loss = s / (double)ny;
  }
  return tc_status(f);
}

fh_status fh_fno_adam_step(fh_fno* f, float lr, float beta1, float beta2, float eps, int step) {
  if (!f || step < 1) { fh::set_error("bad argument"); return FH_ERR_ARG; }
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid_for(f->nparam), kT, 0, f->stream>>>(f->nparam, f->prm, f->grd, f->m1, f->m2, lr, beta1, beta2, eps, c1, c2);
  FCK(cudaGetLastError());
  fh_status rc = refresh_bf16(f);
  if (rc != FH_OK) return rc;
  FCK(cudaStreamSynchronize(f->stream));
  return FH_OK;
}

}  // extern "C"
