// Shared-memory mixed-radix FFT used by the pattern-DFT passes.
//
// The pattern DFT of the paper's Eq. (Fouriermatrix) becomes, through the
// Smith-normal-form index map, an ordinary multi-dimensional DFT on the
// stored grid.  Every pass of the solver transforms a batch of lines that sit
// in shared memory; this file holds that line transform: a Stockham
// (self-sorting) radix decomposition L = r_0 r_1 ... with radices
// 2, 3, 4, 5, 8 written out, 7, 11, 13 done as small direct DFTs, and any
// larger prime factor by a direct-DFT stage with one thread per output.
//
// Forward (DIR = -1) computes X_k = sum_n x_n exp(-2 pi i k n / L); inverse
// (DIR = +1) the same with +i and no 1/L factor.  Twiddles come from a table
// tw[t] = exp(-2 pi i t / L), t = 0..L-1, computed once on the host in FP64
// (and rounded to FP32 for the FP32 path); no trigonometric function is
// evaluated on the device.
#pragma once

#include <cuda_runtime.h>

namespace fh {

template <typename T> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };

template <typename T> using cplx = typename cplx_t<T>::type;

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// padd / psub: the same sums, in FP32 as one packed two-wide instruction
// (sm_100 and later) instead of two, each part rounded as the scalar operation
// would be (a - b as b * (-1) + a: one rounding of an exact product).  Used
// where both operands are plain values; where an operand is a product (the
// sqrt(1/2) rotations of the 8-point DFT) the scalar form lets the compiler
// fuse the multiplication into the addition instead.
template <typename C> __device__ __forceinline__ C padd(C a, C b) { return cadd(a, b); }
template <typename C> __device__ __forceinline__ C psub(C a, C b) { return csub(a, b); }
// a + s b and s a per part (scalar s)
template <typename C> __device__ __forceinline__ C pfma(decltype(C::x) s, C b, C a) {
  C r;
  r.x = fma(s, b.x, a.x);
  r.y = fma(s, b.y, a.y);
  return r;
}
template <typename C> __device__ __forceinline__ C pscale(decltype(C::x) s, C a) {
  C r;
  r.x = s * a.x;
  r.y = s * a.y;
  return r;
}
template <> __device__ __forceinline__ float2 pfma<float2>(float s, float2 b, float2 a) {
  return __ffma2_rn(make_float2(s, s), b, a);
}
template <> __device__ __forceinline__ float2 pscale<float2>(float s, float2 a) { return __fmul2_rn(make_float2(s, s), a); }
template <> __device__ __forceinline__ float2 padd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 psub<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// the packed or the plain form, chosen per caller: the packed form pays in the
// register-resident warp FFTs of the row pass and measured slower in the
// shared-memory column passes
template <bool PK, typename C> __device__ __forceinline__ C kadd(C a, C b) {
  if constexpr (PK) return padd(a, b);
  else return cadd(a, b);
}
template <bool PK, typename C> __device__ __forceinline__ C ksub(C a, C b) {
  if constexpr (PK) return psub(a, b);
  else return csub(a, b);
}
// multiply by DIR * i   (DIR = -1: -i, DIR = +1: +i)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
  C r;
  if (DIR > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }

struct DevPlan {
  int L;
  int np;
  int r[24];
};

constexpr int MAX_RADIX = 13;

// Small DFTs in registers, X_k = sum_t v_t w^{kt}, w = exp(DIR 2 pi i / r).
template <int DIR, typename T, bool PK = false>
__device__ __forceinline__ void dft2(cplx<T>* v) {
  cplx<T> a = v[0], b = v[1];
  v[0] = kadd<PK>(a, b);
  v[1] = ksub<PK>(a, b);
}

template <int DIR, typename T, bool PK = false>
__device__ __forceinline__ void dft4(cplx<T>* v) {
  cplx<T> t0 = kadd<PK>(v[0], v[2]), t1 = ksub<PK>(v[0], v[2]);
  cplx<T> t2 = kadd<PK>(v[1], v[3]), t3 = mul_i<DIR>(ksub<PK>(v[1], v[3]));
  v[0] = kadd<PK>(t0, t2);
  v[2] = ksub<PK>(t0, t2);
  v[1] = kadd<PK>(t1, t3);
  v[3] = ksub<PK>(t1, t3);
}

template <int DIR, typename T, bool PK = false>
__device__ __forceinline__ void dft8(cplx<T>* v) {
  const T h = T(0.70710678118654752440084436210485);
  cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<DIR, T, PK>(e);
  dft4<DIR, T, PK>(o);
  // w8^k with w8 = (1 + DIR i)/sqrt2
  cplx<T> o1, o2, o3;
  o1.x = h * (o[1].x - DIR * o[1].y);
  o1.y = h * (o[1].y + DIR * o[1].x);
  o2 = mul_i<DIR>(o[2]);
  o3.x = h * (-o[3].x - DIR * o[3].y);
  o3.y = h * (-o[3].y + DIR * o[3].x);
  v[0] = kadd<PK>(e[0], o[0]); v[4] = ksub<PK>(e[0], o[0]);
  v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
  v[2] = kadd<PK>(e[2], o2); v[6] = ksub<PK>(e[2], o2);
  v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}

template <int DIR, typename T>
__device__ __forceinline__ void dft3(cplx<T>* v) {
  const T c = T(-0.5);
  const T s = T(0.86602540378443864676372317075294);  // sqrt(3)/2
  cplx<T> sum = cadd(v[1], v[2]);
  cplx<T> dif = csub(v[1], v[2]);
  cplx<T> a = v[0];
  cplx<T> m;
  m.x = a.x + c * sum.x;
  m.y = a.y + c * sum.y;
  cplx<T> r = mul_i<DIR>(cscale(dif, s));
  v[0] = cadd(a, sum);
  v[1] = cadd(m, r);
  v[2] = csub(m, r);
}

template <int DIR, typename T>
__device__ __forceinline__ void dft5(cplx<T>* v) {
  const T c1 = T(0.30901699437494742410229341718282);   // cos(2 pi/5)
  const T c2 = T(-0.80901699437494742410229341718282);  // cos(4 pi/5)
  const T s1 = T(0.95105651629515357211643933337938);   // sin(2 pi/5)
  const T s2 = T(0.58778525229247312916870595463907);   // sin(4 pi/5)
  cplx<T> a = v[0];
  cplx<T> p1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
  cplx<T> p2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
  cplx<T> m1, m2, q1, q2;
  m1.x = a.x + c1 * p1.x + c2 * p2.x; m1.y = a.y + c1 * p1.y + c2 * p2.y;
  m2.x = a.x + c2 * p1.x + c1 * p2.x; m2.y = a.y + c2 * p1.y + c1 * p2.y;
  q1.x = s1 * d1.x + s2 * d2.x; q1.y = s1 * d1.y + s2 * d2.y;
  q2.x = s2 * d1.x - s1 * d2.x; q2.y = s2 * d1.y - s1 * d2.y;
  q1 = mul_i<DIR>(q1);
  q2 = mul_i<DIR>(q2);
  v[0] = cadd(a, cadd(p1, p2));
  v[1] = cadd(m1, q1);
  v[4] = csub(m1, q1);
  v[2] = cadd(m2, q2);
  v[3] = csub(m2, q2);
}

// direct DFT of a small prime radix R; w^{kt} = tw[((k t) mod R) * (L / R)]
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_direct(cplx<T>* v, const cplx<T>* __restrict__ tw, int L) {
  cplx<T> out[R];
  const int step = L / R;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    cplx<T> acc = v[0];
#pragma unroll
    for (int t = 1; t < R; ++t) {
      cplx<T> w = tw[((k * t) % R) * step];
      if (DIR > 0) w.y = -w.y;
      acc = cadd(acc, cmul(v[t], w));
    }
    out[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_small(cplx<T>* v, const cplx<T>* __restrict__ tw, int L) {
  if (R == 2) dft2<DIR, T>(v);
  else if (R == 3) dft3<DIR, T>(v);
  else if (R == 4) dft4<DIR, T>(v);
  else if (R == 5) dft5<DIR, T>(v);
  else if (R == 8) dft8<DIR, T>(v);
  else dft_direct<R, DIR, T>(v, tw, L);
}

// Integer division by a runtime divisor through a float reciprocal: exact for
// 0 <= n < 2^22 (the product is off by at most one and corrected).
struct FDiv {
  int d;
  float inv;
};
__host__ __device__ inline FDiv make_fdiv(int d) { FDiv f; f.d = d; f.inv = 1.0f / (float)d; return f; }
__device__ __forceinline__ int fdiv(int n, FDiv f) {
  int q = (int)((float)n * f.inv);
  const int r = n - q * f.d;
  if (r < 0) --q;
  else if (r >= f.d) ++q;
  return q;
}

// One Stockham stage of radix R: sub-transforms of size Ns are combined into
// size Ns*R.  Butterfly j reads in[j + t*L/R] (t < R), applies the twiddles
// w^{t k}, k = j mod Ns, w = exp(DIR 2 pi i / (Ns R)), does a length-R DFT and
// writes out[(j / Ns) * Ns * R + k + t*Ns].
// Position of element i inside a padded line: one spare slot after every
// 2^PADSH elements (PADSH = 0: no padding).  With 2^PADSH elements per 128-byte
// shared-memory wavefront, the strided writes of the early Stockham stages
// (stride R) then spread over all banks.
template <int PADSH> __device__ __forceinline__ int padi(int i) { return PADSH ? i + (i >> PADSH) : i; }
template <int PADSH> __host__ __device__ inline int padded_len(int L) { return PADSH ? L + (L >> PADSH) + 1 : L; }

template <int R, int DIR, typename T, int PADSH = 0>
__device__ __forceinline__ void stockham_stage(const cplx<T>* in, cplx<T>* out, int nlines, int ls, int L, int Ns,
                                               const cplx<T>* __restrict__ tw, int tid, int nthr) {
  const int nb = L / R;
  const int stride = L / (Ns * R);
  const int total = nlines * nb;
  const FDiv fnb = make_fdiv(nb), fns = make_fdiv(Ns);
  for (int idx = tid; idx < total; idx += nthr) {
    const int line = fdiv(idx, fnb);
    const int j = idx - line * nb;
    const cplx<T>* li = in + line * ls;
    cplx<T>* lo = out + line * ls;
    const int jq = fdiv(j, fns);
    const int k = j - jq * Ns;
    cplx<T> v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = li[padi<PADSH>(j + t * nb)];
    if (k != 0) {
#pragma unroll
      for (int t = 1; t < R; ++t) {
        cplx<T> w = tw[t * k * stride];
        if (DIR > 0) w.y = -w.y;
        v[t] = cmul(v[t], w);
      }
    }
    dft_small<R, DIR, T>(v, tw, L);
    const int base = jq * Ns * R + k;
#pragma unroll
    for (int t = 0; t < R; ++t) lo[padi<PADSH>(base + t * Ns)] = v[t];
  }
}

// Stage of any other prime radix R (the factors above 13 of an axis length):
// one thread per output.  Output o = jq Ns R + t_out Ns + k of group
// j = jq Ns + k is sum_t v_t w_L^{t k stride} w_R^{t_out t}, v_t = in[j + t nb];
// both twiddles come from the table as one exponent t k stride +
// ((t_out t) mod R) L / R, reduced mod L.  The work per point grows with R
// (2 R flops of complex multiply-add) where the written-out radices need
// O(log R); it makes every axis length up to 4096 usable.
template <int DIR, typename T, int PADSH = 0>
__device__ __forceinline__ void stockham_stage_prime(const cplx<T>* in, cplx<T>* out, int nlines, int ls, int L,
                                                     int Ns, int R, const cplx<T>* __restrict__ tw, int tid,
                                                     int nthr) {
  const int nb = L / R;
  const int stride = L / (Ns * R);
  const int step = L / R;
  const int total = nlines * L;
  for (int idx = tid; idx < total; idx += nthr) {
    const int line = idx / L;
    const int o = idx - line * L;
    const int k = o % Ns;
    const int rest = o / Ns;
    const int t_out = rest % R;
    const int jq = rest / R;
    const int j = jq * Ns + k;
    const cplx<T>* li = in + line * ls;
    cplx<T> acc = li[padi<PADSH>(j)];
    for (int t = 1; t < R; ++t) {
      int e = t * k * stride + ((t_out * t) % R) * step;
      if (e >= L) e -= L;
      cplx<T> w = tw[e];
      if (DIR > 0) w.y = -w.y;
      acc = cadd(acc, cmul(li[padi<PADSH>(j + t * nb)], w));
    }
    out[line * ls + padi<PADSH>(o)] = acc;
  }
}

// Barrier of a team of threads: the whole block (nthr == blockDim.x), else the
// first nthr threads (a multiple of 32) on named barrier 1.
__device__ __forceinline__ void team_sync(int nthr) {
  if (nthr == (int)blockDim.x) __syncthreads();
  else asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
}

// Transform `nlines` lines of length plan.L held in shared memory.  Line q
// occupies buf[q*ls .. q*ls + L); tmp has the same shape (ping-pong buffer).
// Every thread of the team (threads tid = 0 .. nthr-1; by default the whole
// block) must call this.  Returns the buffer (buf or tmp) that holds the
// result; a team barrier has been executed on return.
// POW2: the plan uses radices 2, 4 and 8 only (the caller checks); the other
// stage kernels are then not compiled in, which keeps register use low.
template <int DIR, typename T, int PADSH = 0, bool POW2 = false>
__device__ cplx<T>* fft_lines_pp(cplx<T>* buf, cplx<T>* tmp, int nlines, int ls, const DevPlan& plan,
                                 const cplx<T>* __restrict__ tw, int tid = -1, int nthr = 0) {
  if (nthr == 0) { tid = threadIdx.x; nthr = blockDim.x; }
  const int L = plan.L;
  cplx<T>* in = buf;
  cplx<T>* out = tmp;
  int Ns = 1;
  for (int s = 0; s < plan.np; ++s) {
    const int r = plan.r[s];
    if constexpr (POW2) {
      switch (r) {
        case 2: stockham_stage<2, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 4: stockham_stage<4, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        default: stockham_stage<8, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
      }
    } else {
      switch (r) {
        case 2: stockham_stage<2, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 3: stockham_stage<3, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 4: stockham_stage<4, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 5: stockham_stage<5, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 7: stockham_stage<7, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 8: stockham_stage<8, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 11: stockham_stage<11, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        case 13: stockham_stage<13, DIR, T, PADSH>(in, out, nlines, ls, L, Ns, tw, tid, nthr); break;
        default: stockham_stage_prime<DIR, T, PADSH>(in, out, nlines, ls, L, Ns, r, tw, tid, nthr); break;
      }
    }
    team_sync(nthr);
    cplx<T>* sw = in; in = out; out = sw;
    Ns *= r;
  }
  return in;
}

}  // namespace fh
