// Warp-per-row variant of the row pass for 3-D grids (n_v = 6) whose
// contiguous axis has length L = 32 P, P in {1, 2, 4, 8}.
//
// One warp owns one grid row of one load at a time.  The six strain
// components of the row form three complex lines (components 2p and 2p+1 as
// real and imaginary parts), held in registers with lane l owning the points
// l + 32 j, j < P.  The line DFT is done without block barriers:
//   forward  - length-P DFT over j in registers, twiddles w_L^{l q}, then a
//              32-point decimation-in-frequency DFT across the lanes with
//              shuffles; lane l ends with frequency q + P * bitrev5(l);
//   inverse  - the mirror image (decimation in time across lanes from that
//              bit-reversed layout, twiddles, length-P DFT), ending with the
//              points back in natural order.
// Since every lane holds all six components of its points, the pointwise
// stage (E update, Cauchy-residual sums, tau = (C - C0):(E + eps0)) needs no
// data exchange.  Half-spectrum rows move between global and a per-warp
// shared-memory scratch line with coalesced accesses.
#pragma once

#include "kernels.cuh"

namespace fh {

__device__ __forceinline__ int bitrev5(int v) { return (int)(__brev((unsigned)v) >> 27); }

template <typename T>
__device__ __forceinline__ cplx<T> shfl_xor_c(cplx<T> v, int m) {
  cplx<T> r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return r;
}

// 16-point DFT in registers, X_k = sum_n v_n w^{nk}, w = exp(DIR 2 pi i / 16):
// n = 4 n1 + n2, k = k1 + 4 k2; length-4 DFTs over n1, twiddles w^{n2 k1},
// length-4 DFTs over n2.
template <int DIR, typename T>
__device__ __forceinline__ void dft16(cplx<T>* v) {
  const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), h = T(0.70710678118654752440);
  cplx<T> y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    cplx<T> a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
    dft4<DIR, T>(a);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = a[k1];
  }
  auto tw16 = [&](int m) {   // exp(DIR 2 pi i m / 16) for m in {1, 2, 3, 4, 6, 9}
    cplx<T> w;
    switch (m) {
      case 1: w.x = c1; w.y = s1; break;
      case 2: w.x = h; w.y = h; break;
      case 3: w.x = s1; w.y = c1; break;
      case 4: w.x = T(0); w.y = T(1); break;
      case 6: w.x = -h; w.y = h; break;
      default: w.x = -c1; w.y = -s1; break;
    }
    if (DIR < 0) w.y = -w.y;
    return w;
  };
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) y[n2][k1] = cmul(y[n2][k1], tw16(n2 * k1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cplx<T> a[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
    dft4<DIR, T>(a);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = a[k2];
  }
}

template <int P, int DIR, typename T, bool PK = false>
__device__ __forceinline__ void small_dft(cplx<T>* v) {
  if (P == 2) dft2<DIR, T, PK>(v);
  else if (P == 4) dft4<DIR, T, PK>(v);
  else if (P == 8) dft8<DIR, T, PK>(v);
  else if (P == 16) dft16<DIR, T>(v);
}

// w_L^{DIR t} from the table tw[t] = exp(-2 pi i t / L)
template <int DIR, typename T>
__device__ __forceinline__ cplx<T> twl(const cplx<T>* tw, int t) {
  cplx<T> w = tw[t];
  if (DIR > 0) w.y = -w.y;
  return w;
}

// Radix-2 exchange stage h of the 32-point lane DFT, with sgn = -1 on the
// upper lane of each pair (lane bit h set) and +1 on the lower lane.
//   forward (decimation in frequency):  lower <- a + b,  upper <- (a - b) w
//     computed as  t = partner + sgn * own,  then  t * w' (w' = 1 on the lower lane)
//   inverse (decimation in time):       lower <- a + w b,  upper <- a - w b
//     computed as  own' = own * w' (w' = 1 on the lower lane), then partner' + sgn * own'
// where a and b are the lower and upper lane's values.  Every line of the
// warp takes the same twiddle, loaded once per stage.

// forward: natural (lane l, register j: point l + 32 j) -> bit-reversed
// frequencies (lane l, register q: frequency q + P * bitrev5(l)), NL lines
template <int P, int NL, typename T>
__device__ __forceinline__ void warp_fft_fwd(cplx<T> (&v)[NL][P], const cplx<T>* tw, int lane) {
  constexpr int L = 32 * P;
#pragma unroll
  for (int n = 0; n < NL; ++n) {
    small_dft<P, -1, T>(v[n]);
#pragma unroll
    for (int q = 1; q < P; ++q) v[n][q] = cmul(v[n][q], twl<-1, T>(tw, lane * q));
  }
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
    const T sgn = upper ? T(-1) : T(1);
    cplx<T> w;
    if (h > 1) {
      w = twl<-1, T>(tw, (lane & (h - 1)) * (L / (2 * h)));
      if (!upper) { w.x = T(1); w.y = T(0); }
    }
#pragma unroll
    for (int n = 0; n < NL; ++n)
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const cplx<T> p = shfl_xor_c<T>(v[n][q], h);
        cplx<T> t;
        t.x = fma(sgn, v[n][q].x, p.x);
        t.y = fma(sgn, v[n][q].y, p.y);
        v[n][q] = h > 1 ? cmul(t, w) : t;
      }
  }
}

// inverse (unnormalised): bit-reversed frequencies -> natural points, NL lines
template <int P, int NL, typename T>
__device__ __forceinline__ void warp_fft_inv(cplx<T> (&v)[NL][P], const cplx<T>* tw, int lane) {
  constexpr int L = 32 * P;
#pragma unroll
  for (int h = 1; h <= 16; h <<= 1) {
    const bool upper = (lane & h) != 0;
    const T sgn = upper ? T(-1) : T(1);
    cplx<T> w;
    if (h > 1) {
      w = twl<+1, T>(tw, (lane & (h - 1)) * (L / (2 * h)));
      if (!upper) { w.x = T(1); w.y = T(0); }
    }
#pragma unroll
    for (int n = 0; n < NL; ++n)
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const cplx<T> o = h > 1 ? cmul(v[n][q], w) : v[n][q];
        const cplx<T> p = shfl_xor_c<T>(o, h);
        v[n][q].x = fma(sgn, o.x, p.x);
        v[n][q].y = fma(sgn, o.y, p.y);
      }
  }
#pragma unroll
  for (int n = 0; n < NL; ++n) {
#pragma unroll
    for (int q = 1; q < P; ++q) v[n][q] = cmul(v[n][q], twl<+1, T>(tw, lane * q));
    small_dft<P, +1, T>(v[n]);
  }
}

// Paired form of the 32-point lane exchange, for P >= 2 values per lane:
// registers 2j and 2j+1 hold two independent lane DFTs (x and y).  In stage h
// the lower lane of each pair keeps x and sends y, the upper lane keeps y and
// sends x, so each lane receives one complex value and computes one whole
// radix-2 butterfly in registers: half the shuffles of warp_fft_fwd, and no
// multiplication by a unit twiddle.  After the five stages lane l, register q
// holds frequency pair_freq(l, q, P) (lane bit 4 then names the DFT of the
// pair, register bit 0 the lowest position bit); the inverse takes that layout
// back to natural order (lane l, register j: point l + 32 j).
__device__ __forceinline__ int pair_freq(int lane, int q, int P) {
  return 2 * (q >> 1) + (lane >> 4) + P * bitrev5(((lane & 15) << 1) | (q & 1));
}

template <int P, int NL, typename T, bool PK = false>
__device__ __forceinline__ void warp_fft_fwd_pairs(cplx<T> (&v)[NL][P], const cplx<T>* tw, int lane) {
  constexpr int L = 32 * P;
#pragma unroll
  for (int n = 0; n < NL; ++n) {
    small_dft<P, -1, T, PK>(v[n]);
#pragma unroll
    for (int q = 1; q < P; ++q) v[n][q] = cmul(v[n][q], twl<-1, T>(tw, lane * q));
  }
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
    const T sgn = upper ? T(-1) : T(1);
    cplx<T> w;
    if (h > 1) {
      w = twl<-1, T>(tw, (lane & (h - 1)) * (L / (2 * h)));
      w.x *= sgn;
      w.y *= sgn;
    }
#pragma unroll
    for (int n = 0; n < NL; ++n)
#pragma unroll
      for (int j = 0; j < P / 2; ++j) {
        const cplx<T> r0 = v[n][2 * j], r1 = v[n][2 * j + 1];
        const cplx<T> s = upper ? r1 : r0;
        const cplx<T> t = shfl_xor_c<T>(upper ? r0 : r1, h);
        v[n][2 * j] = kadd<PK>(s, t);
        const cplx<T> d = ksub<PK>(s, t);
        if (h > 1) {
          v[n][2 * j + 1] = cmul(d, w);
        } else if (PK) {
          v[n][2 * j + 1] = pscale(sgn, d);
        } else {
          v[n][2 * j + 1].x = sgn * d.x;
          v[n][2 * j + 1].y = sgn * d.y;
        }
      }
  }
}

template <int P, int NL, typename T, bool PK = false>
__device__ __forceinline__ void warp_fft_inv_pairs(cplx<T> (&v)[NL][P], const cplx<T>* tw, int lane) {
  constexpr int L = 32 * P;
#pragma unroll
  for (int h = 1; h <= 16; h <<= 1) {
    const bool upper = (lane & h) != 0;
    const T sgn = upper ? T(-1) : T(1);
    cplx<T> w;
    if (h > 1) {
      w = twl<+1, T>(tw, (lane & (h - 1)) * (L / (2 * h)));
      w.x *= sgn;
      w.y *= sgn;
    }
#pragma unroll
    for (int n = 0; n < NL; ++n)
#pragma unroll
      for (int j = 0; j < P / 2; ++j) {
        const cplx<T> r0 = v[n][2 * j], r1 = v[n][2 * j + 1];
        cplx<T> s2, d2;
        if (h > 1) {
          const cplx<T> u = cmul(r1, w);
          s2 = kadd<PK>(r0, u);
          d2 = ksub<PK>(r0, u);
        } else if (PK) {   // r0 +- sgn r1, one rounding each as in the fused scalar form
          s2 = pfma(sgn, r1, r0);
          d2 = pfma(-sgn, r1, r0);
        } else {
          cplx<T> u;
          u.x = sgn * r1.x;
          u.y = sgn * r1.y;
          s2 = cadd(r0, u);
          d2 = csub(r0, u);
        }
        const cplx<T> recv = shfl_xor_c<T>(d2, h);
        v[n][2 * j] = upper ? recv : s2;
        v[n][2 * j + 1] = upper ? s2 : recv;
      }
  }
#pragma unroll
  for (int n = 0; n < NL; ++n) {
#pragma unroll
    for (int q = 1; q < P; ++q) v[n][q] = cmul(v[n][q], twl<+1, T>(tw, lane * q));
    small_dft<P, +1, T, PK>(v[n]);
  }
}

// The warp line FFT used by the kernels: the paired exchange for P >= 2, the
// plain one for P = 1.  warp_freq gives the frequency that lane l, register q
// holds after the forward transform (and must hold before the inverse).
template <int P>
__device__ __forceinline__ int warp_freq(int lane, int q) {
  return P >= 2 ? pair_freq(lane, q, P) : q + P * bitrev5(lane);
}
// PK: packed two-wide FP32 additions (the row pass)
template <int P, int NL, typename T, bool PK = false>
__device__ __forceinline__ void warp_fft_fwd_any(cplx<T> (&v)[NL][P], const cplx<T>* tw, int lane) {
  if constexpr (P >= 2) warp_fft_fwd_pairs<P, NL, T, PK>(v, tw, lane);
  else warp_fft_fwd<P, NL, T>(v, tw, lane);
}
template <int P, int NL, typename T, bool PK = false>
__device__ __forceinline__ void warp_fft_inv_any(cplx<T> (&v)[NL][P], const cplx<T>* tw, int lane) {
  if constexpr (P >= 2) warp_fft_inv_pairs<P, NL, T, PK>(v, tw, lane);
  else warp_fft_inv<P, NL, T>(v, tw, lane);
}

// shared-memory index with one spare slot per 16 entries: the stride-P
// accesses of the bit-reversed layout then spread evenly over the banks
__device__ __forceinline__ int wpad(int i) { return i + (i >> 4); }

// rows 2a and 2a + 1 of one phase's 6 x 6 stiffness table (12 entries,
// 16-byte aligned), loaded with 16-byte accesses
template <typename T>
__device__ __forceinline__ void load_rows(const T* p, T (&d)[12]);
template <>
__device__ __forceinline__ void load_rows<float>(const float* p, float (&d)[12]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float4 v = q[i];
    d[4 * i] = v.x; d[4 * i + 1] = v.y; d[4 * i + 2] = v.z; d[4 * i + 3] = v.w;
  }
}
template <>
__device__ __forceinline__ void load_rows<double>(const double* p, double (&d)[12]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double2 v = q[i];
    d[2 * i] = v.x; d[2 * i + 1] = v.y;
  }
}

// Two independent 32-point lines transformed together with the paired lane
// exchange (line x in r0, line y in r1, lane l holding point l of each); after
// the forward stages lane l, register r holds line (l < 16 ? x : y) at
// frequency bitrev5(((l & 15) << 1) | r); the inverse undoes the stages.
template <typename T>
__device__ __forceinline__ void lane_pairs_fwd(cplx<T>& r0, cplx<T>& r1, const cplx<T>* tw, int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
    const T sgn = upper ? T(-1) : T(1);
    const cplx<T> s = upper ? r1 : r0;
    const cplx<T> t = shfl_xor_c<T>(upper ? r0 : r1, h);
    r0 = cadd(s, t);
    const cplx<T> d = csub(s, t);
    if (h > 1) {
      cplx<T> w = twl<-1, T>(tw, (lane & (h - 1)) * (16 / h));
      w.x *= sgn;
      w.y *= sgn;
      r1 = cmul(d, w);
    } else {
      r1.x = sgn * d.x;
      r1.y = sgn * d.y;
    }
  }
}
template <typename T>
__device__ __forceinline__ void lane_pairs_inv(cplx<T>& r0, cplx<T>& r1, const cplx<T>* tw, int lane) {
#pragma unroll
  for (int h = 1; h <= 16; h <<= 1) {
    const bool upper = (lane & h) != 0;
    const T sgn = upper ? T(-1) : T(1);
    cplx<T> u;
    if (h > 1) {
      cplx<T> w = twl<+1, T>(tw, (lane & (h - 1)) * (16 / h));
      w.x *= sgn;
      w.y *= sgn;
      u = cmul(r1, w);
    } else {
      u.x = sgn * r1.x;
      u.y = sgn * r1.y;
    }
    const cplx<T> s2 = cadd(r0, u);
    const cplx<T> recv = shfl_xor_c<T>(csub(r0, u), h);
    r0 = upper ? recv : s2;
    r1 = upper ? s2 : recv;
  }
}

// Lines of 32 points, two per warp at a time (the last one of an odd count
// paired with zeros), in place; ends with a team barrier.
template <int DIR, int PS, typename T>
__device__ __forceinline__ void warp_lines32_pairs(cplx<T>* buf, int nlines, int ls, const cplx<T>* tw, int tid,
                                                   int nthr) {
  const int lane = tid & 31, nwarps = nthr >> 5;
  const int half = lane >> 4;
  const int fpos = bitrev5(((lane & 15) << 1));   // frequency of register 0; register 1: fpos + 16
  for (int pr = tid >> 5; 2 * pr < nlines; pr += nwarps) {
    cplx<T>* bx = buf + (size_t)(2 * pr) * ls;
    const bool has_y = 2 * pr + 1 < nlines;
    cplx<T>* by = has_y ? bx + ls : bx;
    cplx<T>* mine = half ? by : bx;   // the line this lane holds after the forward stages
    cplx<T> r0, r1;
    if (DIR < 0) {
      r0 = bx[padi<PS>(lane)];
      if (has_y) r1 = by[padi<PS>(lane)];
      else { r1.x = T(0); r1.y = T(0); }
      lane_pairs_fwd<T>(r0, r1, tw, lane);
      __syncwarp();
      if (!half || has_y) {
        mine[padi<PS>(fpos)] = r0;
        mine[padi<PS>(fpos + 16)] = r1;
      }
    } else {
      if (!half || has_y) {
        r0 = mine[padi<PS>(fpos)];
        r1 = mine[padi<PS>(fpos + 16)];
      } else {
        r0.x = r0.y = r1.x = r1.y = T(0);
      }
      lane_pairs_inv<T>(r0, r1, tw, lane);
      __syncwarp();
      bx[padi<PS>(lane)] = r0;
      if (has_y) by[padi<PS>(lane)] = r1;
    }
    __syncwarp();
  }
  team_sync(nthr);
}

// In-place transform of `nlines` lines of length L = 32 P held in shared
// memory (line q at buf + q * ls, entry i at padi<PS>(i)), one warp per line,
// by the warps of a thread team (threads 0 .. nthr-1).  Forward takes natural
// order to natural order through the bit-reversed register layout of
// warp_fft_fwd; inverse (unnormalised) likewise.  Ends with a team barrier.
template <int DIR, int P, int PS, typename T>
__device__ __forceinline__ void warp_lines(cplx<T>* buf, int nlines, int ls, const cplx<T>* tw, int tid, int nthr) {
  const int lane = tid & 31, nwarps = nthr >> 5;
  for (int line = tid >> 5; line < nlines; line += nwarps) {
    cplx<T>* b = buf + (size_t)line * ls;
    cplx<T> v[1][P];
    if (DIR < 0) {
#pragma unroll
      for (int j = 0; j < P; ++j) v[0][j] = b[padi<PS>(lane + 32 * j)];
      warp_fft_fwd_any<P, 1, T>(v, tw, lane);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < P; ++q) b[padi<PS>(warp_freq<P>(lane, q))] = v[0][q];
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) v[0][q] = b[padi<PS>(warp_freq<P>(lane, q))];
      warp_fft_inv_any<P, 1, T>(v, tw, lane);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < P; ++j) b[padi<PS>(lane + 32 * j)] = v[0][j];
    }
    __syncwarp();
  }
  team_sync(nthr);
}

// warp_lines for a runtime line length L (32, 64, 128, 256 or 512); returns
// false (and does nothing) for any other length
template <int DIR, int PS, typename T>
__device__ __forceinline__ bool warp_lines_any(cplx<T>* buf, int nlines, int ls, int L, const cplx<T>* tw, int tid,
                                               int nthr) {
  switch (L) {
    case 32: warp_lines32_pairs<DIR, PS, T>(buf, nlines, ls, tw, tid, nthr); return true;
    case 64: warp_lines<DIR, 2, PS, T>(buf, nlines, ls, tw, tid, nthr); return true;
    case 128: warp_lines<DIR, 4, PS, T>(buf, nlines, ls, tw, tid, nthr); return true;
    case 256: warp_lines<DIR, 8, PS, T>(buf, nlines, ls, tw, tid, nthr); return true;
    case 512: warp_lines<DIR, 16, PS, T>(buf, nlines, ls, tw, tid, nthr); return true;
    default: return false;
  }
}

// Forward row transform of a 2-D cluster CTA with the split into half
// spectra done by the warp that owns the line (no block barrier between
// transform and split).  Line p carries the real rows 2p and 2p+1 (the last
// one zero when nreal is odd) as real and imaginary parts: natural order in
// `buf` -> forward transform -> A = (Z_k + conj Z_{L-k}) / 2 and
// B = (Z_k - conj Z_{L-k}) / 2i written to `S` (rows of H entries, natural
// order); `buf` serves as the warp's staging line.
template <int P, int PS, typename T>
__device__ __forceinline__ void warp_rows_fwd_split(cplx<T>* buf, int nlines, int ls, cplx<T>* S, int H, int nreal,
                                                    const cplx<T>* tw, int tid, int nthr) {
  constexpr int L = 32 * P;
  const int lane = tid & 31, nwarps = nthr >> 5;
  for (int line = tid >> 5; line < nlines; line += nwarps) {
    cplx<T>* b = buf + (size_t)line * ls;
    cplx<T> v[1][P];
#pragma unroll
    for (int j = 0; j < P; ++j) v[0][j] = b[padi<PS>(lane + 32 * j)];
    warp_fft_fwd_any<P, 1, T>(v, tw, lane);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < P; ++q) b[padi<PS>(warp_freq<P>(lane, q))] = v[0][q];
    __syncwarp();
    const int fa = 2 * line, fb = fa + 1;
    for (int k = lane; k < H; k += 32) {
      const cplx<T> zk = b[padi<PS>(k)];
      const cplx<T> zm = b[padi<PS>(k == 0 ? 0 : L - k)];
      cplx<T> A, B;
      A.x = T(0.5) * (zk.x + zm.x);
      A.y = T(0.5) * (zk.y - zm.y);
      B.x = T(0.5) * (zk.y + zm.y);
      B.y = T(-0.5) * (zk.x - zm.x);
      S[fa * H + k] = A;
      if (fb < nreal) S[fb * H + k] = B;
    }
    __syncwarp();
  }
}

// the above for a runtime row length L (32..512); false for other lengths
template <int PS, typename T>
__device__ __forceinline__ bool warp_rows_fwd_split_any(cplx<T>* buf, int nlines, int ls, int L, cplx<T>* S, int H,
                                                        int nreal, const cplx<T>* tw, int tid, int nthr) {
  switch (L) {
    case 32: warp_rows_fwd_split<1, PS, T>(buf, nlines, ls, S, H, nreal, tw, tid, nthr); return true;
    case 64: warp_rows_fwd_split<2, PS, T>(buf, nlines, ls, S, H, nreal, tw, tid, nthr); return true;
    case 128: warp_rows_fwd_split<4, PS, T>(buf, nlines, ls, S, H, nreal, tw, tid, nthr); return true;
    case 256: warp_rows_fwd_split<8, PS, T>(buf, nlines, ls, S, H, nreal, tw, tid, nthr); return true;
    case 512: warp_rows_fwd_split<16, PS, T>(buf, nlines, ls, S, H, nreal, tw, tid, nthr); return true;
    default: return false;
  }
}

constexpr int kWarpRowThreads = 256;

// Rows are dealt to the warps of the grid round-robin; a launch sizes its grid
// to the resident blocks, so every warp handles many rows and the block
// barrier of the residual reduction is met once per launch.  All global loads
// of a row (half spectra, old strain, phase indices) are issued together
// before any of them is used.
// KINV (with FIRST = false): the inverse half of a Krylov operator
// application, as in row_pass: W = X - y to Wout (X = E, y the inverse
// transform), block sums of W . Yaux (Yaux = X when null) and W . W.
template <typename T, int P, bool FIRST, bool KINV = false>
__global__ void __launch_bounds__(kWarpRowThreads, (P <= 4 ? 2 : 1)) row_pass_warp6(GridInfo g, const cplx<T>* __restrict__ twg,
                                                                  T* __restrict__ E, cplx<T>* __restrict__ S,
                                                                  const uint8_t* __restrict__ phase,
                                                                  const T* __restrict__ dC, Control* ctl,
                                                                  LoadState* st, double* __restrict__ partials,
                                                                  double* __restrict__ hist, int blocks_per_load,
                                                                  T* __restrict__ Wout = nullptr,
                                                                  const T* __restrict__ Yaux = nullptr) {
  static_assert(!(FIRST && KINV), "the inverse-only pass follows a transform");
  constexpr int NV = 6, L = 32 * P, H = L / 2 + 1;
  constexpr int WS = ((6 * H > 3 * L ? 6 * H : 3 * L) * 17 + 15) / 16 + 2;
  constexpr int NW = kWarpRowThreads / 32;
  constexpr int KI = (H + 31) / 32;   // half-spectrum entries per lane and component
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);          // L
  cplx<T>* scratch = tw + L;                                    // NW * WS
  __shared__ __align__(16) T dcs[16 * NV * NV];
  __shared__ __align__(16) T dcp[16 * 12];   // the 12 nonzeros of decoupled phase matrices
  __shared__ double red[32];
  __shared__ int s_skip;
  const int load = blockIdx.x / blocks_per_load;
  const int qb = blockIdx.x - load * blocks_per_load;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool decoupled = ctl->decoupled != 0;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < 16 * NV * NV; i += blockDim.x) dcs[i] = dC[i];
  if (decoupled)
    for (int i = threadIdx.x; i < 16 * 12; i += blockDim.x) dcp[i] = decoupled_entry(dC + (i / 12) * NV * NV, i % 12);
  if (threadIdx.x == 0) s_skip = st[load].done;
  __syncthreads();
  ResAcc<T> acc_d, acc_n;
  cplx<T>* ws = scratch + warp * WS;
  if (!s_skip) {
    T e0[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) e0[c] = (T)ctl->eps0[load][c];
    const T scale = (T)g.inv_m;
    const bool incremental = ctl->form == 1;
    const size_t cstrS = (size_t)g.nrows * H;
    const size_t cstrE = (size_t)g.m;
    const T* Eload = E + (size_t)load * NV * cstrE;
    cplx<T>* Sload = S + (size_t)load * NV * cstrS;
    for (long long row = (long long)qb * NW + warp; row < g.nrows; row += (long long)blocks_per_load * NW) {
      // checked build: the largest S, E, phase and scratch offsets of the row
      // (every access of the row lies between the row's first and these)
      if (!(FH_IN(CK_WROW_S, ((long long)load * NV + NV - 1) * (long long)cstrS + row * H + H - 1,
                  (long long)ctl->nload * NV * g.nhalf) &&
            FH_IN(CK_WROW_E, ((long long)load * NV + NV - 1) * (long long)cstrE + row * L + L - 1,
                  (long long)ctl->nload * NV * g.m) &&
            FH_IN(CK_WROW_PHASE, row * L + L - 1, g.m) &&
            FH_IN(CK_WROW_SCRATCH, wpad((6 * H > 3 * L ? 6 * H : 3 * L) - 1), WS)))
        continue;
      T* Er = E + (size_t)load * NV * cstrE + row * L;
      cplx<T>* Sr = Sload + row * H;
      // 1. every global load of the row
      cplx<T> sv[NV][KI];
      T ev[NV][P];
      int ph[P];
      if (!FIRST) {
#pragma unroll
        for (int c = 0; c < NV; ++c)
#pragma unroll
          for (int i = 0; i < KI; ++i) {
            const int k = lane + 32 * i;
            if (k < H) sv[c][i] = Sr[c * cstrS + k];
          }
      }
#pragma unroll
      for (int c = 0; c < NV; ++c)
#pragma unroll
        for (int j = 0; j < P; ++j) ev[c][j] = Eload[c * cstrE + row * L + lane + 32 * j];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        ph[j] = KINV ? 0 : phase[row * L + lane + 32 * j];
        if (!FH_IN(CK_WROW_PHASE, ph[j], 16)) ph[j] = 0;
      }
      cplx<T> z[3][P];
      if (!FIRST) {
        // 2. Z = A + i B per line pair from the half spectra, inverse FFT
#pragma unroll
        for (int c = 0; c < NV; ++c)
#pragma unroll
          for (int i = 0; i < KI; ++i) {
            const int k = lane + 32 * i;
            if (k < H) ws[wpad(c * H + k)] = sv[c][i];
          }
        __syncwarp();
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = 0; q < P; ++q) {
            const int k = warp_freq<P>(lane, q);
            const bool lo = k <= L / 2;
            const int kk = lo ? k : L - k;
            cplx<T> A = ws[wpad((2 * p) * H + kk)], B = ws[wpad((2 * p + 1) * H + kk)];
            if (!lo) { A.y = -A.y; B.y = -B.y; }
            z[p][q].x = A.x - B.y;
            z[p][q].y = A.y + B.x;
          }
        __syncwarp();
        warp_fft_inv_any<P, 3, T, true>(z, tw, lane);
      }
      if constexpr (KINV) {
        const T* Yl = Yaux ? Yaux + (size_t)load * NV * cstrE : Eload;
        T* Wl = Wout + (size_t)load * NV * cstrE;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const size_t x = row * L + lane + 32 * j;
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            const T w = ev[c][j] - ((c & 1) ? z[c >> 1][j].y : z[c >> 1][j].x) * scale;
            Wl[c * cstrE + x] = w;
            acc_d.add_prod(w, Yaux ? Yl[c * cstrE + x] : ev[c][j]);
            acc_n.add_sq(w);
          }
        }
        continue;
      }
      // 3. pointwise: E_new, residual sums, tau
      T rd = T(0), rn = T(0);
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const int x = lane + 32 * j;
        T en[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          if (FIRST) {
            en[c] = ev[c][j];
          } else {
            en[c] = ((c & 1) ? z[c >> 1][j].y : z[c >> 1][j].x) * scale;
            if (incremental) en[c] += ev[c][j];
            const T dd = en[c] - ev[c][j], nn = en[c] + e0[c];
            rd = fma(dd, dd, rd);
            rn = fma(nn, nn, rn);
            Er[c * cstrE + x] = en[c];
          }
        }
        if (decoupled) {
          T dc[12], xv[NV], tau[NV];
          load_rows<T>(dcp + ph[j] * 12, dc);
#pragma unroll
          for (int b = 0; b < NV; ++b) xv[b] = en[b] + e0[b];
          stress6_decoupled<T>(dc, xv, tau);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            z[a][j].x = tau[2 * a];
            z[a][j].y = tau[2 * a + 1];
          }
        } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          T dc[12];
          load_rows<T>(dcs + ph[j] * NV * NV + 12 * a, dc);
          T t0 = T(0), t1 = T(0);
#pragma unroll
          for (int b = 0; b < NV; ++b) {
            t0 = fma(dc[b], en[b] + e0[b], t0);
            t1 = fma(dc[NV + b], en[b] + e0[b], t1);
          }
          z[a][j].x = t0;
          z[a][j].y = t1;
        }
        }
      }
      if (!FIRST) {
        acc_d.add(rd);
        acc_n.add(rn);
      }
      // 4. forward FFT, then split each line's spectrum into the half
      //    spectra of its two components
      warp_fft_fwd_any<P, 3, T, true>(z, tw, lane);
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < P; ++q) ws[wpad(p * L + warp_freq<P>(lane, q))] = z[p][q];
      __syncwarp();
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int i = 0; i < KI; ++i) {
          const int k = lane + 32 * i;
          if (k < H) {
            const cplx<T> zk = ws[wpad(p * L + k)];
            const cplx<T> zm = ws[wpad(p * L + (k == 0 ? 0 : L - k))];
            cplx<T> A, B;
            A.x = T(0.5) * (zk.x + zm.x);
            A.y = T(0.5) * (zk.y - zm.y);
            B.x = T(0.5) * (zk.y + zm.y);
            B.y = T(-0.5) * (zk.x - zm.x);
            Sr[(2 * p) * cstrS + k] = A;
            Sr[(2 * p + 1) * cstrS + k] = B;
          }
        }
      __syncwarp();
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

template <typename T>
__host__ inline size_t warprow_smem(int L) {
  const int H = L / 2 + 1;
  const int ws = ((6 * H > 3 * L ? 6 * H : 3 * L) * 17 + 15) / 16 + 2;
  return (size_t)(L + (kWarpRowThreads / 32) * ws) * sizeof(T) * 2;
}

}  // namespace fh
