// Tensor-core (tcgen05) form of the network's hidden 1 x 1 layers:
//
//   u[b][o][p] = sum_c W[o][c] v[b][c][p] + w[o] (+ s[b][o][p]),   v' = gelu(u),
//
// for W channels in and out (W = 16, 32 or 64).  One CTA of 128 threads takes
// tiles of 128 voxels: the tile is a GEMM D[p][o] = A[p][c] B[o][c] with
// M = 128 voxels, N = W outputs, accumulated in FP32 in tensor memory (TMEM).
// The weights are BF16 (as in the SIMT layer); each FP32 activation is split
// into three BF16 terms, v = hi + mid + lo (hi = bf16(v), mid = bf16(v - hi),
// lo = bf16(v - hi - mid)), which represent it to about 2^-24 relative, and
// the three terms form one operand of K = 3 W columns against the weights
// repeated three times, so one MMA sequence sums all of hi W + mid W + lo W.
// Operands sit in shared memory in the K-major layout without swizzle: 8 x 8
// BF16 core matrices of 128 bytes, core matrices along K 128 B apart (the
// leading-dimension offset), 8-row groups K/8 * 128 B apart (the stride
// offset).  One thread issues the MMAs (tcgen05.mma, kind::f16, BF16 inputs,
// FP32 accumulator), tcgen05.commit signals an mbarrier, and each warp reads
// its 32 TMEM lanes (32 voxels x W columns) with tcgen05.ld for the epilogue
// (bias, the spectral branch, GELU) with coalesced stores along the voxels.
// Waits on the mbarrier give up after a bounded number of polls: the kernel
// then records an error and frees its TMEM before returning.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace fhtc {

constexpr int kTcThreads = 128;
constexpr int kTcTile = 128;   // voxels per tile = MMA M

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle (layout type 0),
// descriptor version 1, base offset 0
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcTile >> 4) << 24);
}

// byte offset of element (r, k) of a K-major operand with K columns
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ float gelu_tc(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* r);

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float* r) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(v[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float* r) {
  tmem_ld<16>(taddr, r);
  tmem_ld<16>(taddr + 16, r + 16);
}

template <>
__device__ __forceinline__ void tmem_ld<64>(uint32_t taddr, float* r) {
  tmem_ld<32>(taddr, r);
  tmem_ld<32>(taddr + 32, r + 32);
}

// Hidden layer on tensor cores; requires N3 % 128 == 0.  err: set to 1 when an
// mbarrier wait gave up (the outputs are then not valid).
template <int W>
__global__ void __launch_bounds__(kTcThreads, 1) k_pointwise_tc(int B, int N3, const __nv_bfloat16* __restrict__ Wbf,
                                                               const float* __restrict__ bias,
                                                               const float* __restrict__ x,
                                                               const float* __restrict__ add,
                                                               float* __restrict__ u_out, float* __restrict__ y,
                                                               int act, int* err) {
  constexpr int K3 = 3 * W;                          // split-BF16 K
  constexpr int NCOL = W < 32 ? 32 : W;              // TMEM columns (power of two >= 32)
  static_assert(W % 16 == 0 && W <= 64, "W must be 16, 32 or 64");
  __shared__ __align__(1024) __nv_bfloat16 As[kTcTile * K3];
  __shared__ __align__(1024) __nv_bfloat16 Bs[W * K3];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* Ab = reinterpret_cast<unsigned char*>(As);
  unsigned char* Bb = reinterpret_cast<unsigned char*>(Bs);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // B' = [W | W | W]: row o, column k' -> W[o][k' mod W]
  for (int i = tid; i < W * K3; i += kTcThreads) {
    const int o = i / K3, k = i - o * K3;
    *reinterpret_cast<__nv_bfloat16*>(Bb + kmajor_off(o, k, K3)) = Wbf[o * W + (k % W)];
  }
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(W);
  const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
  const int tiles_per_sample = N3 / kTcTile;
  const int ntiles = B * tiles_per_sample;
  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = tile / tiles_per_sample;
    const int p0 = (tile - b * tiles_per_sample) * kTcTile;
    // A' = [hi | mid | lo] of the activations: thread tid owns voxel row tid
    for (int c = 0; c < W; ++c) {
      const float v = x[((size_t)b * W + c) * N3 + p0 + tid];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(hi);
      const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
      const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
      *reinterpret_cast<__nv_bfloat16*>(Ab + kmajor_off(tid, c, K3)) = hi;
      *reinterpret_cast<__nv_bfloat16*>(Ab + kmajor_off(tid, W + c, K3)) = mid;
      *reinterpret_cast<__nv_bfloat16*>(Ab + kmajor_off(tid, 2 * W + c, K3)) = lo;
    }
    // the operands written by the threads become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int kk = 0; kk < K3 / 16; ++kk) {
        // 16 columns = two core matrices along K = 256 bytes further on
        const uint64_t ad = sdesc(a0 + kk * 256, 128, (K3 / 8) * 128);
        const uint64_t bd = sdesc(b0 + kk * 256, 128, (K3 / 8) * 128);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_addr(&mbar))
                   : "memory");
    }
    // wait for the MMAs (bounded)
    {
      uint32_t done = 0;
      for (int it = 0; it < (1 << 20) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(&mbar)), "r"(phase)
            : "memory");
      }
      if (!done) s_abort = 1;
    }
    __syncthreads();
    if (s_abort) {
      if (tid == 0) atomicExch(err, 1);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: warp w holds voxels 32 w .. 32 w + 31 in its TMEM lanes
    float r[W];
    tmem_ld<W>(tmem + ((uint32_t)(32 * warp) << 16), r);
    const int p = p0 + 32 * warp + lane;
#pragma unroll
    for (int o = 0; o < W; ++o) {
      const size_t oi = ((size_t)b * W + o) * N3 + p;
      float a = r[o] + bias[o];
      if (add) a += add[oi];
      if (u_out) u_out[oi] = a;
      y[oi] = act ? gelu_tc(a) : a;
    }
    // every warp has read the accumulator before the next tile's MMAs overwrite it
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
}

}  // namespace fhtc
