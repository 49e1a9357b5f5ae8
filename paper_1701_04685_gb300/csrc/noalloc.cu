// Allocation-free variant of the mean-stress reduction (fh_mean_stress_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a result:
// real-time or latency-bound loops where an allocation may block or fail, and
// applications (a larger simulation that embeds this solver, for example)
// whose device memory is owned entirely by their own arena allocator with a
// fixed budget.  For them this entry point keeps all of its scratch -- the
// per-block partial sums, the block counter, an error word and the result --
// in one fixed array that lives in the library image, so no call ever
// allocates.  The caller passes the inputs (strain field, phase ids, phase
// stiffnesses, macroscopic strains) and the output buffer.
//
// The array is a host-side symbol in host code; its device address is looked
// up with cudaGetSymbolAddress once per device, on the first call made while
// that device is current, and cached.  That first call should come before any
// stream capture.  The cached address belongs to the device's context of that
// moment: after cudaDeviceReset the next context has a new copy of the array,
// so a process that resets a device must not call this entry point again.
// Every call shares the array: calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it.  Each call synchronises its
// stream before it returns.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>

#include "internal.hpp"

namespace {

constexpr int kMaxV = 6;                       // Mandel components, n_v <= 6
constexpr int kNaMaxLoads = FH_MAX_LOADS;      // 16 load cases
constexpr int kNaMaxBlocks = 64;               // blocks per load case
constexpr int kNaPartials = kNaMaxLoads * kNaMaxBlocks * kMaxV;
constexpr int kNaOut = kNaMaxLoads * kMaxV;
constexpr int kNaTotal = kNaPartials + kNaOut + 32;  // + block counter and error word

// 6272 doubles = 49 KB, resident on every GPU that loads the library.
static __device__ __align__(256) double g_noalloc_scratch[kNaTotal];

__device__ __forceinline__ double na_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block sum in a fixed order; the result is valid in thread 0
__device__ __forceinline__ double na_block_sum(double v, double* red) {
  v = na_warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < (int)((blockDim.x + 31) >> 5) ? red[lane] : 0.0;
    t = na_warp_sum(t);
  }
  return t;
}

struct NaParams {
  double Cp[16 * 36];
  double eps0[kNaMaxLoads * 6];
  int nphase, nv, nload;
  long long m;
};

__global__ void __launch_bounds__(256) mean_stress_noalloc(NaParams P, const double* __restrict__ E,
                                                           const uint8_t* __restrict__ phase, double* scratch,
                                                           int blocks_per_load) {
  __shared__ double red[32];
  __shared__ unsigned int s_ticket;
  double* partials = scratch;
  double* out = scratch + kNaPartials;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNaPartials + kNaOut);
  unsigned int* bad_id = ticket + 1;  // set when a phase id >= nphase is met
  const int load = blockIdx.x / blocks_per_load;
  const int q = blockIdx.x - load * blocks_per_load;
  const int nv = P.nv;
  double acc[kMaxV] = {0, 0, 0, 0, 0, 0};
  const size_t base = (size_t)load * nv * P.m;
  for (long long i = (long long)q * blockDim.x + threadIdx.x; i < P.m; i += (long long)blocks_per_load * blockDim.x) {
    const int ph = phase[i];
    if (ph >= P.nphase) {  // never index the parameter block with an id it does not hold
      *bad_id = 1u;
      continue;
    }
    double e[kMaxV];
    for (int c = 0; c < nv; ++c) e[c] = E[base + (size_t)c * P.m + i] + P.eps0[load * 6 + c];
    const double* C = P.Cp + ph * 36;
    for (int a = 0; a < nv; ++a) {
      double s = 0.0;
      for (int b = 0; b < nv; ++b) s += C[a * nv + b] * e[b];
      acc[a] += s;
    }
  }
  for (int a = 0; a < nv; ++a) {
    const double v = na_block_sum(acc[a], red);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMaxV + a] = v;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_ticket = atomicAdd(ticket, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  for (int l = 0; l < P.nload; ++l)
    for (int a = 0; a < nv; ++a) {
      double s = 0.0;
      for (int qq = threadIdx.x; qq < blocks_per_load; qq += blockDim.x)
        s += __ldcg(&partials[((size_t)l * blocks_per_load + qq) * kMaxV + a]);
      s = na_block_sum(s, red);
      if (threadIdx.x == 0) out[l * kMaxV + a] = s / (double)P.m;
    }
  if (threadIdx.x == 0) *ticket = 0u;
}

// device address of the scratch array, looked up once per device; the slots are
// atomic so that host threads calling on different devices at once do not race
double* scratch_address(int device, fh_status* rc) {
  static std::atomic<double*> addr[64];  // static storage: every slot starts null
  if (device < 0 || device >= 64) {
    fh::set_error("device ordinal out of range");
    *rc = FH_ERR_ARG;
    return nullptr;
  }
  double* a = addr[device].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      fh::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      *rc = FH_ERR_CUDA;
      return nullptr;
    }
    a = static_cast<double*>(p);
    addr[device].store(a, std::memory_order_release);  // every thread finds the same address
  }
  *rc = FH_OK;
  return a;
}

}  // namespace

extern "C" fh_status fh_mean_stress_noalloc(int d, long long m, int nload, const double* E, const uint8_t* phase,
                                            int nphase, const double* Cp, const double* eps0, double* mean_stress,
                                            void* cuda_stream) {
  if (d != 2 && d != 3) { fh::set_error("d must be 2 or 3"); return FH_ERR_ARG; }
  if (!E || !phase || !Cp || !eps0 || !mean_stress) { fh::set_error("null argument"); return FH_ERR_ARG; }
  if (m < 1) { fh::set_error("m must be positive"); return FH_ERR_ARG; }
  if (nload < 1 || nload > kNaMaxLoads) {
    fh::set_error("nload must be 1..16: the fixed scratch array holds partial sums for at most 16 load cases");
    return FH_ERR_ARG;
  }
  if (nphase < 1 || nphase > 16) { fh::set_error("nphase must be 1..16"); return FH_ERR_ARG; }
  const int nv = d == 2 ? 3 : 6;
  NaParams P{};
  for (int q = 0; q < nphase; ++q)
    for (int a = 0; a < nv; ++a)
      for (int b = 0; b < nv; ++b) P.Cp[q * 36 + a * nv + b] = Cp[(q * nv + a) * nv + b];
  for (int l = 0; l < nload; ++l)
    for (int c = 0; c < nv; ++c) {
      P.eps0[l * 6 + c] = eps0[l * nv + c];
      if (!std::isfinite(eps0[l * nv + c])) { fh::set_error("non-finite eps0"); return FH_ERR_ARG; }
    }
  P.nphase = nphase;
  P.nv = nv;
  P.nload = nload;
  P.m = m;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { fh::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return FH_ERR_CUDA; }
  fh_status rc;
  double* scratch = scratch_address(dev, &rc);
  if (!scratch) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNaPartials + kNaOut);
  e = cudaMemsetAsync(ticket, 0, 2 * sizeof(unsigned int), st);  // block counter and error word start at zero
  if (e != cudaSuccess) { fh::set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)); return FH_ERR_CUDA; }
  const int bpl = (int)std::min<long long>((m + 255) / 256, kNaMaxBlocks);
  mean_stress_noalloc<<<nload * bpl, 256, 0, st>>>(P, E, phase, scratch, bpl);
  e = cudaGetLastError();
  if (e != cudaSuccess) { fh::set_error(std::string("launch: ") + cudaGetErrorString(e)); return FH_ERR_CUDA; }
  // gather the (nload x MAXV) result rows into the caller's nload x nv buffer
  for (int l = 0; l < nload; ++l) {
    e = cudaMemcpyAsync(mean_stress + l * nv, scratch + kNaPartials + l * kMaxV, nv * sizeof(double),
                        cudaMemcpyDefault, st);
    if (e != cudaSuccess) { fh::set_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e)); return FH_ERR_CUDA; }
  }
  unsigned int bad = 0;
  e = cudaMemcpyAsync(&bad, ticket + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) { fh::set_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e)); return FH_ERR_CUDA; }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { fh::set_error(std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e)); return FH_ERR_CUDA; }
  if (bad) {
    fh::set_error("a phase id >= nphase was found; the mean stress written is not valid");
    return FH_ERR_ARG;
  }
  return FH_OK;
}
