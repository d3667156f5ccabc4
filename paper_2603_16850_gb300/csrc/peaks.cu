// Peak-rate microbenchmarks of the GPU the library runs on (deer_measure_peak): the
// denominators of the rooflines the benchmark reports for the ALU- and tensor-bound
// kernels. Every kernel runs on all SMs (the SM count is read from the device), its work is
// counted exactly, and it is timed with CUDA events on the caller's stream (best of several
// launches after warm-up).
//   FP32 FMA: independent chains of the packed two-wide FMA and of the scalar FMA per
//             thread, 2048 threads per SM; the faster of the two is the FP32 peak.
//   FP64 FMA: independent scalar chains, 2048 threads per SM.
//   tcgen05:  one CTA per SM whose elected thread issues back-to-back dense MMAs
//             (M = 128, N = 256, K = 8 for kind::tf32 or 16 for kind::f16 with bf16
//             operands) on operands resident in shared memory, accumulating in tensor
//             memory; all MMAs are committed to an mbarrier that the CTA waits on
//             (bounded).
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc.cuh"

namespace deer {
namespace {

__device__ float g_sink_f;
__device__ double g_sink_d;
__device__ int g_peak_timeout;

constexpr int kChains = 8;

__global__ void __launch_bounds__(512) k_peak_ffma2(int iters, float seed) {
  float2 a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j)
    a[j] = make_float2(seed + (float)(threadIdx.x + j), seed - (float)j);
  const float2 m = make_float2(0.9999999f, 1.0000001f), c = make_float2(1e-7f, -1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j].x + a[j].y;
  if (s == 1.2345f) g_sink_f = s;  // keeps the chains from being removed
}

__global__ void __launch_bounds__(512) k_peak_ffma(int iters, float seed) {
  float a[2 * kChains];
#pragma unroll
  for (int j = 0; j < 2 * kChains; ++j) a[j] = seed + (float)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 2 * kChains; ++j) a[j] = __fmaf_rn(a[j], 0.9999999f, 1e-7f);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 2 * kChains; ++j) s += a[j];
  if (s == 1.2345f) g_sink_f = s;
}

__global__ void __launch_bounds__(512) k_peak_dfma(int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = seed + (double)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = __fma_rn(a[j], 0.9999999999, 1e-12);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1.2345) g_sink_d = s;
}

// dense tcgen05 MMAs, M = 128, N = 256; operands: 128 x 32 B (A) and 256 x 32 B (B) in the
// canonical no-swizzle K-major layout, filled with hashed values of magnitude 0.5 to 1 and
// random signs (operands of realistic bit activity: the power a tensor core draws, and so
// the clock it holds, depends on the data)
constexpr int kMmaM = 128, kMmaN = 256;
constexpr unsigned kPeakWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// a word of operand data: two bf16 or one tf32 value with exponent 126 (|v| in [0.5, 1))
template <bool BF16>
__device__ __forceinline__ uint32_t operand_word(uint32_t i) {
  const uint32_t h = hash32(i * 2654435761u + 12345u);
  if (BF16) return (h & 0x807F807Fu) | 0x3F003F00u;
  return (h & 0x807FE000u) | 0x3F000000u;
}

template <bool BF16>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int n_mma) {
  __shared__ __align__(1024) unsigned char A[kMmaM * 32];
  __shared__ __align__(1024) unsigned char B[kMmaN * 32];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x;
  for (int i = tid; i < kMmaM * 32 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(A)[i] = operand_word<BF16>(i);
  for (int i = tid; i < kMmaN * 32 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(B)[i] = operand_word<BF16>(i + 4096);
  const uint32_t bar = tc::su32(&mbar);
  if (tid == 0) tc::bar_init(bar, 1);
  if (tid < 32) tc::tmem_alloc(tc::su32(&tmem_sh), kMmaN);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_sh;
  if (tid == 0) {
    const uint64_t ad = tc::sdesc(tc::su32(A), (kMmaM / 8) * 128, 128);
    const uint64_t bd = tc::sdesc(tc::su32(B), (kMmaN / 8) * 128, 128);
    if (BF16) {
      const uint32_t id = tc::idesc_bf16(kMmaN, kMmaM);
      for (int i = 0; i < n_mma; ++i) tc::mma_f16(tmem, ad, bd, id, i > 0 ? 1u : 0u);
    } else {
      const uint32_t id = tc::idesc_tf32(kMmaN, kMmaM);
      for (int i = 0; i < n_mma; ++i) tc::mma_tf32(tmem, ad, bd, id, i > 0 ? 1u : 0u);
    }
    tc::mma_commit(bar);
  }
  const bool ok = tc::bar_wait(bar, 0, kPeakWaitLimit);
  if (!ok && tid == 0) atomicExch(&g_peak_timeout, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid < 32) tc::tmem_dealloc(tmem, kMmaN);
}

}  // namespace
}  // namespace deer

using namespace deer;

extern "C" deer_status deer_measure_peak(int32_t what, deer_stream_t stream,
                                         double* flops_per_s) {
  if (!flops_per_s || what < 0 || what > 3) return DEER_ERR_INVALID;
  *flops_per_s = 0.0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    return DEER_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DEER_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DEER_ERR_CUDA;
  }
  const int zero = 0;
  cudaMemcpyToSymbolAsync(g_peak_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  double best = 0.0;
  const int kVariants = what == 0 ? 2 : 1;
  deer_status ret = DEER_OK;
  for (int v = 0; v < kVariants && ret == DEER_OK; ++v) {
    // work per launch (flop) and the launch itself
    double flop = 0.0;
    auto launch = [&]() {
      if (what == 0) {
        const int iters = 8192;
        flop = 2.0 * 2 * kChains * iters * (double)sms * 4 * 512;
        if (v == 0) k_peak_ffma2<<<sms * 4, 512, 0, st>>>(iters, 1.f);
        else k_peak_ffma<<<sms * 4, 512, 0, st>>>(iters, 1.f);
      } else if (what == 1) {
        const int iters = 512;
        flop = 2.0 * kChains * iters * (double)sms * 4 * 512;
        k_peak_dfma<<<sms * 4, 512, 0, st>>>(iters, 1.0);
      } else {
        const int n = 4096;
        const int k = what == 3 ? 16 : 8;
        flop = 2.0 * kMmaM * kMmaN * k * (double)n * sms;
        if (what == 3) k_peak_mma<true><<<sms, 128, 0, st>>>(n);
        else k_peak_mma<false><<<sms, 128, 0, st>>>(n);
      }
      note_launch();
    };
    for (int r = 0; r < 7; ++r) {
      if (cudaEventRecord(e0, st) != cudaSuccess) { ret = DEER_ERR_CUDA; break; }
      launch();
      if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess) {
        ret = DEER_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { ret = DEER_ERR_CUDA; break; }
      if (r >= 2 && ms > 0.f) {
        const double rate = flop / (ms * 1e-3);
        if (rate > best) best = rate;
      }
    }
  }
  int timed_out = 0;
  if (ret == DEER_OK &&
      (cudaMemcpyFromSymbol(&timed_out, g_peak_timeout, sizeof(int)) != cudaSuccess))
    ret = DEER_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ret != DEER_OK) return ret;
  if (timed_out) return DEER_ERR_TIMEOUT;
  *flops_per_s = best;
  return DEER_OK;
}
