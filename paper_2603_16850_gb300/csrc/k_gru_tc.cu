// GRU (d = d_in = 64, float32) linearisation on the 5th-generation tensor cores.
//
// Per row t with h = s_{t-1} the step needs three products with fixed 64 x 64 weights
// (GRU cell with zero biases, as in k_gru.cu):
//   G1 = h [Uz; Ur]^T (128 outputs), G2 = (r o h) Uh^T, G3 = (h o r o (1 - r)) M^T,
// M = Uh o Ur^T. For a tile of 128 rows these are 128 x N x 64 matrix products with the
// weights shared by every row, i.e. real GEMMs: they run as tcgen05.mma (kind::tf32) with
// the float32 accumulators in tensor memory. float32 accuracy comes from a three-term split
// x = x_hi + x_lo (x_hi = x truncated to tf32): A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// relative error about 2^-21 per product, so the residual the Newton iteration is refined
// against keeps float32 accuracy.
//
// One persistent CTA per SM (192 KB of shared memory): the weights are split and staged
// once in the canonical no-swizzle K-major layout; each tile stages its activations
// (h, then r o h, then h o r o (1 - r)) into the same layout and one thread issues the
// MMAs; the 16 warps read the accumulators with tcgen05.ld (warp w reads tensor-memory
// lanes 32 (w % 4) .. + 31 = tile rows, a quarter w / 4 of the columns) for the gates, the
// diagonal Jacobian and the residual; h and r stay in registers across the three stages. Every mbarrier wait is bounded; a wait that gives up sets the
// timeout flag and the kernel winds down, freeing its tensor memory.
#include "kernels.h"
#include "tc.cuh"

namespace deer {
namespace {

using namespace tc;

constexpr int kD = 64;        // state size = input size
constexpr int kTM = 128;      // rows per tile = MMA M
constexpr int kThreads = 512;  // 16 warps: lane quadrant w % 4, column quarter w / 4
constexpr int kCols = kD / 4;   // columns of each 64-wide block per thread
constexpr uint32_t kTmemCols = 256;  // D1: 128 columns, D2: 64, D3: 64
constexpr unsigned kWaitLimit = 1u << 24;

// Canonical no-swizzle K-major layout of an R x 64 float32 operand: core matrices of
// 8 rows x 16 bytes (4 elements) stored contiguously (128 B); core (r / 8, k / 4) at
// ((k / 4) (R / 8) + r / 8) 128 bytes. Leading-dimension byte offset (next core along K)
// R / 8 x 128, stride-dimension byte offset (next 8 rows) 128.
__host__ __device__ constexpr uint32_t core_off(int R, int r, int k) {
  return (uint32_t)(((k >> 2) * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

struct TcSmem {
  float B1h[128 * kD], B1l[128 * kD];  // [Uz; Ur]
  float B2h[kD * kD], B2l[kD * kD];    // Uh
  float B3h[kD * kD], B3l[kD * kD];    // M
  float Ah[kTM * kD], Al[kTM * kD];    // activations
};

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xffffe000u);
}

__device__ __forceinline__ void split_store4(float* hi, float* lo, uint32_t byte_off,
                                             float4 v) {
  const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
  *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(hi) + byte_off) = h;
  *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(lo) + byte_off) =
      make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  return tc::bar_wait(bar, parity, kWaitLimit);
}

// D (+)= A B^T over K = 64 with the three-term split: 8 K-steps of 8 (two core matrices)
__device__ __forceinline__ void gemm3(uint32_t dtmem, const float* Ah, const float* Al,
                                      const float* Bh, const float* Bl, int N) {
  const uint32_t idesc = idesc_tf32(N, kTM);
  const uint32_t lboA = (kTM / 8) * 128, lboB = (uint32_t)(N / 8) * 128, sbo = 128;
  const uint32_t ah = su32(Ah), al = su32(Al), bh = su32(Bh), bl = su32(Bl);
#pragma unroll
  for (int s = 0; s < kD / 8; ++s) {
    const uint32_t ao = (uint32_t)s * 2 * lboA, bo = (uint32_t)s * 2 * lboB;
    mma_tf32(dtmem, sdesc(ah + ao, lboA, sbo), sdesc(bh + bo, lboB, sbo), idesc, s > 0);
    mma_tf32(dtmem, sdesc(ah + ao, lboA, sbo), sdesc(bl + bo, lboB, sbo), idesc, 1u);
    mma_tf32(dtmem, sdesc(al + ao, lboA, sbo), sdesc(bh + bo, lboB, sbo), idesc, 1u);
  }
}

__device__ __forceinline__ float fsig(float v) { return 1.f / (1.f + __expf(-v)); }

__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_gru_lin_tc(GruTileArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smraw);
  __shared__ float diag_z[kD], diag_h[kD];
  __shared__ float rmx[kTM], rsq[kTM];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int qd = warp & 3, qc = warp >> 2;
  const int rl = 32 * qd + lane;  // tile row = tensor-memory lane
  const int c0 = kCols * qc;      // this thread's columns c0 .. c0 + kCols - 1 of each block
  const float* Uz = a.dv.params + 3 * kD * a.dv.d_in;
  const float* Ur = Uz + kD * kD;
  const float* Uh = Ur + kD * kD;
  // weights, split and staged once: row = output, K = input
  for (int e = tid; e < kD * (kD / 4); e += kThreads) {
    const int i = e / (kD / 4), k = 4 * (e % (kD / 4));
    split_store4(S.B1h, S.B1l, core_off(128, i, k), ldg4(Uz + i * kD + k));
    split_store4(S.B1h, S.B1l, core_off(128, kD + i, k), ldg4(Ur + i * kD + k));
    split_store4(S.B2h, S.B2l, core_off(kD, i, k), ldg4(Uh + i * kD + k));
    split_store4(S.B3h, S.B3l, core_off(kD, i, k), ldg4(a.dv.gru_M + i * kD + k));
  }
  if (tid < kD) {
    diag_z[tid] = Uz[tid * kD + tid];
    diag_h[tid] = Uh[tid * kD + tid];
  }
  const uint32_t bar = su32(&mbar);
  if (tid == 0) {
    s_ok = 1;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16);  // this warp's lanes, column 0
  uint32_t phase = 0, last = 0;
  const float kk = a.dparam;

  // make this thread's staged activations visible to the tensor core, let one thread
  // issue the products of a stage, and wait (bounded) for them
  auto run_stage = [&](int which) -> bool {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      if (which == 1) gemm3(tmem, S.Ah, S.Al, S.B1h, S.B1l, 128);
      else if (which == 2) gemm3(tmem + 128, S.Ah, S.Al, S.B2h, S.B2l, kD);
      else gemm3(tmem + 192, S.Ah, S.Al, S.B3h, S.B3l, kD);
      mma_commit(bar);
    }
    last = phase;
    const bool ok = bar_wait(bar, last);
    phase ^= 1u;
    fence_after();
    if (!ok) s_ok = 0;
    __syncthreads();
    return s_ok != 0;
  };

  const int64_t n_tiles = (a.bt.act_rows() + kTM - 1) / kTM;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int64_t ar = tile * kTM + rl;
    const bool v = ar < a.bt.act_rows();
    int64_t seq = 0, row = 0;
    if (v) act_row(a.bt, ar, seq, row);
    const float* hp = a.s0;
    const float* xp = a.xproj;
    if (v) {
      hp = row == __ldg(a.bt.offsets + seq) ? a.s0 + seq * kD : a.s + (row - 1) * kD;
      xp = a.xproj + row * (3 * kD);
    }
    if (qc == 0) { rmx[rl] = 0.f; rsq[rl] = 0.f; }
    // stage 1: h (kept in registers for the later stages)
    float h[kCols], xr[kCols];
#pragma unroll
    for (int j = 0; j < kCols; j += 4) {
      const float4 h4 = v ? ldg4(hp + c0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 x4 = v ? ldg4(xp + kD + c0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      h[j] = h4.x; h[j + 1] = h4.y; h[j + 2] = h4.z; h[j + 3] = h4.w;
      xr[j] = x4.x; xr[j + 1] = x4.y; xr[j + 2] = x4.z; xr[j + 3] = x4.w;
      split_store4(S.Ah, S.Al, core_off(kTM, rl, c0 + j), h4);
    }
    if (!(ok = run_stage(1))) break;
    // stage 2: r = sig(Wr x + Ur h) (kept), then r o h
    float r[kCols];
    {
      float rp[kCols];
      tmem_ld16(tl + kD + c0, rp);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < kCols; ++j) r[j] = fsig(rp[j] + xr[j]);
#pragma unroll
      for (int j = 0; j < kCols; j += 4)
        split_store4(S.Ah, S.Al, core_off(kTM, rl, c0 + j),
                     make_float4(r[j] * h[j], r[j + 1] * h[j + 1], r[j + 2] * h[j + 2],
                                 r[j + 3] * h[j + 3]));
    }
    // the epilogue's row inputs, loaded now so that they arrive while the products run
    float xz[kCols], xh[kCols], sc[kCols];
#pragma unroll
    for (int j = 0; j < kCols; j += 4) {
      float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f), b4 = a4, c4 = a4;
      if (v) {
        a4 = ldg4(xp + c0 + j);
        b4 = ldg4(xp + 2 * kD + c0 + j);
        c4 = *reinterpret_cast<const float4*>(a.s + row * kD + c0 + j);
      }
      xz[j] = a4.x; xz[j + 1] = a4.y; xz[j + 2] = a4.z; xz[j + 3] = a4.w;
      xh[j] = b4.x; xh[j + 1] = b4.y; xh[j + 2] = b4.z; xh[j + 3] = b4.w;
      sc[j] = c4.x; sc[j + 1] = c4.y; sc[j + 2] = c4.z; sc[j + 3] = c4.w;
    }
    if (!(ok = run_stage(2))) break;
    // stage 3: h o r o (1 - r)
#pragma unroll
    for (int j = 0; j < kCols; j += 4)
      split_store4(S.Ah, S.Al, core_off(kTM, rl, c0 + j),
                   make_float4(h[j] * r[j] * (1.f - r[j]), h[j + 1] * r[j + 1] * (1.f - r[j + 1]),
                               h[j + 2] * r[j + 2] * (1.f - r[j + 2]),
                               h[j + 3] * r[j + 3] * (1.f - r[j + 3])));
    if (!(ok = run_stage(3))) break;
    // gates, F, diagonal Jacobian, residual (two halves of 8 columns)
    float mx = 0.f, sq = 0.f;
#pragma unroll
    for (int hh = 0; hh < kCols; hh += 8) {
      float zp[8], hq[8], mc[8];
      tmem_ld8(tl + c0 + hh, zp);
      tmem_ld8(tl + 128 + c0 + hh, hq);
      tmem_ld8(tl + 192 + c0 + hh, mc);
      tmem_wait_ld();
      if (v) {
#pragma unroll
        for (int jj = 0; jj < 8; jj += 4) {
          const int j = hh + jj, k = c0 + j;
          float bo[4], ao[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int o = k + e;
            const float zi = fsig(zp[jj + e] + xz[j + e]);
            const float ri = r[j + e];
            const float ht = tanhf(hq[jj + e] + xh[j + e]);
            const float hv = h[j + e];
            const float F = (1.f - zi) * hv + zi * ht;
            float ai;
            if (a.jac == DEER_JAC_DIAG) {
              ai = (1.f - zi) + (ht - hv) * zi * (1.f - zi) * diag_z[o] +
                   zi * (1.f - ht * ht) * (diag_h[o] * ri + mc[jj + e]);
            } else {
              ai = a.jac == DEER_JAC_IDENTITY ? 1.f : 0.f;
            }
            if (a.damp == DEER_DAMP_SCALE) ai *= (1.f - kk);
            else if (a.damp == DEER_DAMP_CLIP) ai = fminf(fmaxf(ai, -kk), kk);
            ao[e] = ai;
            bo[e] = F - ai * hv;
            const float res = sc[j + e] - F;
            const float sa = fabsf(sc[j + e]);
            const float m = fabsf(res) / (sa > 1.f ? sa : 1.f);
            mx = (m > mx || m != m) ? m : mx;
            sq += res * res;
          }
          *reinterpret_cast<float4*>(a.b + row * kD + k) = make_float4(bo[0], bo[1], bo[2], bo[3]);
          if (a.jac == DEER_JAC_DIAG)
            *reinterpret_cast<float4*>(a.A + row * kD + k) =
                make_float4(ao[0], ao[1], ao[2], ao[3]);
        }
      }
    }
    if (v) {
      // non-negative floats order like their bit patterns
      atomicMax(reinterpret_cast<int*>(&rmx[rl]), __float_as_int(mx));
      atomicAdd(&rsq[rl], sq);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (qc == 0)
      acc_resid_f(a.acc, seq, v, rmx[rl], rsq[rl],
                  bad_key(!(rmx[rl] <= a.tol_f), row - (v ? __ldg(a.bt.offsets + seq) : 0)));
  }
  if (!ok) {
    if (tid == 0) atomicExch(&a.status->timeout, 1);
    // products may still be in flight: give them (bounded) time before tensor memory is
    // released
    bar_wait(bar, last);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

cudaError_t launch_gru_lin_tc(const GruTileArgs& a, cudaStream_t st) {
  if (a.bt.act_rows() == 0) return cudaSuccess;
  const int smem = (int)sizeof(TcSmem);
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(k_gru_lin_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (a.bt.act_rows() + kTM - 1) / kTM;
  const int64_t g = tiles < sms ? tiles : sms;
  k_gru_lin_tc<<<(unsigned)(g > 0 ? g : 1), kThreads, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace deer
