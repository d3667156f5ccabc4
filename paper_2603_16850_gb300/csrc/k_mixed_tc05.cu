// Mixed-precision chunk pass (d = 16, stored bf16 Jacobians E_t = A_t - I) on tcgen05:
// the chunk products of 8 chunks per CTA as one block-diagonal MMA chain.
//
// P_t = (I + E_t) P_{t-1} = P_{t-1} + E_t P_{t-1}. The accumulator D in tensor memory holds
// the 8 chunks' P stacked (128 lanes = 8 x 16 rows, 16 columns, float32); every row step
// adds blockdiag(E_t) x stacked(P_{t-1}) to it as 8 MMAs of M = 128, N = 16, K = 16
// (kind::f16, bf16 operands): K-step c multiplies an A tile that is zero except chunk c's
// 16 x 16 block E_t^(c) with rows 16c .. 16c + 15 of the B operand, chunk c's P_{t-1} in
// bf16. So 1/8 of the issued multiply-adds are useful: the independent 16 x 16 products of
// the chunks have nothing to share, and the smallest MMA with an accumulator in tensor
// memory is 128 rows tall. Each step reads D back (tcgen05.ld), rounds it to bf16 into the
// B operand in shared memory and issues the next MMAs; the vector part
// v <- v + E_t v + b_t of every chunk is formed on the side (thread (c, i): chunk c, row
// i). The mbarrier waits are bounded; a wait that gives up sets the timeout flag, waits
// (bounded) for the MMAs in flight and frees the tensor memory.
#include "kernels.h"
#include "tc.cuh"

namespace deer {
namespace {

constexpr int kT05Chunks = 8;            // chunks per CTA = K-steps per row step
constexpr int kT05Threads = 128;         // thread (c, i) = 16 c + i
constexpr uint32_t kT05TmemCols = 32;
constexpr unsigned kT05WaitLimit = 1u << 24;

struct T05Smem {
  // A tile of K-step c: 128 x 16 bf16, K-major no-swizzle cores (row-core stride 128 B,
  // K-core stride 2048 B); only rows 16c .. 16c + 15 are ever nonzero
  __nv_bfloat16 A[kT05Chunks][128 * 16];
  // B operand: K = 128 (stacked P rows) x N = 16, K-major (n-core stride 128 B, K-core
  // stride 256 B)
  __nv_bfloat16 B[128 * 16];
  float v[kT05Chunks][16];
  float b[kT05Chunks][16];
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

}  // namespace

__global__ void __launch_bounds__(kT05Threads, 1) k_mixed_chunk_tcgen05(MixedScanArgs a) {
  __shared__ __align__(1024) T05Smem S;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_sh;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c_loc = tid >> 4, i = tid & 15;  // this thread's chunk of the tile, and row
  // this thread's chunk (ragged: a tile may end early)
  const int64_t ac = blockIdx.x * (int64_t)kT05Chunks + c_loc;
  const bool has = ac < a.bt.act_chunks();
  int64_t seq = 0, c = 0, r0 = 0;
  int n = 0;
  if (has) act_chunk(a.bt, ac, seq, c, r0, n);
  // the longest chunk of the tile sets the row steps; shorter ones step with E = 0, b = 0
  __shared__ int s_n[kT05Chunks];
  if (i == 0) s_n[c_loc] = has ? n : 0;
  // zero the A tiles once (their off-diagonal blocks stay zero)
  for (int w = tid; w < (int)(sizeof(S.A) / 16); w += kT05Threads)
    reinterpret_cast<uint4*>(S.A)[w] = make_uint4(0u, 0u, 0u, 0u);
  S.v[c_loc][i] = 0.f;
  const uint32_t bar = tc::su32(&mbar);
  if (tid == 0) {
    s_ok = 1;
    tc::bar_init(bar, 1);
  }
  if (warp == 0) tc::tmem_alloc(tc::su32(&tmem_sh), kT05TmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's lanes
  int nmax = 0;
#pragma unroll
  for (int k = 0; k < kT05Chunks; ++k) nmax = s_n[k] > nmax ? s_n[k] : nmax;
  {
    // D = stacked identities: lane 16c + i holds row i of I
    float r[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) r[j] = j == (lane & 15) ? 1.f : 0.f;
    tmem_st16(tl, r);
  }
  const uint32_t adesc_lbo = 2048, bdesc_lbo = 256, sbo = 128;
  const uint32_t idesc = tc::idesc_bf16(16, 128);
  uint32_t phase = 0;
  bool ok = true;
  // byte offsets of this thread's E row in A tile c_loc: K-cores 0 (k 0..7) and 1 (8..15)
  const uint32_t a_off0 = tc::core_off_bytes(128, 16 * c_loc + i, 0);
  const uint32_t a_off1 = tc::core_off_bytes(128, 16 * c_loc + i, 16);
  for (int t = 0; t < nmax && ok; ++t) {
    const bool live = t < n;
    // E_t row i of this chunk (16 bf16 = two 16-byte pieces) and b_t[i]
    uint4 e_lo = make_uint4(0u, 0u, 0u, 0u), e_hi = e_lo;
    float bt = 0.f;
    if (live) {
      const uint4* Er = reinterpret_cast<const uint4*>(a.E + (r0 + t) * 256 + i * 16);
      e_lo = __ldg(Er);
      e_hi = __ldg(Er + 1);
      bt = __ldg(a.b + (r0 + t) * 16 + i);
    }
    unsigned char* At = reinterpret_cast<unsigned char*>(S.A[c_loc]);
    *reinterpret_cast<uint4*>(At + a_off0) = e_lo;
    *reinterpret_cast<uint4*>(At + a_off1) = e_hi;
    // read D = stacked P_{t-1}: lane k of the accumulator is row k of the stack
    float p[16];
    tc::tmem_ld16(tl, p);
    tc::tmem_wait_ld();
    // B[k][n] = P stacked, K-major: element (n, k) in n-core n / 8, K-core k / 8
    unsigned char* Bb = reinterpret_cast<unsigned char*>(S.B);
    const int k = tid;  // this thread's accumulator row = K index of the B operand
#pragma unroll
    for (int nn = 0; nn < 16; ++nn)
      *reinterpret_cast<__nv_bfloat16*>(Bb + ((k >> 3) * 2 + (nn >> 3)) * 128 + (nn & 7) * 16 +
                                        (k & 7) * 2) = __float2bfloat16_rn(p[nn]);
    // vector part: v <- v + E v + b (old v of the chunk read from shared memory)
    float ev = 0.f;
    {
      const uint32_t w[8] = {e_lo.x, e_lo.y, e_lo.z, e_lo.w, e_hi.x, e_hi.y, e_hi.z, e_hi.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        ev += __uint_as_float(w[q] << 16) * S.v[c_loc][2 * q] +
              __uint_as_float(w[q] & 0xffff0000u) * S.v[c_loc][2 * q + 1];
      }
    }
    const float vnew = S.v[c_loc][i] + ev + bt;
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();  // A, B complete; every read of the old v done
    tc::fence_after();
    S.v[c_loc][i] = vnew;
    if (tid == 0) {
#pragma unroll
      for (int kc = 0; kc < kT05Chunks; ++kc) {
        const uint64_t ad = tc::sdesc(tc::su32(S.A[kc]), adesc_lbo, sbo);
        const uint64_t bd = tc::sdesc(tc::su32(S.B) + 512u * kc, bdesc_lbo, sbo);
        tc::mma_f16(tmem, ad, bd, idesc, 1u);
      }
      tc::mma_commit(bar);
    }
    const bool got = tc::bar_wait(bar, phase, kT05WaitLimit);
    phase ^= 1u;
    tc::fence_after();
    if (!got) s_ok = 0;
    __syncthreads();
    ok = s_ok != 0;
  }
  if (ok) {
    float p[16];
    tc::tmem_ld16(tl, p);
    tc::tmem_wait_ld();
    if (has) {
      float* Po = a.aggP + c * 256;
#pragma unroll
      for (int j = 0; j < 16; ++j) Po[i * 16 + j] = p[j];
      a.aggv[c * 16 + i] = S.v[c_loc][i];
    }
  } else {
    if (tid == 0 && a.status) atomicExch(&a.status->timeout, 1);
    tc::bar_wait(bar, phase ^ 1u, kT05WaitLimit);  // the MMAs in flight, bounded
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, kT05TmemCols);
}

// enqueues the chunk pass; the caller counts the launch with the rest of its scan
cudaError_t launch_mixed_chunk_tcgen05(const MixedScanArgs& a, cudaStream_t st) {
  if (a.bt.act_chunks() == 0) return cudaSuccess;
  const unsigned g = grid_for(a.bt.act_chunks(), kT05Chunks);
  k_mixed_chunk_tcgen05<<<g, kT05Threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace deer
