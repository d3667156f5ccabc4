// Mixed-precision full-Jacobian iteration for mass-action kinetics with d = 16 / 32 (see
// MixedLinArgs / MixedScanArgs in kernels.h). The residual the Newton iteration is refined
// against, and the state, stay in float64; the Jacobian only steers the correction, so it
// is formed in float32 and stored (minus the identity) in bfloat16, halving its traffic.
#include "kernels.h"
#include "tc.cuh"

namespace deer {

template <int D>
__device__ __forceinline__ unsigned gmask_mixed() {
  return D == 32 ? 0xffffffffu : (0xffffu << (16 * ((threadIdx.x >> 4) & 1)));
}

// Species adjacency: for sequence b and species i, the reactions r that change species i
// and the change nu_{r,i} (reactants -1 each, products +1 each).
__global__ void k_ma_adjacency(int64_t n_seq, int d, int R, const int32_t* __restrict__ topo,
                               int64_t tstride, int32_t* __restrict__ adj_off,
                               int32_t* __restrict__ adj_e) {
  const int64_t seq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (seq >= n_seq) return;
  const int32_t* tt = topo + seq * tstride;
  int32_t* off = adj_off + seq * (d + 1);
  int32_t* e = adj_e + seq * (int64_t)(4 * R);
  int pos = 0;
  for (int i = 0; i < d; ++i) {
    off[i] = pos;
    for (int r = 0; r < R; ++r) {
      const int i1 = tt[4 * r], i2 = tt[4 * r + 1], p1 = tt[4 * r + 2], p2 = tt[4 * r + 3];
      const int nu = (i == p1) + (i == p2) - (i == i1) - (i == i2);
      if (nu != 0 && pos < 4 * R) e[pos++] = r | ((nu + 4) << 16);
    }
  }
  off[d] = pos;
}

cudaError_t launch_ma_adjacency(int64_t n_seq, int d, int R, const int32_t* topo,
                                int64_t tstride, int32_t* adj_off, int32_t* adj_e,
                                cudaStream_t st) {
  if (n_seq == 0) return cudaSuccess;
  k_ma_adjacency<<<grid_for(n_seq, 128), 128, 0, st>>>(n_seq, d, R, topo, tstride, adj_off,
                                                     adj_e);
  note_launch();
  return cudaGetLastError();
}

// Float32 value of a float64 by truncating its mantissa with integer operations (no FP64
// pipe, the scarce unit on this GPU). Used only where the float32 value steers the
// Jacobian, or for a float32 evaluation far from convergence, so rounding toward zero
// (relative error < 2^-23) is immaterial. Magnitudes below the float32 normal range give
// zero, above it the largest float32; NaN stays NaN.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7f7fffffu);
  return __uint_as_float(sign | ((unsigned)fe << 23) | m);
}

// Stoichiometric change nu in {-2, -1, 1, 2} as a float64 assembled from its bit pattern.
__device__ __forceinline__ double nu_f64(int nu) {
  const unsigned m = (unsigned)(nu < 0 ? -nu : nu);
  const unsigned hi = (nu < 0 ? 0x80000000u : 0u) | (m == 2u ? 0x40000000u : 0x3ff00000u);
  return __hiloint2double((int)hi, 0);
}

// Scaled residual above which a sequence's rows are evaluated in float32: the float32
// rounding error (~1e-7 relative) is then far below the residual being removed. A float32
// evaluation never reports less than kMixedFloor, so only float64 evaluations can pass the
// convergence test.
constexpr double kMixedFastAbove = 1e-4;
constexpr float kMixedFloor = 1e-6f;

// One row of the mixed linearisation with the dynamics' value path (stage states, reaction
// rates, slopes, F, residual) in V = float or double; the Jacobian path is float32 either
// way. Writes E and b for the row and returns its scaled residual and squared residual.
// A row of D floats from shared memory in 16-byte pieces (16-byte aligned).
template <int D>
__device__ __forceinline__ void ld_row4(const float* p, float (&v)[D]) {
#pragma unroll
  for (int j = 0; j < D; j += 4) {
    const float4 q = *reinterpret_cast<const float4*>(p + j);
    v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
  }
}

// The row's outputs go to Eo (its D x D block of E, row-major bf16) and bo (its entry
// of b = -r): in global memory for the materialised path, in shared memory for the
// recomputing one. sc is the row's own state s_t (read by the caller).
template <class V, int D, bool RK4, int RPL>
__device__ __forceinline__ void mixed_row(const MixedLinArgs& a, bool valid, int64_t row,
                                          int lane, unsigned gm, double s_prev_d, double sc,
                                          const int4 (&q)[RPL], const double (&kd)[RPL],
                                          const float (&kf)[RPL], int R, const int4* tt,
                                          const int32_t* ae, int e0, int e1,
                                          float (*sG)[D + 4], float (*sK)[D + 4], V* sRate,
                                          float* sD1, float* sD2, float& mx, float& sq,
                                          int64_t seq, unsigned long long& key,
                                          __nv_bfloat16* Eo, float* bo,
                                          float* Eo32 = nullptr) {
  constexpr bool F64 = sizeof(V) == 8;
  const V s_prev = F64 ? (V)s_prev_d : (V)d2f_trunc(s_prev_d);
  const V h = F64 ? (V)a.dv.dt : (V)a.dt_f;
  const float hf = a.dt_f;
  V c = s_prev, acc = V(0);
  float Kacc[D];
#pragma unroll
  for (int j = 0; j < D; ++j) Kacc[j] = 0.f;
  const int nst = RK4 ? 4 : 1;
  for (int stage = 0; stage < nst; ++stage) {
    // RK4 tableau: stage derivative weights (1, 2, 2, 1), stage offsets (h/2, h/2, h)
    const float cK = stage == 0 ? 0.f : (stage == 3 ? hf : 0.5f * hf);
    const V w = (stage == 1 || stage == 2) ? V(2) : V(1);
    const float cf = F64 ? d2f_trunc((double)c) : (float)c;
    // every reaction's rate once (reaction r on lane r mod d) and its two partials
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = k * D + lane;
      const int j2 = q[k].y < 0 ? 0 : q[k].y;
      const V c1 = __shfl_sync(gm, c, q[k].x, D);
      const V c2 = __shfl_sync(gm, c, j2, D);
      const float c1f = __shfl_sync(gm, cf, q[k].x, D);
      const float c2f = __shfl_sync(gm, cf, j2, D);
      if (r < R) {
        const bool bi = q[k].y >= 0;
        const V kr = F64 ? (V)kd[k] : (V)kf[k];
        sRate[r] = bi ? kr * c1 * c2 : kr * c1;
        sD1[r] = bi ? kf[k] * c2f : kf[k];
        sD2[r] = kf[k] * c1f;
      }
    }
#pragma unroll
    for (int j = 0; j < D; j += 4)
      *reinterpret_cast<float4*>(&sG[lane][j]) = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp(gm);
    // this species' slope and its row of the rate Jacobian, from its own reactions
    V g = V(0);
    for (int e = e0; e < e1; ++e) {
      const int code = __ldg(ae + e);
      const int r = code & 0xffff;
      const int nu = (code >> 16) - 4;
      g += (F64 ? (V)nu_f64(nu) : (V)nu) * sRate[r];
      const int4 qq = __ldg(tt + r);
      const float nuf = (float)nu;
      sG[lane][qq.x] += nuf * sD1[r];
      if (qq.y >= 0) sG[lane][qq.y] += nuf * sD2[r];
    }
    __syncwarp(gm);
    float Gi[D], Kn[D];
    ld_row4<D>(&sG[lane][0], Gi);
#pragma unroll
    for (int j = 0; j < D; ++j) Kn[j] = Gi[j];
    if (stage > 0) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        float km[D];
        ld_row4<D>(&sK[m][0], km);  // the same row for every lane of the group
        axpy_row<D>(cK * Gi[m], km, Kn);
      }
    }
    __syncwarp(gm);
    const float wf = (stage == 1 || stage == 2) ? 2.f : 1.f;
#pragma unroll
    for (int j = 0; j < D; j += 4)
      *reinterpret_cast<float4*>(&sK[lane][j]) = make_float4(Kn[j], Kn[j + 1], Kn[j + 2], Kn[j + 3]);
    axpy_row<D>(wf, Kn, Kacc);
    acc += w * g;
    const V cs = stage == 2 ? h : V(0.5) * h;
    c = s_prev + cs * g;
    __syncwarp(gm);
  }
  const V hw = RK4 ? h / V(6) : h;
  const V F = s_prev + hw * acc;
  if (valid) {
    const float scf = d2f_trunc(sc);
    float rf;
    if constexpr (F64) rf = d2f_trunc(sc - (double)F);
    else rf = scf - (float)F;
    const float sabs = fabsf(scf);
    float m = fabsf(rf) / (sabs > 1.f ? sabs : 1.f);
    if (!F64 && !(m != m)) m = m > kMixedFloor ? m : kMixedFloor;
    mx = nanmaxf(mx, m);
    sq += rf * rf;
    if (!(m <= a.tol_f) && key == 0ull) key = bad_key(true, row - __ldg(a.bt.offsets + seq));
    const float scale = a.scale_f;
    const float hwf = RK4 ? hf / 6.f : hf;
    // E = A - I with A = I + hw Kacc (scaled by (1 - k) under scale-ELK: E = s A - I):
    // bf16 row-major, or float32 with rows padded to 20 (the recomputing path)
    if (Eo32) {
      float* Er = Eo32 + lane * 20;
#pragma unroll
      for (int j = 0; j < D; j += 4)
        *reinterpret_cast<float4*>(Er + j) =
            make_float4(scale * hwf * Kacc[j] + (j == lane ? scale - 1.f : 0.f),
                        scale * hwf * Kacc[j + 1] + (j + 1 == lane ? scale - 1.f : 0.f),
                        scale * hwf * Kacc[j + 2] + (j + 2 == lane ? scale - 1.f : 0.f),
                        scale * hwf * Kacc[j + 3] + (j + 3 == lane ? scale - 1.f : 0.f));
    } else {
      Eo += lane * D;
#pragma unroll
      for (int j = 0; j < D; j += 2) {
        const float x0 = scale * hwf * Kacc[j] + (j == lane ? scale - 1.f : 0.f);
        const float x1 = scale * hwf * Kacc[j + 1] + (j + 1 == lane ? scale - 1.f : 0.f);
        *reinterpret_cast<__nv_bfloat162*>(Eo + j) = __floats2bfloat162_rn(x0, x1);
      }
    }
    bo[lane] = -rf;
  }
}

template <int D, bool RK4>
__global__ void __launch_bounds__(128) k_lin_ma_mixed(MixedLinArgs a) {
  constexpr int GROUPS = 128 / D;
  constexpr int RMAX = 64;         // reactions per network held in shared memory
  constexpr int RPL = RMAX / D;    // reactions per lane
  // rows padded to D + 4 floats: 16-byte row accesses of eight lanes fall in distinct
  // banks; one padding row per group of sK: the two groups of a warp read their (common)
  // K rows from banks 20 apart (same-bank reads of different groups would serialise)
  __shared__ __align__(16) float sG[GROUPS][D][D + 4];
  __shared__ __align__(16) float sK[GROUPS][D + 1][D + 4];
  __shared__ double sRate[GROUPS][RMAX];  // float rates use the first half in float32 mode
  __shared__ float sD1[GROUPS][RMAX], sD2[GROUPS][RMAX];  // d rate / d c_i1, d c_i2
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = gmask_mixed<D>();
  const int64_t ar = blockIdx.x * (int64_t)GROUPS + grp;
  const bool valid = ar < a.bt.act_rows();
  int64_t seq = 0, row = 0;
  if (valid) act_row(a.bt, ar, seq, row);
  const double s_prev = valid ? (row == __ldg(a.bt.offsets + seq) ? a.s0[seq * D + lane]
                                                                : a.s[(row - 1) * D + lane])
                              : 0.0;
  const double* kk = a.dv.params + seq * a.dv.pstride;
  const int4* tt = reinterpret_cast<const int4*>(a.dv.topo + seq * a.dv.tstride);
  const int32_t* aoff = a.adj_off + (a.adj_stride ? seq : 0) * (D + 1);
  const int32_t* ae = a.adj_e + (a.adj_stride ? seq : 0) * a.adj_stride;
  const int e0 = __ldg(aoff + lane), e1 = __ldg(aoff + lane + 1);
  const int R = a.dv.R < RMAX ? a.dv.R : RMAX;
  int4 q[RPL];
  double kd[RPL];
  float kf[RPL];
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int r = k * D + lane;
    q[k] = __ldg(tt + (r < R ? r : 0));
    kd[k] = r < R ? __ldg(kk + r) : 0.0;
    kf[k] = d2f_trunc(kd[k]);
  }
  const bool fast = !valid || a.it == 0 || a.info[seq].max_resid > kMixedFastAbove;
  float mx = 0.f, sq = 0.f;
  unsigned long long key = 0ull;  // first failing row (sliding window)
  const double sc = valid ? a.s[row * D + lane] : 0.0;
  __nv_bfloat16* Eo = a.E + (valid ? row : 0) * (int64_t)(D * D);
  float* bo = a.b + (valid ? row : 0) * D;
  if (fast)
    mixed_row<float, D, RK4, RPL>(a, valid, row, lane, gm, s_prev, sc, q, kd, kf, R, tt, ae,
                                  e0, e1, sG[grp], sK[grp],
                                  reinterpret_cast<float*>(sRate[grp]), sD1[grp], sD2[grp],
                                  mx, sq, seq, key, Eo, bo);
  else
    mixed_row<double, D, RK4, RPL>(a, valid, row, lane, gm, s_prev, sc, q, kd, kf, R, tt, ae,
                                   e0, e1, sG[grp], sK[grp], sRate[grp], sD1[grp], sD2[grp],
                                   mx, sq, seq, key, Eo, bo);
  acc_resid_f(a.acc, seq, valid, mx, sq, key);
}

// ---- mixed dense scan: lane j owns column j of P and entry j of the vectors ----------
template <int D>
__global__ void __launch_bounds__(128) k_mixed_chunk(MixedScanArgs a) {
  constexpr int G = 128 / D;
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = gmask_mixed<D>();
  const int64_t ac = blockIdx.x * (int64_t)G + grp;
  const bool valid = ac < a.bt.act_chunks();
  int64_t seq = 0, c = 0, r0 = 0;
  int n = 0;
  if (valid) act_chunk(a.bt, ac, seq, c, r0, n);
  const bool need_P = valid && c != win_first(a.bt, seq);
  float Pc[D];
  float v = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) Pc[i] = i == lane ? 1.f : 0.f;
  for (int t = 0; t < n; ++t) {
    const __nv_bfloat16* Et = a.E + (r0 + t) * (int64_t)(D * D);
    float nv = __ldg(a.b + (r0 + t) * D + lane) + v;
#pragma unroll
    for (int k = 0; k < D; ++k)
      nv += __bfloat162float(Et[lane * D + k]) * __shfl_sync(gm, v, k, D);
    v = nv;
    if (need_P) {
      float np[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        float x = Pc[i];
#pragma unroll
        for (int k = 0; k < D; ++k) x += __bfloat162float(Et[i * D + k]) * Pc[k];
        np[i] = x;
      }
#pragma unroll
      for (int i = 0; i < D; ++i) Pc[i] = np[i];
    }
  }
  if (valid) {
    float* Po = a.aggP + c * (int64_t)(D * D);
#pragma unroll
    for (int i = 0; i < D; ++i) Po[i * D + lane] = Pc[i];
    a.aggv[c * D + lane] = v;
  }
}

template <int D>
__global__ void __launch_bounds__(128) k_mixed_carry(MixedScanArgs a) {
  constexpr int G = 128 / D;
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = gmask_mixed<D>();
  const int64_t kq = blockIdx.x * (int64_t)G + grp;
  const bool valid = kq < a.bt.n_act();
  const int64_t seq = valid ? a.bt.act_seq[kq] : 0;
  const int64_t c0 = valid ? win_first(a.bt, seq) : 0;
  const int64_t c1 = valid ? a.bt.chunk_first[seq + 1] : 0;
  float x = 0.f;
  for (int64_t c = c0; c < c1; ++c) {
    a.cin[c * D + lane] = x;
    const float* P = a.aggP + c * (int64_t)(D * D);
    float y = a.aggv[c * D + lane];
    if (c > c0) {
#pragma unroll
      for (int k = 0; k < D; ++k) y += P[lane * D + k] * __shfl_sync(gm, x, k, D);
    }
    x = y;
  }
}

template <int D>
__global__ void __launch_bounds__(128) k_mixed_apply(MixedScanArgs a) {
  constexpr int G = 128 / D;
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = gmask_mixed<D>();
  const int64_t ac = blockIdx.x * (int64_t)G + grp;
  const bool valid = ac < a.bt.act_chunks();
  int64_t seq = 0, c = 0, r0 = 0;
  int n = 0;
  if (valid) act_chunk(a.bt, ac, seq, c, r0, n);
  float x = valid ? a.cin[c * D + lane] : 0.f;
  for (int t = 0; t < n; ++t) {
    const int64_t row = r0 + t;
    const __nv_bfloat16* Et = a.E + row * (int64_t)(D * D) + lane * D;
    float y = __ldg(a.b + row * D + lane) + x;
#pragma unroll
    for (int k = 0; k < D; ++k) y += __bfloat162float(Et[k]) * __shfl_sync(gm, x, k, D);
    x = y;
    double* sp = a.s + row * D + lane;
    double nsv = *sp + (double)y;
    if (a.reset && !(nsv <= a.reset_thr && nsv >= -a.reset_thr)) nsv = 0.0;
    *sp = nsv;
  }
}

// ---- d = 16 on the tensor cores: one warp per chunk --------------------------------
// The chunk aggregate P <- (I + E_t) P is carried transposed, P^T <- P^T + P^T E_t^T, as
// one warp-level bf16 MMA pair (m16n8k16, float32 accumulate) per row: the float32
// accumulator fragment of P^T is exactly the A-operand fragment of the next product once
// rounded to bf16, and the B operand E_t^T is read straight from the row-major bf16 E_t
// (lane (g, t) of the warp, g = lane / 4, t = lane % 4, holds E[g][2t..2t+1],
// E[g][2t+8..2t+9] for columns 0-7 and the same entries of row g + 8 for columns 8-15).
// The vector part v <- v + E_t v + b_t stays in float32 on the same fragments: lane (g, t)
// forms the partial dot products of rows g and g + 8 over its four columns, a two-step
// shuffle sums the four lanes of row g, and each lane then fetches the four entries
// (2t, 2t+1, 2t+8, 2t+9) it needs for the next row.
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One row of the vector recurrence x <- x + E x + b on the fragments described above.
// lo / hi: x[g], x[g + 8] (same in the four lanes of row g); q[0..3]: x[2t], x[2t+1],
// x[2t+8], x[2t+9]. e0..e3: the lane's four words of E (rows g and g + 8).
__device__ __forceinline__ void frag_matvec16(uint32_t e0, uint32_t e1, uint32_t e2,
                                              uint32_t e3, float b_lo, float b_hi, float& lo,
                                              float& hi, float (&q)[4], int t) {
  float pl = bf_lo(e0) * q[0] + bf_hi(e0) * q[1] + bf_lo(e1) * q[2] + bf_hi(e1) * q[3];
  float ph = bf_lo(e2) * q[0] + bf_hi(e2) * q[1] + bf_lo(e3) * q[2] + bf_hi(e3) * q[3];
  pl += __shfl_xor_sync(0xffffffffu, pl, 1);
  ph += __shfl_xor_sync(0xffffffffu, ph, 1);
  pl += __shfl_xor_sync(0xffffffffu, pl, 2);
  ph += __shfl_xor_sync(0xffffffffu, ph, 2);
  lo = lo + pl + b_lo;
  hi = hi + ph + b_hi;
  q[0] = __shfl_sync(0xffffffffu, lo, 8 * t);
  q[1] = __shfl_sync(0xffffffffu, lo, 8 * t + 4);
  q[2] = __shfl_sync(0xffffffffu, hi, 8 * t);
  q[3] = __shfl_sync(0xffffffffu, hi, 8 * t + 4);
}

__global__ void __launch_bounds__(128) k_mixed_chunk_tc16(MixedScanArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t ac = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (ac >= a.bt.act_chunks()) return;  // whole warps
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const bool need_P = c != win_first(a.bt, seq);
  // P^T = I: fragment entries (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1) of the two tiles
  float p0[4] = {g == 2 * t ? 1.f : 0.f, g == 2 * t + 1 ? 1.f : 0.f, 0.f, 0.f};
  float p1[4] = {0.f, 0.f, g == 2 * t ? 1.f : 0.f, g == 2 * t + 1 ? 1.f : 0.f};
  float lo = 0.f, hi = 0.f, q[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < n; ++k) {
    const int64_t row = r0 + k;
    const uint32_t* Ew = reinterpret_cast<const uint32_t*>(a.E + row * 256);
    const uint32_t e0 = __ldg(Ew + g * 8 + t), e1 = __ldg(Ew + g * 8 + t + 4);
    const uint32_t e2 = __ldg(Ew + (g + 8) * 8 + t), e3 = __ldg(Ew + (g + 8) * 8 + t + 4);
    const float b_lo = __ldg(a.b + row * 16 + g), b_hi = __ldg(a.b + row * 16 + g + 8);
    if (need_P) {
      const uint32_t A[4] = {pack_bf16x2(p0[0], p0[1]), pack_bf16x2(p0[2], p0[3]),
                             pack_bf16x2(p1[0], p1[1]), pack_bf16x2(p1[2], p1[3])};
      mma_bf16_16816(p0, A, e0, e1);
      mma_bf16_16816(p1, A, e2, e3);
    }
    frag_matvec16(e0, e1, e2, e3, b_lo, b_hi, lo, hi, q, t);
  }
  // P[i][j] = P^T[j][i]: tile 0 holds P^T[g][2t], P^T[g][2t+1], P^T[g+8][2t], P^T[g+8][2t+1]
  float* Po = a.aggP + c * 256;
  Po[(2 * t) * 16 + g] = p0[0];
  Po[(2 * t + 1) * 16 + g] = p0[1];
  Po[(2 * t) * 16 + g + 8] = p0[2];
  Po[(2 * t + 1) * 16 + g + 8] = p0[3];
  Po[(2 * t + 8) * 16 + g] = p1[0];
  Po[(2 * t + 9) * 16 + g] = p1[1];
  Po[(2 * t + 8) * 16 + g + 8] = p1[2];
  Po[(2 * t + 9) * 16 + g + 8] = p1[3];
  if (t == 0) {
    a.aggv[c * 16 + g] = lo;
    a.aggv[c * 16 + g + 8] = hi;
  }
}

// |x| >= 2^60 (about 1.15e18), Inf or NaN, from the exponent bits (no FP64 pipe)
__device__ __forceinline__ bool overflowed(double x) {
  return ((((unsigned)__double2hiint(x)) >> 20) & 0x7ffu) >= 1023u + 60u;
}

__global__ void __launch_bounds__(128) k_mixed_apply_tc16(MixedScanArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t ac = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (ac >= a.bt.act_chunks()) return;  // whole warps
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const float* ci = a.cin + c * 16;
  float lo = ci[g], hi = ci[g + 8];
  float q[4] = {ci[2 * t], ci[2 * t + 1], ci[2 * t + 8], ci[2 * t + 9]};
  for (int k = 0; k < n; ++k) {
    const int64_t row = r0 + k;
    const uint32_t* Ew = reinterpret_cast<const uint32_t*>(a.E + row * 256);
    const uint32_t e0 = __ldg(Ew + g * 8 + t), e1 = __ldg(Ew + g * 8 + t + 4);
    const uint32_t e2 = __ldg(Ew + (g + 8) * 8 + t), e3 = __ldg(Ew + (g + 8) * 8 + t + 4);
    const float b_lo = __ldg(a.b + row * 16 + g), b_hi = __ldg(a.b + row * 16 + g + 8);
    frag_matvec16(e0, e1, e2, e3, b_lo, b_hi, lo, hi, q, t);
    // s += Delta in float64; lanes t = 0 (row g) and t = 1 (row g + 8) write
    if (t < 2) {
      double* sp = a.s + row * 16 + g + 8 * t;
      double v = *sp + (double)(t == 0 ? lo : hi);
      if (a.reset && overflowed(v)) v = 0.0;
      *sp = v;
    }
  }
}

// ---- d = 16 without stored Jacobians: one warp per chunk ----------------------------
// The two half-warps linearise rows t and t + 1 of the chunk (16 lanes per row, as in
// k_lin_ma_mixed) into shared memory; the whole warp then folds them into the chunk
// aggregate (pass 1) or applies the correction to them (pass 2). The Jacobians never go to
// HBM here, so they are kept in float32 and the chunk product is formed to float32
// accuracy: P^T <- P^T + P^T E_t^T as warp-level tf32 MMAs (m16n8k8) with the three-term
// split x = x_hi + x_lo, the accumulator of P^T re-laid into the next A operand by quad
// shuffles (as in k_dense_chunk_mma32). Over horizons of 1e5 steps the rounding of E_t
// to bf16 compounds in the chunk products and slows Newton's convergence to linear on
// the stiffer networks; float32 Jacobians keep it fast. The vector part
// v <- v + E_t v + b_t: lane l forms half a row (row l mod 16, columns 8 (l / 16) ..) and
// the two halves meet by a shuffle.
constexpr int kRcWarps = 4;
constexpr int kRcRmax = 64;
constexpr int kRcES = 20;  // float32 E rows padded: the fragment reads hit distinct banks

struct RcSmem {
  float G[2][16][20];
  float K[2][17][20];
  double rate[2][kRcRmax];
  float d1[2][kRcRmax], d2[2][kRcRmax];
  float E[2][16 * kRcES];
  float b[2][16];
  double old[16];  // pass 2: old state of the previous pair's second row
};

// per-lane network data of the sequence (reactions r = k * 16 + lane)
struct RcNet {
  int4 q[kRcRmax / 16];
  double kd[kRcRmax / 16];
  float kf[kRcRmax / 16];
  const int4* tt;
  const int32_t* ae;
  int e0, e1, R;
};

__device__ __forceinline__ void rc_net(const MixedLinArgs& a, int64_t seq, int lane,
                                       RcNet& n) {
  const double* kk = a.dv.params + seq * a.dv.pstride;
  n.tt = reinterpret_cast<const int4*>(a.dv.topo + seq * a.dv.tstride);
  const int32_t* aoff = a.adj_off + (a.adj_stride ? seq : 0) * 17;
  n.ae = a.adj_e + (a.adj_stride ? seq : 0) * a.adj_stride;
  n.e0 = __ldg(aoff + lane);
  n.e1 = __ldg(aoff + lane + 1);
  n.R = a.dv.R < kRcRmax ? a.dv.R : kRcRmax;
#pragma unroll
  for (int k = 0; k < kRcRmax / 16; ++k) {
    const int r = k * 16 + lane;
    n.q[k] = __ldg(n.tt + (r < n.R ? r : 0));
    n.kd[k] = r < n.R ? __ldg(kk + r) : 0.0;
    n.kf[k] = d2f_trunc(n.kd[k]);
  }
}

// linearise one row into the half-warp's shared buffers (float32 E, b): value path per
// `fast`
template <bool RK4>
__device__ __forceinline__ void rc_row(const MixedLinArgs& a, bool fast, bool valid,
                                       int64_t row, int half, int lane, unsigned gm,
                                       double sp, double sc, const RcNet& n, RcSmem& S,
                                       float& mx, float& sq, int64_t seq,
                                       unsigned long long& key) {
  if (fast)
    mixed_row<float, 16, RK4, kRcRmax / 16>(
        a, valid, row, lane, gm, sp, sc, n.q, n.kd, n.kf, n.R, n.tt, n.ae, n.e0, n.e1,
        S.G[half], S.K[half], reinterpret_cast<float*>(S.rate[half]), S.d1[half],
        S.d2[half], mx, sq, seq, key, nullptr, S.b[half], S.E[half]);
  else
    mixed_row<double, 16, RK4, kRcRmax / 16>(
        a, valid, row, lane, gm, sp, sc, n.q, n.kd, n.kf, n.R, n.tt, n.ae, n.e0, n.e1,
        S.G[half], S.K[half], S.rate[half], S.d1[half], S.d2[half], mx, sq, seq, key,
        nullptr, S.b[half], S.E[half]);
}

// P^T <- P^T + P^T E^T for the warp's 16 x 16 accumulator acc[n-tile][4] (lane (g, t):
// rows g, g + 8, columns 8 j + 2 t, + 1), three-term tf32 split
__device__ __forceinline__ void rc_compose(float (&acc)[2][4], const float* E, int g, int t,
                                           int lane) {
  const int qsrc = (lane & ~3) + (t >> 1);
  const bool odd = t & 1;
  uint32_t ah[2][4], al[2][4];
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const float x0 = __shfl_sync(0xffffffffu, acc[kk][0], qsrc);
    const float x1 = __shfl_sync(0xffffffffu, acc[kk][1], qsrc);
    const float x2 = __shfl_sync(0xffffffffu, acc[kk][2], qsrc);
    const float x3 = __shfl_sync(0xffffffffu, acc[kk][3], qsrc);
    const float y0 = __shfl_sync(0xffffffffu, acc[kk][0], qsrc + 2);
    const float y1 = __shfl_sync(0xffffffffu, acc[kk][1], qsrc + 2);
    const float y2 = __shfl_sync(0xffffffffu, acc[kk][2], qsrc + 2);
    const float y3 = __shfl_sync(0xffffffffu, acc[kk][3], qsrc + 2);
    const float av[4] = {odd ? x1 : x0, odd ? x3 : x2, odd ? y1 : y0, odd ? y3 : y2};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ah[kk][e] = tc::tf32_rna(av[e]);
      al[kk][e] = tc::tf32_rna(av[e] - __uint_as_float(ah[kk][e]));
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      // B[k][n] = E^T[k][n] = E[n][k]: n = 8 j + g, k = 8 kk + t (+ 4)
      const float bx0 = E[(8 * j + g) * kRcES + 8 * kk + t];
      const float bx1 = E[(8 * j + g) * kRcES + 8 * kk + t + 4];
      const uint32_t bh0 = tc::tf32_rna(bx0), bh1 = tc::tf32_rna(bx1);
      const uint32_t bl0 = tc::tf32_rna(bx0 - __uint_as_float(bh0));
      const uint32_t bl1 = tc::tf32_rna(bx1 - __uint_as_float(bh1));
      tc::mma_1688_tf32(acc[j], al[kk], bh0, bh1);
      tc::mma_1688_tf32(acc[j], ah[kk], bl0, bl1);
      tc::mma_1688_tf32(acc[j], ah[kk], bh0, bh1);
    }
  }
}

// v <- v + E v + b with lane l holding v[l mod 16]; returns the new v[l mod 16]
__device__ __forceinline__ float rc_matvec(float v, const float* E, const float* b,
                                           int lane) {
  const int i = lane & 15, c = lane >> 4;
  float part = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    part += E[i * kRcES + 8 * c + k] * __shfl_sync(0xffffffffu, v, 8 * c + k);
  part += __shfl_xor_sync(0xffffffffu, part, 16);
  return v + part + b[i];
}

template <bool RK4>
__global__ void __launch_bounds__(32 * kRcWarps) k_mixed_lin_agg16(MixedRcArgs r) {
  __shared__ __align__(16) RcSmem smem[kRcWarps];
  const MixedLinArgs& a = r.lin;
  const int warp = threadIdx.x >> 5, l32 = threadIdx.x & 31;
  const int half = l32 >> 4, lane = l32 & 15, g = l32 >> 2, tq = l32 & 3;
  const unsigned gm = gmask_mixed<16>();
  const int64_t ac = blockIdx.x * (int64_t)kRcWarps + warp;
  if (ac >= a.bt.act_chunks()) return;  // whole warps
  RcSmem& S = smem[warp];
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const int64_t base = __ldg(a.bt.offsets + seq);
  RcNet net;
  rc_net(a, seq, lane, net);
  const bool fast = a.it == 0 || a.info[seq].max_resid > kMixedFastAbove;
  if (l32 == 0) r.fastsel[seq] = fast ? 1 : 0;  // the same value from every chunk
  // the old state before the chunk, kept for the second pass (whose neighbouring chunk may
  // already have updated it)
  const double prev0 = r0 == base ? a.s0[seq * 16 + lane] : a.s[(r0 - 1) * 16 + lane];
  if (half == 0 && r0 > base) r.sbound[c * 16 + lane] = prev0;
  const bool need_P = c != win_first(a.bt, seq);
  // P^T = I
  float acc[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int n0 = 8 * j + 2 * tq;
    acc[j][0] = g == n0 ? 1.f : 0.f;
    acc[j][1] = g == n0 + 1 ? 1.f : 0.f;
    acc[j][2] = g + 8 == n0 ? 1.f : 0.f;
    acc[j][3] = g + 8 == n0 + 1 ? 1.f : 0.f;
  }
  float v = 0.f;
  float mx = 0.f, sq = 0.f;
  unsigned long long key = 0ull;
  for (int t = 0; t < n; t += 2) {
    const int tr = t + half;
    const bool vld = tr < n;
    const int64_t row = r0 + (vld ? tr : 0);
    const double sp = tr == 0 ? prev0 : (vld ? a.s[(row - 1) * 16 + lane] : prev0);
    const double sc = vld ? a.s[row * 16 + lane] : prev0;
    rc_row<RK4>(a, fast, vld, row, half, lane, gm, sp, sc, net, S, mx, sq, seq, key);
    __syncwarp();
    for (int h = 0; h < 2 && t + h < n; ++h) {
      if (need_P) rc_compose(acc, S.E[h], g, tq, l32);
      v = rc_matvec(v, S.E[h], S.b[h], l32);
    }
    __syncwarp();
  }
  // P[i][j] = P^T[j][i]
  float* Po = r.aggP + c * 256;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int n0 = 8 * j + 2 * tq;
    Po[n0 * 16 + g] = acc[j][0];
    Po[(n0 + 1) * 16 + g] = acc[j][1];
    Po[n0 * 16 + g + 8] = acc[j][2];
    Po[(n0 + 1) * 16 + g + 8] = acc[j][3];
  }
  if (half == 0) r.aggv[c * 16 + lane] = v;
  acc_resid_f(a.acc, seq, true, mx, sq, key);
}

template <bool RK4>
__global__ void __launch_bounds__(32 * kRcWarps) k_mixed_apply_rc16(MixedRcArgs r) {
  __shared__ __align__(16) RcSmem smem[kRcWarps];
  const MixedLinArgs& a = r.lin;
  const int warp = threadIdx.x >> 5, l32 = threadIdx.x & 31;
  const int half = l32 >> 4, lane = l32 & 15;
  const unsigned gm = gmask_mixed<16>();
  const int64_t ac = blockIdx.x * (int64_t)kRcWarps + warp;
  if (ac >= a.bt.act_chunks()) return;  // whole warps
  RcSmem& S = smem[warp];
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const int64_t base = __ldg(a.bt.offsets + seq);
  RcNet net;
  rc_net(a, seq, lane, net);
  const bool fast = r.fastsel[seq] != 0;
  const double prev0 = r0 == base ? a.s0[seq * 16 + lane] : r.sbound[c * 16 + lane];
  float x = r.cin[c * 16 + lane];  // Delta entering the chunk, entry lane mod 16
  float mx = 0.f, sq = 0.f;  // recomputed statistics, not reported again
  unsigned long long key = 0ull;
  double* s = const_cast<double*>(a.s);
  for (int t = 0; t < n; t += 2) {
    const int tr = t + half;
    const bool vld = tr < n;
    const int64_t row = r0 + (vld ? tr : 0);
    // old s_{t-1}: the chunk's saved boundary, the previous pair's second row (saved
    // before it was updated), or row t of this pair (not updated yet)
    double sp = prev0;
    if (tr > 0) sp = half == 0 ? S.old[lane] : (vld ? s[(row - 1) * 16 + lane] : prev0);
    const double sc = vld ? s[row * 16 + lane] : prev0;
    rc_row<RK4>(a, fast, vld, row, half, lane, gm, sp, sc, net, S, mx, sq, seq, key);
    __syncwarp();
    if (half == 1 && vld) S.old[lane] = sc;
    __syncwarp();
    for (int h = 0; h < 2 && t + h < n; ++h) {
      x = rc_matvec(x, S.E[h], S.b[h], l32);
      if (half == 0) {
        double* sp2 = s + (r0 + t + h) * 16 + lane;
        double nv = *sp2 + (double)x;
        if (r.reset && overflowed(nv)) nv = 0.0;
        *sp2 = nv;
      }
    }
    __syncwarp();
  }
}

cudaError_t launch_mixed_lin_agg(const MixedRcArgs& a, cudaStream_t st) {
  if (a.lin.bt.act_chunks() == 0) return cudaSuccess;
  if (a.lin.dv.d != 16) return cudaErrorInvalidValue;
  const unsigned g = grid_for(a.lin.bt.act_chunks(), kRcWarps);
  if (a.lin.dv.kind == DEER_F_MASSACTION_RK4) k_mixed_lin_agg16<true><<<g, 32 * kRcWarps, 0, st>>>(a);
  else k_mixed_lin_agg16<false><<<g, 32 * kRcWarps, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mixed_apply_rc(const MixedRcArgs& a, const MixedScanArgs& carry,
                                  cudaStream_t st) {
  if (a.lin.bt.act_chunks() == 0) return cudaSuccess;
  if (a.lin.dv.d != 16) return cudaErrorInvalidValue;
  k_mixed_carry<16><<<grid_for(carry.bt.n_act(), 128 / 16), 128, 0, st>>>(carry);
  const unsigned g = grid_for(a.lin.bt.act_chunks(), kRcWarps);
  if (a.lin.dv.kind == DEER_F_MASSACTION_RK4) k_mixed_apply_rc16<true><<<g, 32 * kRcWarps, 0, st>>>(a);
  else k_mixed_apply_rc16<false><<<g, 32 * kRcWarps, 0, st>>>(a);
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_lin_ma_mixed(const MixedLinArgs& a, cudaStream_t st) {
  if (a.bt.act_rows() == 0) return cudaSuccess;
  const bool rk4 = a.dv.kind == DEER_F_MASSACTION_RK4;
  const int d = a.dv.d;
  const unsigned g = grid_for(a.bt.act_rows(), 128 / d);
  if (d == 16) {
    if (rk4) k_lin_ma_mixed<16, true><<<g, 128, 0, st>>>(a);
    else k_lin_ma_mixed<16, false><<<g, 128, 0, st>>>(a);
  } else if (d == 32) {
    if (rk4) k_lin_ma_mixed<32, true><<<g, 128, 0, st>>>(a);
    else k_lin_ma_mixed<32, false><<<g, 128, 0, st>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <int D>
static void mixed_launch(const MixedScanArgs& a, cudaStream_t st) {
  constexpr int G = 128 / D;
  const unsigned gs = grid_for(a.bt.n_act(), G);
  if constexpr (D == 16) {
    const unsigned gw = grid_for(a.bt.act_chunks(), 4);  // one warp per chunk
    if (a.tc_mode == 2) {
      if (launch_mixed_chunk_tcgen05(a, st) != cudaSuccess) return;
    } else {
      k_mixed_chunk_tc16<<<gw, 128, 0, st>>>(a);
    }
    k_mixed_carry<D><<<gs, 128, 0, st>>>(a);
    k_mixed_apply_tc16<<<gw, 128, 0, st>>>(a);
  } else {
    const unsigned gc = grid_for(a.bt.act_chunks(), G);
    k_mixed_chunk<D><<<gc, 128, 0, st>>>(a);
    k_mixed_carry<D><<<gs, 128, 0, st>>>(a);
    k_mixed_apply<D><<<gc, 128, 0, st>>>(a);
  }
  note_launch(3);
}

cudaError_t launch_dense_scan_mixed(const MixedScanArgs& a, cudaStream_t st) {
  if (a.bt.act_rows() == 0) return cudaSuccess;
  if (a.d == 16) mixed_launch<16>(a, st);
  else if (a.d == 32) mixed_launch<32>(a, st);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace deer
