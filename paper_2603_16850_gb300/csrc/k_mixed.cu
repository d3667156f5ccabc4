// Mixed-precision full-Jacobian iteration for mass-action kinetics with d = 16 / 32 (see
// MixedLinArgs / MixedScanArgs in kernels.h). The residual the Newton iteration is refined
// against, and the state, stay in float64; the Jacobian only steers the correction, so it
// is formed in float32 and stored (minus the identity) in bfloat16, halving its traffic.
#include "kernels.h"

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

template <int D, bool RK4>
__global__ void __launch_bounds__(128) k_lin_ma_mixed(MixedLinArgs a) {
  constexpr int GROUPS = 128 / D;
  constexpr int RMAX = 64;  // reactions per network held in shared memory
  __shared__ float sG[GROUPS][D][D + 1];
  __shared__ float sK[GROUPS][D][D];
  __shared__ double sRate[GROUPS][RMAX];
  __shared__ float sD1[GROUPS][RMAX], sD2[GROUPS][RMAX];  // d rate / d c_i1, d c_i2 (no k)
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = gmask_mixed<D>();
  const int64_t ar = blockIdx.x * (int64_t)GROUPS + grp;
  const bool valid = ar < a.bt.act_rows;
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
  const double h = a.dv.dt;
  double c = s_prev, acc = 0.0;
  float Kacc[D];
#pragma unroll
  for (int j = 0; j < D; ++j) Kacc[j] = 0.f;
  const int nst = RK4 ? 4 : 1;
  for (int stage = 0; stage < nst; ++stage) {
    const float cK = stage == 0 ? 0.f : (stage == 3 ? (float)h : 0.5f * (float)h);
    const double w = (stage == 1 || stage == 2) ? 2.0 : 1.0;
    // every reaction's rate once (lane r % D), in float64, and its two partial derivatives
    for (int r0 = 0; r0 < R; r0 += D) {
      const int r = r0 + lane;
      const int4 q = __ldg(tt + (r < R ? r : 0));
      const double c1 = __shfl_sync(gm, c, q.x, D);
      const double c2 = __shfl_sync(gm, c, q.y < 0 ? 0 : q.y, D);
      if (r < R) {
        const double kr = __ldg(kk + r);
        const double f2 = q.y < 0 ? 1.0 : c2;
        sRate[grp][r] = kr * c1 * f2;
        sD1[grp][r] = (float)(kr * f2);
        sD2[grp][r] = (float)(kr * c1);
      }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) sG[grp][lane][j] = 0.f;
    __syncwarp(gm);
    // this species' slope and its row of the rate Jacobian, from its own reactions
    double g = 0.0;
    for (int e = e0; e < e1; ++e) {
      const int code = __ldg(ae + e);
      const int r = code & 0xffff;
      const int nu = (code >> 16) - 4;
      g += (double)nu * sRate[grp][r];
      const int4 q = __ldg(tt + r);
      sG[grp][lane][q.x] += (float)nu * sD1[grp][r];
      if (q.y >= 0) sG[grp][lane][q.y] += (float)nu * sD2[grp][r];
    }
    __syncwarp(gm);
    float Gi[D], Kn[D];
#pragma unroll
    for (int j = 0; j < D; ++j) Gi[j] = sG[grp][lane][j];
#pragma unroll
    for (int j = 0; j < D; ++j) Kn[j] = Gi[j];
    if (stage > 0) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        const float gmv = cK * Gi[m];
#pragma unroll
        for (int j = 0; j < D; ++j) Kn[j] += gmv * sK[grp][m][j];
      }
    }
    __syncwarp(gm);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      sK[grp][lane][j] = Kn[j];
      Kacc[j] += (float)w * Kn[j];
    }
    acc += w * g;
    const double cs = stage == 2 ? h : 0.5 * h;
    c = s_prev + cs * g;
    __syncwarp(gm);
  }
  const double hw = RK4 ? h / 6.0 : h;
  const double F = s_prev + hw * acc;
  double mx = 0.0, sq = 0.0;
  if (valid) {
    const double sc = a.s[row * D + lane];
    const double rr = sc - F;
    const double sabs = fabs(sc);
    mx = fabs(rr) / (sabs > 1.0 ? sabs : 1.0);
    if (rr != rr) mx = rr;
    sq = rr * rr;
    const float scale = a.damp == DEER_DAMP_SCALE ? (float)(1.0 - a.dparam) : 1.f;
    __nv_bfloat16* Eo = a.E + row * (int64_t)(D * D) + lane * D;
    // E = A - I with A = I + hw Kacc (scaled by (1 - k) under scale-ELK: E = s A - I)
#pragma unroll
    for (int j = 0; j < D; j += 2) {
      const float e0 = scale * (float)hw * Kacc[j] + (j == lane ? scale - 1.f : 0.f);
      const float e1 = scale * (float)hw * Kacc[j + 1] + (j + 1 == lane ? scale - 1.f : 0.f);
      *reinterpret_cast<__nv_bfloat162*>(Eo + j) = __floats2bfloat162_rn(e0, e1);
    }
    a.b[row * D + lane] = (float)(-rr);
  }
  acc_resid(a.acc, seq, valid, mx, sq);
}

// ---- mixed dense scan: lane j owns column j of P and entry j of the vectors ----------
template <int D>
__global__ void __launch_bounds__(128) k_mixed_chunk(MixedScanArgs a) {
  constexpr int G = 128 / D;
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = gmask_mixed<D>();
  const int64_t ac = blockIdx.x * (int64_t)G + grp;
  const bool valid = ac < a.bt.act_chunks;
  int64_t seq = 0, c = 0, r0 = 0;
  int n = 0;
  if (valid) act_chunk(a.bt, ac, seq, c, r0, n);
  const bool need_P = valid && c != __ldg(a.bt.chunk_first + seq);
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
  const bool valid = kq < a.bt.n_act;
  const int64_t seq = valid ? a.bt.act_seq[kq] : 0;
  const int64_t c0 = valid ? a.bt.chunk_first[seq] : 0;
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
  const bool valid = ac < a.bt.act_chunks;
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

cudaError_t launch_lin_ma_mixed(const MixedLinArgs& a, cudaStream_t st) {
  if (a.bt.act_rows == 0) return cudaSuccess;
  const bool rk4 = a.dv.kind == DEER_F_MASSACTION_RK4;
  const int d = a.dv.d;
  const unsigned g = grid_for(a.bt.act_rows, 128 / d);
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
  const unsigned gc = grid_for(a.bt.act_chunks, G);
  const unsigned gs = grid_for(a.bt.n_act, G);
  k_mixed_chunk<D><<<gc, 128, 0, st>>>(a);
  k_mixed_carry<D><<<gs, 128, 0, st>>>(a);
  k_mixed_apply<D><<<gc, 128, 0, st>>>(a);
  note_launch(3);
}

cudaError_t launch_dense_scan_mixed(const MixedScanArgs& a, cudaStream_t st) {
  if (a.bt.act_rows == 0) return cudaSuccess;
  if (a.d == 16) mixed_launch<16>(a, st);
  else if (a.d == 32) mixed_launch<32>(a, st);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace deer
