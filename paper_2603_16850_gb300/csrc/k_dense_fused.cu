// Fused full-Jacobian Newton iteration for state sizes d <= 8 (see FusedArgs in
// kernels.h). One pass over HBM per iteration: read A_t, b_t and s_t, write s_t and the new
// A_t, b_t; the chunk aggregates for the next scan are formed on the fly, so the scan's
// separate aggregate pass (another full read of the Jacobians) disappears.
#include "dyn.cuh"
#include "kernels.h"

namespace deer {

template <class real, int D>
__device__ __forceinline__ void ld_vec(const real* __restrict__ p, real (&v)[D]) {
  ldrow<real, D>(p, v);
}

template <class real, int D>
__device__ __forceinline__ void st_vec(real* __restrict__ p, const real (&v)[D]) {
  constexpr int bytes = D * (int)sizeof(real);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i)
      reinterpret_cast<float4*>(p)[i] = reinterpret_cast<const float4*>(v)[i];
  } else if constexpr (bytes % 8 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 8; ++i)
      reinterpret_cast<float2*>(p)[i] = reinterpret_cast<const float2*>(v)[i];
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) p[i] = v[i];
  }
}

// F = f_t(prev), A = df_t/ds at prev
template <class real, int D, int KIND>
__device__ __forceinline__ void lin_eval(const DynView<real>& dv, int64_t seq, int64_t row,
                                         const real (&prev)[D], real (&F)[D],
                                         real (&A)[D][D]) {
  if constexpr (KIND == DEER_F_MASSACTION_EULER || KIND == DEER_F_MASSACTION_RK4) {
    const real* T = dv.ma + seq * dv.ma_stride;
    ma_step_cols<real, D, 1, KIND == DEER_F_MASSACTION_RK4, true>(T, dv.dt, 0, prev, F, A);
  } else {
    eval_f<real, D, KIND, 1>(dv, seq, row, prev, F, A, nullptr);
  }
}

constexpr int kFusedBlock = 128;

template <class real, int D, int KIND, int MODE>
__global__ void __launch_bounds__(kFusedBlock) k_dense_fused(FusedArgs<real> a) {
  constexpr int E = D * D;
  // thread-private scratch: chunk aggregate P, v and the values that must survive the
  // register-heavy linearisation (Delta and the new state of the current row)
  __shared__ real sP[E][kFusedBlock];
  __shared__ real sV[D][kFusedBlock];
  __shared__ real sD[D][kFusedBlock];
  __shared__ real sN[D][kFusedBlock];
  const int tid = threadIdx.x;
  const int64_t ac = blockIdx.x * (int64_t)blockDim.x + tid;
  const bool valid = ac < a.bt.act_chunks;
  int64_t seq = 0;
  double mx = 0.0, sq = 0.0;
  if (valid) {
    int64_t c, r0;
    int n;
    act_chunk(a.bt, ac, seq, c, r0, n);
    const int64_t gi = c >> 5;
    const int lane = (int)(c & 31);
    const int L = a.bt.L;
    const bool first = c == __ldg(a.bt.chunk_first + seq);
    const bool need_P = !first;
    const real k = a.dparam;
    const real scale = a.damp == DEER_DAMP_SCALE ? real(1) - k : real(1);
    real prev[D];
    if (first) {
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = a.s0[seq * D + i];
    } else if (MODE == 0) {
      ld_vec<real, D>(a.s + (r0 - 1) * D, prev);
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = a.sprev[c * D + i];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      sD[i][tid] = MODE == 1 ? a.cin[c * D + i] : real(0);
      sV[i][tid] = real(0);
#pragma unroll
      for (int j = 0; j < D; ++j) sP[i * D + j][tid] = i == j ? real(1) : real(0);
    }
    for (int t = 0; t < n; ++t) {
      const int64_t row = r0 + t;
      real* Arow = a.Ai + ((gi * L + t) * E) * 32 + lane;
      real* brow = a.bi + ((gi * L + t) * D) * 32 + lane;
      real sn[D];
      ld_vec<real, D>(a.s + row * D, sn);
      if constexpr (MODE == 1) {
        // apply the pending scan step: Delta_t = A_t Delta_{t-1} + b_t, s_t += Delta_t
        real dl[D], nd[D];
#pragma unroll
        for (int i = 0; i < D; ++i) dl[i] = sD[i][tid];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real v = brow[i * 32];
#pragma unroll
          for (int j = 0; j < D; ++j) v += Arow[(i * D + j) * 32] * dl[j];
          nd[i] = v;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
          sD[i][tid] = nd[i];
          real x = sn[i] + nd[i];
          if (a.reset && !(x <= a.reset_thr && x >= -a.reset_thr)) x = real(0);
          sn[i] = x;
        }
        st_vec<real, D>(a.s + row * D, sn);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) sN[i][tid] = sn[i];
      // linearise at the new state of the previous row
      real F[D], A[D][D];
      lin_eval<real, D, KIND>(a.dv, seq, row, prev, F, A);
      real r[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const real x = sN[i][tid];
        prev[i] = x;
        r[i] = x - F[i];
        const real sabs = rabs(x);
        mx = nanmax(mx, (double)rabs(r[i]) / (double)(sabs > real(1) ? sabs : real(1)));
        sq += (double)r[i] * (double)r[i];
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        brow[i * 32] = -r[i];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          A[i][j] *= scale;
          Arow[(i * D + j) * 32] = A[i][j];
        }
      }
      // chunk aggregate for the next scan: v <- A v - r, P <- A P (column by column)
      {
        real vv[D], nv[D];
#pragma unroll
        for (int i = 0; i < D; ++i) vv[i] = sV[i][tid];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real x = -r[i];
#pragma unroll
          for (int j = 0; j < D; ++j) x += A[i][j] * vv[j];
          nv[i] = x;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) sV[i][tid] = nv[i];
      }
      if (need_P) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          real col[D], nc[D];
#pragma unroll
          for (int i = 0; i < D; ++i) col[i] = sP[i * D + j][tid];
#pragma unroll
          for (int i = 0; i < D; ++i) {
            real x = real(0);
#pragma unroll
            for (int m = 0; m < D; ++m) x += A[i][m] * col[m];
            nc[i] = x;
          }
#pragma unroll
          for (int i = 0; i < D; ++i) sP[i * D + j][tid] = nc[i];
        }
      }
    }
    real* Po = a.aggP + c * (int64_t)E;
    real* vo = a.aggv + c * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      vo[i] = sV[i][tid];
#pragma unroll
      for (int j = 0; j < D; ++j) Po[i * D + j] = sP[i * D + j][tid];
    }
  }
  acc_resid(a.acc, seq, valid, mx, sq);
}

// Per active sequence: compose the chunk aggregates in order; record the Delta entering
// each chunk and the new state at the row before it (read from the old iterate before the
// fused pass overwrites it).
template <class real, int D>
__global__ void __launch_bounds__(128) k_dense_fused_carry(FusedArgs<real> a) {
  constexpr int E = D * D;
  const int64_t kq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (kq >= a.bt.n_act) return;
  const int64_t seq = a.bt.act_seq[kq];
  const int64_t c0 = a.bt.chunk_first[seq], c1 = a.bt.chunk_first[seq + 1];
  const int64_t base = a.bt.offsets[seq];
  real x[D];
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = real(0);
  real P[E], v[D];
  if (c0 < c1) {
    ld_vec<real, E>(a.aggP + c0 * E, *reinterpret_cast<real(*)[E]>(P));
    ld_vec<real, D>(a.aggv + c0 * D, v);
  }
  for (int64_t c = c0; c < c1; ++c) {
    real Pc[E], vc[D];
#pragma unroll
    for (int e = 0; e < E; ++e) Pc[e] = P[e];
#pragma unroll
    for (int i = 0; i < D; ++i) vc[i] = v[i];
    if (c + 1 < c1) {  // prefetch the next aggregate
      ld_vec<real, E>(a.aggP + (c + 1) * E, *reinterpret_cast<real(*)[E]>(P));
      ld_vec<real, D>(a.aggv + (c + 1) * D, v);
    }
#pragma unroll
    for (int i = 0; i < D; ++i) a.cin[c * D + i] = x[i];
    if (c > c0) {
      const int64_t r0 = base + ((c - c0) << a.bt.log2L);
      real so[D];
      ld_vec<real, D>(a.s + (r0 - 1) * D, so);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        real y = so[i] + x[i];
        if (a.reset && !(y <= a.reset_thr && y >= -a.reset_thr)) y = real(0);
        a.sprev[c * D + i] = y;
      }
    }
    real nx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      real y = vc[i];
      if (c > c0) {
#pragma unroll
        for (int j = 0; j < D; ++j) y += Pc[i * D + j] * x[j];
      }
      nx[i] = y;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = nx[i];
  }
}

template <class real, int D, int KIND>
static void fused_launch(const FusedArgs<real>& a, cudaStream_t st) {
  const unsigned g = grid_for(a.bt.act_chunks, kFusedBlock);
  if (a.mode == 0) k_dense_fused<real, D, KIND, 0><<<g, kFusedBlock, 0, st>>>(a);
  else k_dense_fused<real, D, KIND, 1><<<g, kFusedBlock, 0, st>>>(a);
}

template <class real, int KIND>
static cudaError_t fused_kind(const FusedArgs<real>& a, cudaStream_t st) {
  switch (a.dv.d) {
    case 1: if constexpr (KIND != DEER_F_BRUSSELATOR_EULER) { fused_launch<real, 1, KIND>(a, st); break; }
            return cudaErrorInvalidValue;
    case 2: fused_launch<real, 2, KIND>(a, st); break;
    case 4: if constexpr (KIND != DEER_F_BRUSSELATOR_EULER) { fused_launch<real, 4, KIND>(a, st); break; }
            return cudaErrorInvalidValue;
    case 8: if constexpr (KIND != DEER_F_BRUSSELATOR_EULER) { fused_launch<real, 8, KIND>(a, st); break; }
            return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_dense_fused(const FusedArgs<real>& a, cudaStream_t st) {
  if (a.bt.act_chunks == 0) return cudaSuccess;
  switch (a.dv.kind) {
    case DEER_F_BRUSSELATOR_EULER: return fused_kind<real, DEER_F_BRUSSELATOR_EULER>(a, st);
    case DEER_F_MASSACTION_EULER: return fused_kind<real, DEER_F_MASSACTION_EULER>(a, st);
    case DEER_F_MASSACTION_RK4: return fused_kind<real, DEER_F_MASSACTION_RK4>(a, st);
    case DEER_F_GRU: return fused_kind<real, DEER_F_GRU>(a, st);
    default: return fused_kind<real, DEER_F_LINEAR>(a, st);
  }
}

template <class real>
cudaError_t launch_dense_fused_carry(const FusedArgs<real>& a, cudaStream_t st) {
  if (a.bt.n_act == 0) return cudaSuccess;
  const unsigned g = grid_for(a.bt.n_act, 128);
  switch (a.dv.d) {
    case 1: k_dense_fused_carry<real, 1><<<g, 128, 0, st>>>(a); break;
    case 2: k_dense_fused_carry<real, 2><<<g, 128, 0, st>>>(a); break;
    case 4: k_dense_fused_carry<real, 4><<<g, 128, 0, st>>>(a); break;
    case 8: k_dense_fused_carry<real, 8><<<g, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_dense_fused<float>(const FusedArgs<float>&, cudaStream_t);
template cudaError_t launch_dense_fused<double>(const FusedArgs<double>&, cudaStream_t);
template cudaError_t launch_dense_fused_carry<float>(const FusedArgs<float>&, cudaStream_t);
template cudaError_t launch_dense_fused_carry<double>(const FusedArgs<double>&, cudaStream_t);

}  // namespace deer
