// Dense (full-Jacobian) ELK (Sec. 4.2-4.3): the Kalman filter of the linearised dynamics
// s_t = A_t s_{t-1} + b_t + N(0, I) with the previous iterate as emissions, variance 1/lambda.
// In the correction form of the scan the filtered mean is a linear recurrence again:
// Delta_t = Gamma_t A_t Delta_{t-1} - Gamma_t r_t, Gamma_t = (I + lambda P^-_t)^{-1}, where
// P^-_t = A_t P_{t-1} A_t^T + I, P_t = Gamma_t P^-_t and P = 0 before the first solved row
// (s_0, or the frozen state under a sliding window, is known). This kernel runs the
// covariance recursion and rewrites A_t <- Gamma_t A_t, b_t <- Gamma_t b_t in place; the
// dense scan then solves the mean in parallel over t. The covariance recursion does not
// depend on the emissions, only on A_t; it is a dependent chain over t, run by a group of
// d lanes per sequence (lane i owns row i of every d x d matrix) with the rows exchanged
// through shared memory, and the inverse by Gauss-Jordan elimination (I + lambda P^- is
// symmetric positive definite, so no pivoting).
#include "kernels.h"

namespace deer {

template <class real, int D>
__global__ void __launch_bounds__(128) k_elk_dense(ElkDenseArgs<real> a) {
  constexpr int G = 128 / D;
  constexpr int RS = D + (D >= 4 ? 16 / (int)sizeof(real) : 1);  // padded row stride
  __shared__ real sP[G][D][RS];   // covariance P_{t-1}, then P^-_t
  __shared__ real sA[G][D][RS];   // A_t
  __shared__ real sS[G][2][RS];   // pivot row of the elimination (S and the inverse)
  const int grp = threadIdx.x / D, i = threadIdx.x % D;
  const unsigned gm = D >= 32 ? 0xffffffffu
                              : (((1u << D) - 1u) << ((threadIdx.x & 31) & ~(D - 1)));
  const int64_t k = blockIdx.x * (int64_t)G + grp;
  if (k >= a.bt.n_act) return;  // whole groups
  const int64_t seq = a.bt.act_seq[k];
  const int64_t cf = a.bt.chunk_first[seq];
  const int64_t r_begin = a.bt.offsets[seq] + ((win_first(a.bt, seq) - cf) << a.bt.log2L);
  const int64_t r_end = a.bt.offsets[seq + 1];
  const real lam = a.lambda;
  real (*P)[RS] = sP[grp];
  real (*Am)[RS] = sA[grp];
  real (*Sp)[RS] = sS[grp];
#pragma unroll
  for (int j = 0; j < D; ++j) P[i][j] = real(0);
  __syncwarp(gm);
  for (int64_t row = r_begin; row < r_end; ++row) {
    real* Ar = a.A + row * (int64_t)(D * D) + i * D;
    real arow[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      arow[j] = Ar[j];
      Am[i][j] = arow[j];
    }
    __syncwarp(gm);
    // (A P)_i = sum_m A_im P_m
    real ap[D];
#pragma unroll
    for (int j = 0; j < D; ++j) ap[j] = real(0);
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int j = 0; j < D; ++j) ap[j] += arow[m] * P[m][j];
    // P^-_ij = sum_m (A P)_im A_jm + delta_ij; S = I + lambda P^-, augmented with I
    real pm[D], s[D], e[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      real x = j == i ? real(1) : real(0);
#pragma unroll
      for (int m = 0; m < D; ++m) x += ap[m] * Am[j][m];
      pm[j] = x;
      s[j] = (j == i ? real(1) : real(0)) + lam * x;
      e[j] = j == i ? real(1) : real(0);
    }
    __syncwarp(gm);
#pragma unroll
    for (int j = 0; j < D; ++j) P[i][j] = pm[j];  // P^- rows for the update below
    // Gauss-Jordan: S e = I row by row; pivot row c is broadcast through shared memory
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (i == c) {
        const real inv = real(1) / s[c];
#pragma unroll
        for (int j = 0; j < D; ++j) { s[j] *= inv; e[j] *= inv; Sp[0][j] = s[j]; Sp[1][j] = e[j]; }
      }
      __syncwarp(gm);
      if (i != c) {
        const real fct = s[c];
#pragma unroll
        for (int j = 0; j < D; ++j) { s[j] -= fct * Sp[0][j]; e[j] -= fct * Sp[1][j]; }
      }
      __syncwarp(gm);
    }
    // e = row i of Gamma = S^{-1}; P_t = Gamma P^-; A <- Gamma A; b <- Gamma b
    real np[D], na[D];
#pragma unroll
    for (int j = 0; j < D; ++j) { np[j] = real(0); na[j] = real(0); }
#pragma unroll
    for (int m = 0; m < D; ++m) {
      const real g = e[m];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        np[j] += g * P[m][j];
        na[j] += g * Am[m][j];
      }
    }
    const real bi = a.b[row * D + i];
    real nb = real(0);
#pragma unroll
    for (int m = 0; m < D; ++m) nb += e[m] * __shfl_sync(gm, bi, m, D);
    __syncwarp(gm);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      P[i][j] = np[j];
      Ar[j] = na[j];
    }
    a.b[row * D + i] = nb;
    __syncwarp(gm);
  }
}

template <class real>
cudaError_t launch_elk_dense(const ElkDenseArgs<real>& a, cudaStream_t st) {
  if (a.bt.n_act == 0) return cudaSuccess;
  switch (a.d) {
    case 1: k_elk_dense<real, 1><<<grid_for(a.bt.n_act, 128), 128, 0, st>>>(a); break;
    case 2: k_elk_dense<real, 2><<<grid_for(a.bt.n_act, 64), 128, 0, st>>>(a); break;
    case 4: k_elk_dense<real, 4><<<grid_for(a.bt.n_act, 32), 128, 0, st>>>(a); break;
    case 8: k_elk_dense<real, 8><<<grid_for(a.bt.n_act, 16), 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_elk_dense<float>(const ElkDenseArgs<float>&, cudaStream_t);
template cudaError_t launch_elk_dense<double>(const ElkDenseArgs<double>&, cudaStream_t);

}  // namespace deer
