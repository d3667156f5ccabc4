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
// symmetric positive definite, so no pivoting). For few, long sequences the covariance
// recursion runs in parallel over time instead (chunk elements, carry, then this
// recursion per chunk from the carried covariance; see below).
#include "kernels.h"

namespace deer {

// One group of D lanes per sequence (CHUNKED = false: the covariance starts at zero at the
// sequence's first row) or per chunk (CHUNKED = true: it starts from the filtered
// covariance the carry pass computed for the chunk).
// lanes per block: 128, or 64 for d >= 16 (the shared buffers of the float64 kernels)
template <int D>
constexpr int elk_block() { return D >= 16 ? 64 : 128; }

template <class real, int D, bool CHUNKED>
__global__ void __launch_bounds__(128) k_elk_dense(ElkDenseArgs<real> a) {
  constexpr int G = elk_block<D>() / D;
  constexpr int RS = D + (D >= 4 ? 16 / (int)sizeof(real) : 1);  // padded row stride
  __shared__ real sP[G][D][RS];   // covariance P_{t-1}, then P^-_t
  __shared__ real sA[G][D][RS];   // A_t
  __shared__ real sS[G][2][RS];   // pivot row of the elimination (S and the inverse)
  const int grp = threadIdx.x / D, i = threadIdx.x % D;
  const unsigned gm = D >= 32 ? 0xffffffffu
                              : (((1u << D) - 1u) << ((threadIdx.x & 31) & ~(D - 1)));
  const int64_t k = blockIdx.x * (int64_t)G + grp;
  int64_t r_begin, r_end;
  const real lam = a.lambda;
  real (*P)[RS] = sP[grp];
  real (*Am)[RS] = sA[grp];
  real (*Sp)[RS] = sS[grp];
  if constexpr (CHUNKED) {
    if (k >= a.bt.act_chunks()) return;  // whole groups
    int64_t seq, c;
    int n;
    act_chunk(a.bt, k, seq, c, r_begin, n);
    r_end = r_begin + n;
    const real* Pin = a.cov_in + c * (int64_t)(D * D);
#pragma unroll
    for (int j = 0; j < D; ++j) P[i][j] = Pin[i * D + j];
  } else {
    if (k >= a.bt.n_act()) return;  // whole groups
    const int64_t seq = a.bt.act_seq[k];
    const int64_t cf = a.bt.chunk_first[seq];
    r_begin = a.bt.offsets[seq] + ((win_first(a.bt, seq) - cf) << a.bt.log2L);
    r_end = a.bt.offsets[seq + 1];
#pragma unroll
    for (int j = 0; j < D; ++j) P[i][j] = real(0);
  }
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

// ---------------------------------------------------------------------------
// The covariance recursion in parallel over time. One filtering step maps the incoming
// covariance P to A (I + P J)^{-1} P A^T + C with the step's element
// (A, C, J) = (c F_t, c I, lambda c F_t^T F_t), c = 1 / (1 + lambda) (process noise I,
// emission variance 1/lambda); elements combine associatively, e_i then e_j giving
// (A_j N A_i, A_j N C_i A_j^T + C_j, A_i^T N^T J_j A_i + J_i) with N = (I + C_i J_j)^{-1}
// (Sarkka and Garcia-Fernandez's parallel Kalman filter). The chunk pass folds each
// chunk's elements in order; the carry pass walks a sequence's chunks applying their
// aggregates to the covariance (one short chain per sequence: T / L steps instead of T);
// the per-chunk recursion above then rewrites (A_t, b_t) from the carried covariance.
// Lane i of a group owns row i of every d x d matrix; products read the other operand's
// rows from the group's shared buffers; inverses by Gauss-Jordan elimination with partial
// pivoting (I + C J is not symmetric).
// ---------------------------------------------------------------------------

// row i of Y = X M for X's row x (registers) and M's rows in shared memory
template <class real, int D, int RS>
__device__ __forceinline__ void row_times(const real (&x)[D], const real (*M)[RS], real (&y)[D]) {
#pragma unroll
  for (int j = 0; j < D; ++j) y[j] = real(0);
#pragma unroll
  for (int m = 0; m < D; ++m)
#pragma unroll
    for (int j = 0; j < D; ++j) y[j] += x[m] * M[m][j];
}

// row i of S^{-1} for S's row s (destroyed); piv: two shared rows, out: D shared rows
template <class real, int D, int RS>
__device__ __forceinline__ void gj_inverse(real (&s)[D], real (&inv)[D], int i, unsigned gm,
                                           real (*piv)[RS], real (*out)[RS]) {
  real e[D];
#pragma unroll
  for (int j = 0; j < D; ++j) e[j] = j == i ? real(1) : real(0);
  bool used = false;
  int mycol = 0;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    // pivot: the unused row with the largest |s_c| (ties to the lower lane)
    real key = used ? real(-1) : (s[c] < real(0) ? -s[c] : s[c]);
    int who = i;
#pragma unroll
    for (int o = D / 2; o > 0; o >>= 1) {
      const real ok = __shfl_xor_sync(gm, key, o, D);
      const int ow = __shfl_xor_sync(gm, who, o, D);
      if (ok > key || (ok == key && ow < who)) { key = ok; who = ow; }
    }
    if (i == who) {
      const real ip = real(1) / s[c];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        s[j] *= ip;
        e[j] *= ip;
        piv[0][j] = s[j];
        piv[1][j] = e[j];
      }
      used = true;
      mycol = c;
    }
    __syncwarp(gm);
    if (i != who) {
      const real f = s[c];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        s[j] -= f * piv[0][j];
        e[j] -= f * piv[1][j];
      }
    }
    __syncwarp(gm);
  }
  // the lane that pivoted on column c holds row c of the inverse
#pragma unroll
  for (int j = 0; j < D; ++j) out[mycol][j] = e[j];
  __syncwarp(gm);
#pragma unroll
  for (int j = 0; j < D; ++j) inv[j] = out[i][j];
  __syncwarp(gm);
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_elk_cov_chunk(ElkDenseArgs<real> a) {
  constexpr int G = elk_block<D>() / D;
  constexpr int RS = D + (D >= 4 ? 16 / (int)sizeof(real) : 1);
  __shared__ real sM[G][4][D][RS];  // exchange buffers
  __shared__ real sV[G][2][RS];
  const int grp = threadIdx.x / D, i = threadIdx.x % D;
  const unsigned gm = D >= 32 ? 0xffffffffu
                              : (((1u << D) - 1u) << ((threadIdx.x & 31) & ~(D - 1)));
  const int64_t k = blockIdx.x * (int64_t)G + grp;
  if (k >= a.bt.act_chunks()) return;  // whole groups
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, k, seq, c, r0, n);
  const real lam = a.lambda;
  const real cc = real(1) / (real(1) + lam);
  real (*F)[RS] = sM[grp][0];
  real (*B1)[RS] = sM[grp][1];
  real (*B2)[RS] = sM[grp][2];
  real (*B3)[RS] = sM[grp][3];
  real Aa[D], Ca[D], Ja[D];  // rows i of the chunk's aggregate element
  for (int t = 0; t < n; ++t) {
    const real* Fr = a.A + (r0 + t) * (int64_t)(D * D) + i * D;
    real f[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      f[j] = Fr[j];
      F[i][j] = f[j];
    }
    __syncwarp(gm);
    // J_e row i = lambda c sum_m F_mi F_m
    real je[D];
#pragma unroll
    for (int j = 0; j < D; ++j) je[j] = real(0);
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int j = 0; j < D; ++j) je[j] += F[m][i] * F[m][j];
#pragma unroll
    for (int j = 0; j < D; ++j) je[j] *= lam * cc;
    if (t == 0) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        Aa[j] = cc * f[j];
        Ca[j] = j == i ? cc : real(0);
        Ja[j] = je[j];
      }
      __syncwarp(gm);
      continue;
    }
    // N = (I + C_a J_e)^{-1}
#pragma unroll
    for (int j = 0; j < D; ++j) B1[i][j] = je[j];
    __syncwarp(gm);
    real sr[D], nr[D];
    row_times<real, D, RS>(Ca, B1, sr);
#pragma unroll
    for (int j = 0; j < D; ++j) sr[j] += j == i ? real(1) : real(0);
    __syncwarp(gm);
    gj_inverse<real, D, RS>(sr, nr, i, gm, sV[grp], B2);
    // X = N A_a, Y = N C_a (rows i)
#pragma unroll
    for (int j = 0; j < D; ++j) { B2[i][j] = Aa[j]; B3[i][j] = Ca[j]; }
    __syncwarp(gm);
    real xr[D], yr[D];
    row_times<real, D, RS>(nr, B2, xr);
    row_times<real, D, RS>(nr, B3, yr);
    // V = J_e A_a (row i; B1 holds J_e, B2 holds A_a)
    real vr[D];
    row_times<real, D, RS>(je, B2, vr);
    __syncwarp(gm);
    // A_new = c F X; Z = F Y; C_new = c^2 Z F^T + c I
#pragma unroll
    for (int j = 0; j < D; ++j) { B1[i][j] = xr[j]; B3[i][j] = yr[j]; }
    __syncwarp(gm);
    real an[D], zr[D];
    row_times<real, D, RS>(f, B1, an);
    row_times<real, D, RS>(f, B3, zr);
    real cn[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      real x = real(0);
#pragma unroll
      for (int m = 0; m < D; ++m) x += zr[m] * F[j][m];
      cn[j] = cc * cc * x + (j == i ? cc : real(0));
    }
    // J_new = A_a^T (N^T V) + J_a: W = N^T V (row i = sum_m N_mi V_m), then rows
    // sum_m A_a[m][i] W[m]
    __syncwarp(gm);
#pragma unroll
    for (int j = 0; j < D; ++j) { B1[i][j] = nr[j]; B3[i][j] = vr[j]; }
    __syncwarp(gm);
    real wr[D];
#pragma unroll
    for (int j = 0; j < D; ++j) wr[j] = real(0);
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int j = 0; j < D; ++j) wr[j] += B1[m][i] * B3[m][j];
    __syncwarp(gm);
#pragma unroll
    for (int j = 0; j < D; ++j) B3[i][j] = wr[j];
    __syncwarp(gm);
    real jn[D];
#pragma unroll
    for (int j = 0; j < D; ++j) jn[j] = Ja[j];
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int j = 0; j < D; ++j) jn[j] += B2[m][i] * B3[m][j];
    __syncwarp(gm);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      Aa[j] = cc * an[j];
      Ca[j] = cn[j];
      Ja[j] = jn[j];
    }
  }
  real* out = a.cov_agg + c * (int64_t)(3 * D * D);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    out[i * D + j] = Aa[j];
    out[D * D + i * D + j] = Ca[j];
    out[2 * D * D + i * D + j] = Ja[j];
  }
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_elk_cov_carry(ElkDenseArgs<real> a) {
  constexpr int G = elk_block<D>() / D;
  constexpr int RS = D + (D >= 4 ? 16 / (int)sizeof(real) : 1);
  __shared__ real sM[G][3][D][RS];
  __shared__ real sV[G][2][RS];
  const int grp = threadIdx.x / D, i = threadIdx.x % D;
  const unsigned gm = D >= 32 ? 0xffffffffu
                              : (((1u << D) - 1u) << ((threadIdx.x & 31) & ~(D - 1)));
  const int64_t kq = blockIdx.x * (int64_t)G + grp;
  if (kq >= a.bt.n_act()) return;  // whole groups
  const int64_t seq = a.bt.act_seq[kq];
  const int64_t c0 = win_first(a.bt, seq), c1 = a.bt.chunk_first[seq + 1];
  real (*Pm)[RS] = sM[grp][0];
  real (*B1)[RS] = sM[grp][1];
  real (*B2)[RS] = sM[grp][2];
  real p[D];
#pragma unroll
  for (int j = 0; j < D; ++j) p[j] = real(0);
  for (int64_t c = c0; c < c1; ++c) {
    real* pin = a.cov_in + c * (int64_t)(D * D);
#pragma unroll
    for (int j = 0; j < D; ++j) pin[i * D + j] = p[j];
    const real* e = a.cov_agg + c * (int64_t)(3 * D * D);
    real ar[D], cr[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      ar[j] = e[i * D + j];
      cr[j] = e[D * D + i * D + j];
      B1[i][j] = e[2 * D * D + i * D + j];  // J
      Pm[i][j] = p[j];
    }
    __syncwarp(gm);
    // N = (I + P J)^{-1}; P_out = A N P A^T + C
    real sr[D], nr[D];
    row_times<real, D, RS>(p, B1, sr);
#pragma unroll
    for (int j = 0; j < D; ++j) sr[j] += j == i ? real(1) : real(0);
    __syncwarp(gm);
    gj_inverse<real, D, RS>(sr, nr, i, gm, sV[grp], B2);
    real yr[D];
    row_times<real, D, RS>(nr, Pm, yr);  // (N P)_i
    __syncwarp(gm);
#pragma unroll
    for (int j = 0; j < D; ++j) { B1[i][j] = yr[j]; B2[i][j] = ar[j]; }
    __syncwarp(gm);
    real zr[D];
    row_times<real, D, RS>(ar, B1, zr);  // (A N P)_i
#pragma unroll
    for (int j = 0; j < D; ++j) {
      real x = cr[j];
#pragma unroll
      for (int m = 0; m < D; ++m) x += zr[m] * B2[j][m];
      p[j] = x;
    }
    __syncwarp(gm);
  }
}

template <class real, int D>
static void elk_dense_launch(const ElkDenseArgs<real>& a, cudaStream_t st) {
  constexpr int NT = elk_block<D>();
  constexpr int G = NT / D;
  if (a.cov_agg) {
    const unsigned gc = grid_for(a.bt.act_chunks(), G);
    k_elk_cov_chunk<real, D><<<gc, NT, 0, st>>>(a);
    k_elk_cov_carry<real, D><<<grid_for(a.bt.n_act(), G), NT, 0, st>>>(a);
    k_elk_dense<real, D, true><<<gc, NT, 0, st>>>(a);
    note_launch(3);
  } else {
    k_elk_dense<real, D, false><<<grid_for(a.bt.n_act(), G), NT, 0, st>>>(a);
    note_launch();
  }
}

template <class real>
cudaError_t launch_elk_dense(const ElkDenseArgs<real>& a, cudaStream_t st) {
  if (a.bt.n_act() == 0) return cudaSuccess;
  switch (a.d) {
    case 1: elk_dense_launch<real, 1>(a, st); break;
    case 2: elk_dense_launch<real, 2>(a, st); break;
    case 4: elk_dense_launch<real, 4>(a, st); break;
    case 8: elk_dense_launch<real, 8>(a, st); break;
    case 16: elk_dense_launch<real, 16>(a, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_elk_dense<float>(const ElkDenseArgs<float>&, cudaStream_t);
template cudaError_t launch_elk_dense<double>(const ElkDenseArgs<double>&, cudaStream_t);

}  // namespace deer
