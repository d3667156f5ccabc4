// Generic one-thread-per-row kernels shared by every dynamics kind evaluated through
// eval_f: the initial guess, linearisation + residual, and the sequential rollout, with
// launchers templated on the kind. Each translation unit instantiates the launchers for
// its own kinds (generic_launchers), so the heavy per-kind code compiles in parallel.
#pragma once

#include "dyn.cuh"
#include "kernels.h"

namespace deer {

// ----------------------------------------------------------------------------
// Row loads / stores with the widest aligned vector access.
// ----------------------------------------------------------------------------
template <class real, int D>
__device__ __forceinline__ void load_row(const real* __restrict__ p, real* v) {
  constexpr int bytes = D * (int)sizeof(real);
  if constexpr (bytes % 16 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i) {
      float4 w = __ldg(q + i);
      reinterpret_cast<float4*>(v)[i] = w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = __ldg(p + i);
  }
}

template <class real, int D>
__device__ __forceinline__ void store_row(real* __restrict__ p, const real* v) {
  constexpr int bytes = D * (int)sizeof(real);
  if constexpr (bytes % 16 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i) q[i] = reinterpret_cast<const float4*>(v)[i];
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) p[i] = v[i];
  }
}

// ----------------------------------------------------------------------------
// Initial guess
// ----------------------------------------------------------------------------
template <class real, int D, int KIND>
__global__ void __launch_bounds__(128) k_init(InitArgs<real> a) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= a.bt.N) return;
  const int64_t seq = find_seq(a.bt.offsets, a.bt.B, row);
  real v[D];
  if (a.init == DEER_INIT_ZEROS) {
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) v[i] = real(0);
  } else if (a.init == DEER_INIT_S0) {
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) v[i] = a.s0[seq * D + i];
  } else {  // Jacobi: f_t(0)
    real z[D];
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) z[i] = real(0);
    eval_f<real, D, KIND, 0>(a.dv, seq, row, z, v, nullptr, nullptr);
  }
  store_row<real, D>(a.s + row * D, v);
}

// ----------------------------------------------------------------------------
// Linearise + residual (one thread per row): F_t = f_t(s_{t-1}), A~_t, r_t = s_t - F_t.
//   FULL (correction form, Eq. lin_rr):  A[row] = A~_t (D x D), b[row] = -r_t
//   DIAG family (standard form, Eq. quasi_lds): a[row] = diag A~_t (DIAG only),
//                                               b[row] = F_t - a_t * s_{t-1}
// Rows of converged sequences are skipped. max |r| and sum r^2 go to the sequence's
// accumulator (float64).
// ----------------------------------------------------------------------------
template <class real, int D, int KIND, int JAC>
__global__ void __launch_bounds__(128) k_linearize(LinArgs<real> a) {
  const int64_t ar = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = ar < a.bt.act_rows();
  int64_t seq = 0, row = 0;
  real mx = real(0), sq = real(0);
  unsigned long long key = 0ull;  // first failing row (sliding window)
  if (valid) act_row(a.bt, ar, seq, row);
  if (valid) {
    const int64_t first = __ldg(a.bt.offsets + seq);
    real sp[D], sc[D], F[D];
    if (row == first) {
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i) sp[i] = __ldg(a.s0 + seq * D + i);
    } else {
      load_row<real, D>(a.s + (row - 1) * D, sp);
    }
    load_row<real, D>(a.s + row * D, sc);
    const real k = a.dparam;
    if constexpr (JAC == DEER_JAC_FULL) {
      real A[D][D];
      eval_f<real, D, KIND, 1>(a.dv, seq, row, sp, F, A, nullptr);
      const real scale = (a.damp == DEER_DAMP_SCALE) ? real(1) - k : real(1);
      real* Ao = a.A + row * (int64_t)(D * D);
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i) {
        real rowv[D];
#pragma unroll Unroll<D>::n
        for (int j = 0; j < D; ++j) rowv[j] = scale * A[i][j];
        store_row<real, D>(Ao + i * D, rowv);
      }
      real b[D];
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i) {
        real r = sc[i] - F[i];
        b[i] = -r;
        const real sabs = rabs(sc[i]);
        const real sr = rabs(r) / (sabs > real(1) ? sabs : real(1));
        mx = (sr > mx || sr != sr) ? sr : mx;
        if (!(sr <= a.tol)) key = bad_key(true, row - __ldg(a.bt.offsets + seq));
        sq += r * r;
      }
      store_row<real, D>(a.b + row * D, b);
    } else {
      real ad_[D];
      if constexpr (JAC == DEER_JAC_DIAG) {
        eval_f<real, D, KIND, 2>(a.dv, seq, row, sp, F, nullptr, ad_);
      } else {
        eval_f<real, D, KIND, 0>(a.dv, seq, row, sp, F, nullptr, nullptr);
      }
      real b[D];
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i) {
        real ai;
        if constexpr (JAC == DEER_JAC_DIAG) ai = ad_[i];
        else if constexpr (JAC == DEER_JAC_IDENTITY) ai = real(1);
        else ai = real(0);
        if (a.damp == DEER_DAMP_SCALE) ai *= (real(1) - k);
        else if (a.damp == DEER_DAMP_CLIP) ai = ai > k ? k : (ai < -k ? -k : ai);
        ad_[i] = ai;
        b[i] = F[i] - ai * sp[i];
        real r = sc[i] - F[i];
        const real sabs = rabs(sc[i]);
        const real sr = rabs(r) / (sabs > real(1) ? sabs : real(1));
        mx = (sr > mx || sr != sr) ? sr : mx;
        if (!(sr <= a.tol)) key = bad_key(true, row - __ldg(a.bt.offsets + seq));
        sq += r * r;
      }
      if constexpr (JAC == DEER_JAC_DIAG) store_row<real, D>(a.A + row * D, ad_);
      store_row<real, D>(a.b + row * D, b);
    }
  }
  acc_resid_t(a.acc, seq, valid, mx, sq, key);
}

// ----------------------------------------------------------------------------
// Sequential rollout (baseline), one thread per trajectory.
// ----------------------------------------------------------------------------
template <class real, int D, int KIND>
__global__ void __launch_bounds__(128) k_rollout_generic(RolloutArgs<real> a) {
  const int64_t seq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (seq >= a.B) return;
  int64_t r0, r1;
  rollout_rows(a, seq, r0, r1);
  real c[D], F[D];
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) c[i] = a.s0[seq * D + i];
  for (int64_t row = r0; row < r1; ++row) {
    eval_f<real, D, KIND, 0>(a.dv, seq, row, c, F, nullptr, nullptr);
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) c[i] = F[i];
    store_row<real, D>(a.s + row * D, c);
  }
}

// State sizes the generic kernels are instantiated for, per kind.
constexpr bool kind_has_d(int kind, int d, bool full) {
  return kind == DEER_F_BRUSSELATOR_EULER ? d == 2
       : kind == DEER_F_LORENZ96_DP5 ? (d == 4 || d == 5 || d == 8)
       : kind == DEER_F_PERMUTE ? (d == 2 || d == 4 || d == 5 || d == 8 || d == 16 || d == 32)
       : kind == DEER_F_GRU ? (d == 1 || d == 2 || d == 4 || d == 8 || d == 16 || d == 32 ||
                               (d == 64 && !full))
       : (d == 1 || d == 2 || d == 4 || d == 8 || d == 16 || d == 32);
}

#define DEER_GENERIC_D(X) X(1) X(2) X(4) X(5) X(8) X(16) X(32) X(64)

// Jacobi guess of an autonomous recurrence (mass action: f_t does not depend on t or on
// inputs): f(0) once per sequence into its first row, then copied along the sequence,
// instead of evaluating the same step at zero on every row
template <class real, int D, int KIND>
__global__ void __launch_bounds__(128) k_init_jacobi_first(InitArgs<real> a) {
  const int64_t seq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (seq >= a.bt.B) return;
  const int64_t r0 = a.bt.offsets[seq];
  if (a.bt.offsets[seq + 1] == r0) return;  // empty sequence
  real z[D], v[D];
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) z[i] = real(0);
  eval_f<real, D, KIND, 0>(a.dv, seq, r0, z, v, nullptr, nullptr);
  store_row<real, D>(a.s + r0 * D, v);
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_init_copy_first(InitArgs<real> a) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= a.bt.N) return;
  const int64_t r0 = a.bt.offsets[find_seq(a.bt.offsets, a.bt.B, row)];
  if (row == r0) return;
  real v[D];
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) v[i] = a.s[r0 * D + i];
  store_row<real, D>(a.s + row * D, v);
}

template <class real, int KIND>
cudaError_t generic_init(const InitArgs<real>& a, cudaStream_t st) {
  const unsigned g = grid_for(a.bt.N, 128);
  constexpr bool autonomous = KIND == DEER_F_MASSACTION_EULER || KIND == DEER_F_MASSACTION_RK4;
  if (autonomous && a.init == DEER_INIT_JACOBI) {
    switch (a.dv.d) {
#define CASE(DD)                                                                   \
  case DD:                                                                         \
    if constexpr (kind_has_d(KIND, DD, false)) {                                   \
      k_init_jacobi_first<real, DD, KIND><<<grid_for(a.bt.B, 128), 128, 0, st>>>(a); \
      k_init_copy_first<real, DD><<<g, 128, 0, st>>>(a);                           \
      break;                                                                       \
    }                                                                              \
    return cudaErrorInvalidValue;
      DEER_GENERIC_D(CASE)
#undef CASE
      default:
        return cudaErrorInvalidValue;
    }
    note_launch(2);
    return cudaGetLastError();
  }
  switch (a.dv.d) {
#define CASE(DD)                                                              \
  case DD:                                                                    \
    if constexpr (kind_has_d(KIND, DD, false)) {                              \
      k_init<real, DD, KIND><<<g, 128, 0, st>>>(a);                           \
      break;                                                                  \
    }                                                                         \
    return cudaErrorInvalidValue;
    DEER_GENERIC_D(CASE)
#undef CASE
    default:
      return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <class real, int KIND, int JAC>
static cudaError_t generic_linearize_jac(const LinArgs<real>& a, cudaStream_t st) {
  const unsigned g = grid_for(a.bt.act_rows(), 128);
  constexpr bool full = JAC == DEER_JAC_FULL;
  switch (a.dv.d) {
#define CASE(DD)                                                              \
  case DD:                                                                    \
    if constexpr (kind_has_d(KIND, DD, full)) {                               \
      k_linearize<real, DD, KIND, JAC><<<g, 128, 0, st>>>(a);                 \
      break;                                                                  \
    }                                                                         \
    return cudaErrorInvalidValue;
    DEER_GENERIC_D(CASE)
#undef CASE
    default:
      return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <class real, int KIND>
cudaError_t generic_linearize(const LinArgs<real>& a, cudaStream_t st) {
  switch (a.jac) {
    case DEER_JAC_FULL: return generic_linearize_jac<real, KIND, DEER_JAC_FULL>(a, st);
    case DEER_JAC_DIAG: return generic_linearize_jac<real, KIND, DEER_JAC_DIAG>(a, st);
    case DEER_JAC_IDENTITY: return generic_linearize_jac<real, KIND, DEER_JAC_IDENTITY>(a, st);
    default: return generic_linearize_jac<real, KIND, DEER_JAC_ZERO>(a, st);
  }
}

template <class real, int KIND>
cudaError_t generic_rollout(const RolloutArgs<real>& a, cudaStream_t st) {
  const unsigned g = grid_for(a.B, 128);
  switch (a.dv.d) {
#define CASE(DD)                                                              \
  case DD:                                                                    \
    if constexpr (kind_has_d(KIND, DD, false)) {                              \
      k_rollout_generic<real, DD, KIND><<<g, 128, 0, st>>>(a);                \
      break;                                                                  \
    }                                                                         \
    return cudaErrorInvalidValue;
    DEER_GENERIC_D(CASE)
#undef CASE
    default:
      return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

// Input gradient, one thread per row.
template <class real, int D, int KIND>
__global__ void __launch_bounds__(128) k_input_grad(InputGradArgs<real> a) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= a.bt.N) return;
  const int64_t seq = find_seq(a.bt.offsets, a.bt.B, row);
  real h[D], lam[D];
  if (row == __ldg(a.bt.offsets + seq)) {
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) h[i] = __ldg(a.s0 + seq * D + i);
  } else {
    load_row<real, D>(a.s + (row - 1) * D, h);
  }
  load_row<real, D>(a.lam + row * D, lam);
  input_vjp<real, D, KIND>(a.dv, row, h, lam, a.dx + row * (int64_t)a.dv.d_in);
}

template <class real, int KIND>
cudaError_t generic_input_grad(const InputGradArgs<real>& a, cudaStream_t st) {
  const unsigned g = grid_for(a.bt.N, 128);
  switch (a.dv.d) {
#define CASE(DD)                                                              \
  case DD:                                                                    \
    if constexpr (kind_has_d(KIND, DD, true)) {                               \
      k_input_grad<real, DD, KIND><<<g, 128, 0, st>>>(a);                     \
      break;                                                                  \
    }                                                                         \
    return cudaErrorInvalidValue;
    DEER_GENERIC_D(CASE)
#undef CASE
    default:
      return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace deer
