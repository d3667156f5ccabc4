// Generic-kernel launchers (initial guess, linearisation + residual, sequential rollout) of
// the mean-field RNN, the two-well Langevin sampler, Lorenz-96 and the input-selected
// permutation.
#include "lin_generic.cuh"

namespace deer {

template <class real>
cudaError_t launch_init_models(const InitArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_RNN_TANH: return generic_init<real, DEER_F_RNN_TANH>(a, st);
    case DEER_F_LANGEVIN_2WELL: return generic_init<real, DEER_F_LANGEVIN_2WELL>(a, st);
    case DEER_F_LORENZ96_DP5: return generic_init<real, DEER_F_LORENZ96_DP5>(a, st);
    case DEER_F_PERMUTE: return generic_init<real, DEER_F_PERMUTE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

constexpr int kRnnRows = 16;  // consecutive rows per lane group in k_lin_rnn_wide

// ----------------------------------------------------------------------------
// Mean-field RNN, d = 16 / 32: D lanes per row, lane i owns row i of W (registers) and
// entry i of s_{t-1}, F_t, r_t, b_t; tanh(s_j) and its derivative arrive by shuffles and
// lane i writes row i of A_t = W diag(1 - tanh(s_{t-1})^2).
// ----------------------------------------------------------------------------
template <class real, int D, int JAC>
__global__ void __launch_bounds__(128) k_lin_rnn_wide(LinArgs<real> a) {
  constexpr int GROUPS = 128 / D;
  constexpr int VW = 16 / (int)sizeof(real);
  __shared__ __align__(16) real sT[GROUPS][D * (D + 1)];  // transpose tile of A_t
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gmask = D == 32 ? 0xffffffffu : (0xffffu << (16 * ((threadIdx.x >> 4) & 1)));
  // each group walks kRnnRows consecutive active rows; the residual statistics of a
  // sequence are flushed once per group (one sequence usually spans all of them) instead
  // of once per row, which keeps the accumulator atomics of a long sequence uncontended
  const int64_t ar0 = (blockIdx.x * (int64_t)GROUPS + grp) * kRnnRows;
  int64_t cur = -1;
  real mx = real(0), sq = real(0);
  unsigned long long key = 0ull;  // first failing row (sliding window)
  for (int rr_i = 0; rr_i < kRnnRows; ++rr_i) {
    const int64_t ar = ar0 + rr_i;
    if (ar >= a.bt.act_rows()) break;  // uniform over the group
    int64_t seq, row;
    act_row(a.bt, ar, seq, row);
    if (seq != cur) {
      if (cur >= 0) acc_resid_group<D>(a.acc, cur, mx, sq, key, lane, gmask);
      cur = seq;
      mx = real(0);
      sq = real(0);
      key = 0ull;
    }
    const int64_t first = __ldg(a.bt.offsets + seq);
    const real sp = row == first ? a.s0[seq * D + lane] : a.s[(row - 1) * D + lane];
    const real th = tanh(sp);
    const real dth = real(1) - th * th;
    const real* Wr = a.dv.params + seq * a.dv.pstride + lane * D;
    real w[D];
#pragma unroll
    for (int k = 0; k < D; k += VW) {
      if constexpr (sizeof(real) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(Wr + k));
        w[k] = q.x; w[k + 1] = q.y; w[k + 2] = q.z; w[k + 3] = q.w;
      } else {
        const double2 q = __ldg(reinterpret_cast<const double2*>(Wr + k));
        w[k] = q.x; w[k + 1] = q.y;
      }
    }
    real F = a.dv.x ? __ldg(a.dv.x + row * D + lane) : real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) F += w[j] * __shfl_sync(gmask, th, j, D);
    const real sc = a.s[row * D + lane];
    const real rr = sc - F;
    const real sabs = rabs(sc);
    real m1 = rabs(rr) / (sabs > real(1) ? sabs : real(1));
    if (rr != rr) m1 = rr;  // keep NaN
    mx = (m1 > mx || m1 != m1) ? m1 : mx;
    sq += rr * rr;
    if (!(m1 <= a.tol) && key == 0ull) key = bad_key(true, row - first);
    const real k = a.dparam;
    if constexpr (JAC == DEER_JAC_FULL) {
      const real scale = a.damp == DEER_DAMP_SCALE ? real(1) - k : real(1);
      real Arow[D];
#pragma unroll
      for (int j = 0; j < D; ++j) Arow[j] = scale * w[j] * __shfl_sync(gmask, dth, j, D);
      store_block_rows<real, D>(sT[grp], a.A + row * (int64_t)(D * D), Arow, lane, gmask);
      a.b[row * D + lane] = -rr;
    } else {
      real ai;
      if constexpr (JAC == DEER_JAC_DIAG) {
        real wii = real(0);
#pragma unroll
        for (int j = 0; j < D; ++j)
          if (j == lane) wii = w[j];
        ai = wii * dth;
      } else if constexpr (JAC == DEER_JAC_IDENTITY) {
        ai = real(1);
      } else {
        ai = real(0);
      }
      if (a.damp == DEER_DAMP_SCALE) ai *= (real(1) - k);
      else if (a.damp == DEER_DAMP_CLIP) ai = ai > k ? k : (ai < -k ? -k : ai);
      if constexpr (JAC == DEER_JAC_DIAG) a.A[row * D + lane] = ai;
      a.b[row * D + lane] = F - ai * sp;
    }
  }
  if (cur >= 0) acc_resid_group<D>(a.acc, cur, mx, sq, key, lane, gmask);
}

template <class real, int JAC>
static cudaError_t lin_rnn_wide(const LinArgs<real>& a, cudaStream_t st) {
  const int d = a.dv.d;
  const unsigned g = grid_for(a.bt.act_rows(), 128 / d * kRnnRows);
  if (d == 16) k_lin_rnn_wide<real, 16, JAC><<<g, 128, 0, st>>>(a);
  else k_lin_rnn_wide<real, 32, JAC><<<g, 128, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_linearize_models(const LinArgs<real>& a, cudaStream_t st) {
  if (a.dv.kind == DEER_F_RNN_TANH && (a.dv.d == 16 || a.dv.d == 32)) {
    switch (a.jac) {
      case DEER_JAC_FULL: return lin_rnn_wide<real, DEER_JAC_FULL>(a, st);
      case DEER_JAC_DIAG: return lin_rnn_wide<real, DEER_JAC_DIAG>(a, st);
      case DEER_JAC_IDENTITY: return lin_rnn_wide<real, DEER_JAC_IDENTITY>(a, st);
      default: return lin_rnn_wide<real, DEER_JAC_ZERO>(a, st);
    }
  }
  switch (a.dv.kind) {
    case DEER_F_RNN_TANH:
      return generic_linearize<real, DEER_F_RNN_TANH>(a, st);
    case DEER_F_LANGEVIN_2WELL: return generic_linearize<real, DEER_F_LANGEVIN_2WELL>(a, st);
    case DEER_F_LORENZ96_DP5: return generic_linearize<real, DEER_F_LORENZ96_DP5>(a, st);
    case DEER_F_PERMUTE: return generic_linearize<real, DEER_F_PERMUTE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

// Sequential rollout of the mean-field RNN (baseline): D lanes per trajectory, lane i owns
// s_i and row i of W (in registers); every step broadcasts tanh(s_j) by shuffles. All
// groups of a warp run the warp's longest sequence so that the shuffles stay converged.
template <class real, int D>
__global__ void __launch_bounds__(128) k_rollout_rnn(RolloutArgs<real> a) {
  const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / D;
  const int lane = threadIdx.x % D;
  const bool live = gid < a.B;
  const int64_t seq = live ? gid : a.B - 1;
  const unsigned full = 0xffffffffu;
  int64_t r0, r1;
  rollout_rows(a, seq, r0, r1);
  const real* Wr = a.dv.params + seq * a.dv.pstride + lane * D;
  real w[D];
#pragma unroll
  for (int j = 0; j < D; ++j) w[j] = __ldg(Wr + j);
  real c = a.s0[seq * D + lane];
  const int64_t n = live ? r1 - r0 : 0;
  int64_t nmax = n;
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t v = __shfl_xor_sync(full, nmax, o);
    nmax = v > nmax ? v : nmax;
  }
  for (int64_t t = 0; t < nmax; ++t) {
    const real th = tanh(c);
    real v = (a.dv.x && t < n) ? __ldg(a.dv.x + (r0 + t) * D + lane) : real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) v += w[j] * __shfl_sync(full, th, j, D);
    if (t < n) {
      c = v;
      a.s[(r0 + t) * D + lane] = c;
    }
  }
}

template <class real>
cudaError_t launch_rollout_models(const RolloutArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_RNN_TANH: {
      const unsigned g = grid_for(a.B * (int64_t)a.dv.d, 128);
      switch (a.dv.d) {
        case 1: k_rollout_rnn<real, 1><<<g, 128, 0, st>>>(a); break;
        case 2: k_rollout_rnn<real, 2><<<g, 128, 0, st>>>(a); break;
        case 4: k_rollout_rnn<real, 4><<<g, 128, 0, st>>>(a); break;
        case 8: k_rollout_rnn<real, 8><<<g, 128, 0, st>>>(a); break;
        case 16: k_rollout_rnn<real, 16><<<g, 128, 0, st>>>(a); break;
        case 32: k_rollout_rnn<real, 32><<<g, 128, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
      }
      note_launch();
      return cudaGetLastError();
    }
    case DEER_F_LANGEVIN_2WELL: return generic_rollout<real, DEER_F_LANGEVIN_2WELL>(a, st);
    case DEER_F_LORENZ96_DP5: return generic_rollout<real, DEER_F_LORENZ96_DP5>(a, st);
    case DEER_F_PERMUTE: return generic_rollout<real, DEER_F_PERMUTE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_init_models<float>(const InitArgs<float>&, cudaStream_t);
template cudaError_t launch_init_models<double>(const InitArgs<double>&, cudaStream_t);
template cudaError_t launch_linearize_models<float>(const LinArgs<float>&, cudaStream_t);
template cudaError_t launch_linearize_models<double>(const LinArgs<double>&, cudaStream_t);
template cudaError_t launch_rollout_models<float>(const RolloutArgs<float>&, cudaStream_t);
template cudaError_t launch_rollout_models<double>(const RolloutArgs<double>&, cudaStream_t);

template <class real>
cudaError_t launch_input_grad_models(const InputGradArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_RNN_TANH: return generic_input_grad<real, DEER_F_RNN_TANH>(a, st);
    case DEER_F_LANGEVIN_2WELL: return generic_input_grad<real, DEER_F_LANGEVIN_2WELL>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_input_grad_models<float>(const InputGradArgs<float>&, cudaStream_t);
template cudaError_t launch_input_grad_models<double>(const InputGradArgs<double>&, cudaStream_t);

}  // namespace deer
