// Largest Lyapunov exponent along a trajectory (Algorithm alg:LLE_estimate): a unit vector
// is pushed through the step Jacobians J_t = df_t/ds (evaluated at s_{t-1} by the
// linearisation kernels and stored row-major) and renormalised every step; the estimate
// is the mean log stretch. A group of W lanes walks one sequence (W = d rounded up to a
// power of two): lane i < d owns entry i of the vector and row i of J_t, the other entries
// arrive by shuffles and the norm by a butterfly reduction inside the group; lanes i >= d
// hold zeros.
#include "kernels.h"

namespace deer {

constexpr int pow2_ceil(int v) { return v <= 1 ? 1 : 2 * pow2_ceil((v + 1) / 2); }

template <class real, int D>
__global__ void __launch_bounds__(128) k_lle(LleArgs<real> a) {
  constexpr int W = pow2_ceil(D);  // lanes per sequence
  static_assert(W <= 32, "one sequence per warp at most");
  const int lane = threadIdx.x & 31, i = lane % W;
  const bool own = i < D;
  const unsigned gm = W >= 32 ? 0xffffffffu : (((1u << W) - 1u) << (lane & ~(W - 1)));
  const int64_t seq = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / W;
  if (seq >= a.B) return;  // whole groups
  real u = own ? a.u0[seq * D + i] : real(0);
  double acc = 0.0;
  const int64_t r0 = seq * a.T;
  for (int64_t t = 0; t < a.T; ++t) {
    const real* Jr = a.A + (r0 + t) * (int64_t)(D * D) + (own ? i : 0) * D;
    real v = real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const real uj = __shfl_sync(gm, u, j, W);
      if (own) v += __ldg(Jr + j) * uj;
    }
    real n2 = v * v;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) n2 += __shfl_xor_sync(gm, n2, o, W);
    const real lam = sqrt(n2);          // stretch factor
    u = v / lam;                        // renormalise
    if constexpr (sizeof(real) == 8) acc += log(lam);
    else acc += (double)logf(lam);      // accumulate the log stretch
  }
  if (i == 0) a.out[seq] = acc / (double)a.T;
}

template <class real>
cudaError_t launch_lle(const LleArgs<real>& a, cudaStream_t st) {
  if (a.B == 0) return cudaSuccess;
  const int w = a.d == 5 ? 8 : a.d;  // lanes per sequence
  const unsigned g = grid_for(a.B * w, 128);
  switch (a.d) {
    case 1: k_lle<real, 1><<<g, 128, 0, st>>>(a); break;
    case 2: k_lle<real, 2><<<g, 128, 0, st>>>(a); break;
    case 4: k_lle<real, 4><<<g, 128, 0, st>>>(a); break;
    case 5: k_lle<real, 5><<<g, 128, 0, st>>>(a); break;
    case 8: k_lle<real, 8><<<g, 128, 0, st>>>(a); break;
    case 16: k_lle<real, 16><<<g, 128, 0, st>>>(a); break;
    case 32: k_lle<real, 32><<<g, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_lle<float>(const LleArgs<float>&, cudaStream_t);
template cudaError_t launch_lle<double>(const LleArgs<double>&, cudaStream_t);

}  // namespace deer
