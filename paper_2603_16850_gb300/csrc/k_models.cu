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

template <class real>
cudaError_t launch_linearize_models(const LinArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_RNN_TANH:
      return generic_linearize<real, DEER_F_RNN_TANH>(a, st);
    case DEER_F_LANGEVIN_2WELL: return generic_linearize<real, DEER_F_LANGEVIN_2WELL>(a, st);
    case DEER_F_LORENZ96_DP5: return generic_linearize<real, DEER_F_LORENZ96_DP5>(a, st);
    case DEER_F_PERMUTE: return generic_linearize<real, DEER_F_PERMUTE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <class real>
cudaError_t launch_rollout_models(const RolloutArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_RNN_TANH:
      return generic_rollout<real, DEER_F_RNN_TANH>(a, st);
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

}  // namespace deer
