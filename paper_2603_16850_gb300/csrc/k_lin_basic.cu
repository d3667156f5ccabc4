// Generic-kernel launchers (initial guess, linearisation + residual, sequential rollout) of
// the Brusselator, the GRU and the affine recurrence.
#include "lin_generic.cuh"

namespace deer {

template <class real>
cudaError_t launch_init_basic(const InitArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_BRUSSELATOR_EULER: return generic_init<real, DEER_F_BRUSSELATOR_EULER>(a, st);
    case DEER_F_GRU: return generic_init<real, DEER_F_GRU>(a, st);
    case DEER_F_LINEAR: return generic_init<real, DEER_F_LINEAR>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <class real>
cudaError_t launch_linearize_basic(const LinArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_BRUSSELATOR_EULER:
      return generic_linearize<real, DEER_F_BRUSSELATOR_EULER>(a, st);
    case DEER_F_GRU: return generic_linearize<real, DEER_F_GRU>(a, st);
    case DEER_F_LINEAR: return generic_linearize<real, DEER_F_LINEAR>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <class real>
cudaError_t launch_rollout_basic(const RolloutArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_BRUSSELATOR_EULER:
      return generic_rollout<real, DEER_F_BRUSSELATOR_EULER>(a, st);
    case DEER_F_GRU: return generic_rollout<real, DEER_F_GRU>(a, st);
    case DEER_F_LINEAR: return generic_rollout<real, DEER_F_LINEAR>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_init_basic<float>(const InitArgs<float>&, cudaStream_t);
template cudaError_t launch_init_basic<double>(const InitArgs<double>&, cudaStream_t);
template cudaError_t launch_linearize_basic<float>(const LinArgs<float>&, cudaStream_t);
template cudaError_t launch_linearize_basic<double>(const LinArgs<double>&, cudaStream_t);
template cudaError_t launch_rollout_basic<float>(const RolloutArgs<float>&, cudaStream_t);
template cudaError_t launch_rollout_basic<double>(const RolloutArgs<double>&, cudaStream_t);

template <class real>
cudaError_t launch_input_grad_basic(const InputGradArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_GRU: return generic_input_grad<real, DEER_F_GRU>(a, st);
    case DEER_F_LINEAR: return generic_input_grad<real, DEER_F_LINEAR>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_input_grad_basic<float>(const InputGradArgs<float>&, cudaStream_t);
template cudaError_t launch_input_grad_basic<double>(const InputGradArgs<double>&, cudaStream_t);

}  // namespace deer
