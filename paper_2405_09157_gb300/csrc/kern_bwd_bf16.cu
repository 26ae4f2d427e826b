// Instances of the reverse-sweep kernels for bfloat16 points (widened to
// float32 on load; the gradient is float32).
#include "bwd_launch.cuh"

namespace pdscp {

template cudaError_t launch_ses_bwd_seed_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t);
template cudaError_t launch_ses_bwd_step_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t, bool);
template cudaError_t launch_svm_bwd_seed_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t);
template cudaError_t launch_svm_bwd_step_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t, bool);

}  // namespace pdscp
