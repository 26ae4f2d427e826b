// Instances and launches of the reverse-sweep kernels: float32 points here,
// bfloat16 points in kern_bwd_bf16.cu; the entry points pick by dtype.
#include "bwd_launch.cuh"

namespace pdscp {

extern template cudaError_t launch_ses_bwd_seed_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t);
extern template cudaError_t launch_ses_bwd_step_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t, bool);
extern template cudaError_t launch_svm_bwd_seed_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t);
extern template cudaError_t launch_svm_bwd_step_t<__nv_bfloat16>(const BwdParams&, bool, cudaStream_t, bool);

cudaError_t launch_ses_bwd_seed(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream) {
  return bf16 ? launch_ses_bwd_seed_t<__nv_bfloat16>(p, vec, stream) : launch_ses_bwd_seed_t<float>(p, vec, stream);
}
cudaError_t launch_ses_bwd_step(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream, bool pdl) {
  return bf16 ? launch_ses_bwd_step_t<__nv_bfloat16>(p, vec, stream, pdl)
              : launch_ses_bwd_step_t<float>(p, vec, stream, pdl);
}
cudaError_t launch_svm_bwd_seed(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream) {
  return bf16 ? launch_svm_bwd_seed_t<__nv_bfloat16>(p, vec, stream) : launch_svm_bwd_seed_t<float>(p, vec, stream);
}
cudaError_t launch_svm_bwd_step(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream, bool pdl) {
  return bf16 ? launch_svm_bwd_step_t<__nv_bfloat16>(p, vec, stream, pdl)
              : launch_svm_bwd_step_t<float>(p, vec, stream, pdl);
}

}  // namespace pdscp
