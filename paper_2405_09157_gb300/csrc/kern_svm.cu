// Instances of the SVM iteration kernel (float32 and bfloat16 points).
#include "dispatch.cuh"
#include "svm_kernel.cuh"

namespace pdscp {

namespace {
template <typename T>
struct SvmLauncher {
  const SvmParams& p;
  cudaStream_t stream;
  template <typename Kern>
  cudaError_t launch(Kern kern, int points_per_lane_step, int lpp) {
    const int dp = dpad4(p.d);
    size_t smem = (size_t)kWarps * 2 * dp * sizeof(float);
    const size_t fin = (size_t)(svm_partial_stride(p.d) + dp) * sizeof(double);
    if (fin > smem) smem = fin;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    const int grid = pass_grid(kern, smem, p.n, (32 / lpp) * points_per_lane_step * kWarps);
    kern<<<grid, kBlock, smem, stream>>>(p);
    return cudaGetLastError();
  }
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    if constexpr (VW > 1 && NCH == 1) {
      // vector rows of at most 32 chunks: the reduce-scatter form
      constexpr int NI = RoundSize<VW, LPP>::value;
      return launch(svm_iter_t_kernel<T, VW, LPP, NI>, NI, LPP);
    } else {
      constexpr int U = Unroll<VW, NCH>::value;
      return launch(svm_iter_kernel<T, VW, LPP, NCH, U>, U, LPP);
    }
  }
};
}  // namespace

cudaError_t launch_svm(const SvmParams& p, int dtype, bool vec, cudaStream_t stream) {
  if (dtype == PDSCP_F32) return dispatch_shape<4>(p.d, vec, SvmLauncher<float>{p, stream});
  return dispatch_shape<8>(p.d, vec, SvmLauncher<__nv_bfloat16>{p, stream});
}

}  // namespace pdscp
