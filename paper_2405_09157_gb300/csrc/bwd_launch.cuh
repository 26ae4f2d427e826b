// Launchers of the reverse-sweep kernels for one point type T, instantiated
// by kern_bwd.cu (float) and kern_bwd_bf16.cu (bfloat16) so that the two
// compile in parallel.
#pragma once

#include "bwd_kernel.cuh"
#include "dispatch.cuh"

namespace pdscp {

namespace bwd_detail {
template <typename T>
struct BwdStepLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  bool pdl;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    if constexpr (VW > 1 && NCH == 1) {  // rows of one 4-element chunk per lane: the reduce-scatter form
      constexpr int NI = RoundSize<VW, LPP>::value < 8 ? RoundSize<VW, LPP>::value : 8;
      return run(ses_bwd_step_t_kernel<T, VW, LPP, NI>, (32 / LPP) * NI * kWarps);
    } else {
      constexpr int U = Unroll<VW, NCH>::value;
      return run(ses_bwd_step_kernel<T, VW, LPP, NCH, U>, (32 / LPP) * U * kWarps);
    }
  }
  template <typename Kern>
  cudaError_t run(Kern kern, int per_step) {
    const int dp = dpad4(p.d);
    const int st = ses_partial_stride(p.d);
    const size_t pass_smem = (size_t)kWarps * dp * sizeof(float);
    const size_t fin_base = (size_t)st * sizeof(float2);
    size_t smem = pass_smem > fin_base ? pass_smem : fin_base;
    int grid = pass_grid(kern, smem, p.n, per_step);
    BwdParams q = p;
    q.single = single_level(grid, st, kStageBytesManyCta) ? 1 : 0;
    if (q.single) {
      const size_t fin = fin_base + (size_t)grid * st * sizeof(float);
      if (fin > smem) smem = fin;
    }
    {
      cudaError_t e = allow_smem(kern, smem);
      if (e != cudaSuccess) return e;
    }
    return launch_pass(kern, grid, kBlock, smem, stream, pdl, q);
  }
};

template <typename T>
struct BwdArgmaxLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  int* grid_out;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    constexpr int U = Unroll<VW, NCH>::value;
    auto kern = ses_bwd_argmax_kernel<T, VW, LPP, NCH, U>;
    int grid = pass_grid(kern, 0, p.n, (32 / LPP) * U * kWarps);
    if (grid > p.ncand) grid = p.ncand;
    *grid_out = grid;
    kern<<<grid, kBlock, 0, stream>>>(p);
    return cudaGetLastError();
  }
};
template <typename T>
struct SvmBwdStepLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  bool pdl;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    if constexpr (VW > 1 && NCH == 1) {  // rows of one 4-element chunk per lane: the reduce-scatter form
      constexpr int NI = RoundSize<VW, LPP>::value < 8 ? RoundSize<VW, LPP>::value : 8;
      return run(svm_bwd_step_t_kernel<T, VW, LPP, NI>, (32 / LPP) * NI * kWarps);
    } else {
      constexpr int U = Unroll<VW, NCH>::value;
      return run(svm_bwd_step_kernel<T, VW, LPP, NCH, U>, (32 / LPP) * U * kWarps);
    }
  }
  template <typename Kern>
  cudaError_t run(Kern kern, int per_step) {
    const int dp = dpad4(p.d);
    const int st = ses_partial_stride(p.d);
    const size_t pass_smem = (size_t)kWarps * dp * sizeof(float);
    const size_t fin_base = (size_t)st * sizeof(float2);
    size_t smem = pass_smem > fin_base ? pass_smem : fin_base;
    int grid = pass_grid(kern, smem, p.n, per_step);
    BwdParams q = p;
    q.single = single_level(grid, st, kStageBytesManyCta) ? 1 : 0;
    if (q.single) {
      const size_t fin = fin_base + (size_t)grid * st * sizeof(float);
      if (fin > smem) smem = fin;
    }
    cudaError_t e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    return launch_pass(kern, grid, kBlock, smem, stream, pdl, q);
  }
};

template <typename T>
struct SvmBwdArgLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  int* grid_out;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    constexpr int U = Unroll<VW, NCH>::value;
    auto kern = svm_bwd_argmax_kernel<T, VW, LPP, NCH, U>;
    int grid = pass_grid(kern, 0, p.n, (32 / LPP) * U * kWarps);
    if (grid > p.ncand) grid = p.ncand;
    *grid_out = grid;
    kern<<<grid, kBlock, 0, stream>>>(p);
    return cudaGetLastError();
  }
};
}  // namespace bwd_detail

// SES: the argmax pass and the seed (B = dL/dubar^T, step T-1's bookkeeping).
template <typename T>
cudaError_t launch_ses_bwd_seed_t(const BwdParams& p, bool vec, cudaStream_t stream) {
  int grid = 0;
  cudaError_t e = dispatch_shape<4>(p.d, vec, bwd_detail::BwdArgmaxLauncher<T>{p, stream, &grid});
  if (e != cudaSuccess) return e;
  BwdParams q = p;
  q.ncand = grid;
  ses_bwd_seed_kernel<T><<<1, 32, 0, stream>>>(q);
  return cudaGetLastError();
}

// SES reverse step p.s (>= 1).
template <typename T>
cudaError_t launch_ses_bwd_step_t(const BwdParams& p, bool vec, cudaStream_t stream, bool pdl) {
  return dispatch_shape<4>(p.d, vec, bwd_detail::BwdStepLauncher<T>{p, stream, pdl});
}

// SVM: the min/max pass and the seed (B = dL/dwbar^T, step T-1's bookkeeping).
template <typename T>
cudaError_t launch_svm_bwd_seed_t(const BwdParams& p, bool vec, cudaStream_t stream) {
  int grid = 0;
  cudaError_t e = dispatch_shape<4>(p.d, vec, bwd_detail::SvmBwdArgLauncher<T>{p, stream, &grid});
  if (e != cudaSuccess) return e;
  BwdParams q = p;
  q.ncand = grid;
  svm_bwd_seed_kernel<T><<<1, 32, 0, stream>>>(q);
  return cudaGetLastError();
}

// SVM reverse step p.s (>= 0).
template <typename T>
cudaError_t launch_svm_bwd_step_t(const BwdParams& p, bool vec, cudaStream_t stream, bool pdl) {
  return dispatch_shape<4>(p.d, vec, bwd_detail::SvmBwdStepLauncher<T>{p, stream, pdl});
}

}  // namespace pdscp
