// Instances and launches of the SES reverse-sweep kernels (float32 points).
#include "bwd_kernel.cuh"
#include "dispatch.cuh"

namespace pdscp {

namespace {
struct BwdStepLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  bool pdl;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    if constexpr (VW > 1 && NCH == 1) {  // 16-byte chunk rows: the reduce-scatter form
      constexpr int NI = RoundSize<VW, LPP>::value < 8 ? RoundSize<VW, LPP>::value : 8;
      return run(ses_bwd_step_t_kernel<VW, LPP, NI>, (32 / LPP) * NI * kWarps);
    } else {
      constexpr int U = Unroll<VW, NCH>::value;
      return run(ses_bwd_step_kernel<VW, LPP, NCH, U>, (32 / LPP) * U * kWarps);
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

struct BwdArgmaxLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  int* grid_out;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    constexpr int U = Unroll<VW, NCH>::value;
    auto kern = ses_bwd_argmax_kernel<VW, LPP, NCH, U>;
    int grid = pass_grid(kern, 0, p.n, (32 / LPP) * U * kWarps);
    if (grid > p.ncand) grid = p.ncand;
    *grid_out = grid;
    kern<<<grid, kBlock, 0, stream>>>(p);
    return cudaGetLastError();
  }
};
struct SvmBwdStepLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  bool pdl;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    if constexpr (VW > 1 && NCH == 1) {  // 16-byte chunk rows: the reduce-scatter form
      constexpr int NI = RoundSize<VW, LPP>::value < 8 ? RoundSize<VW, LPP>::value : 8;
      return run(svm_bwd_step_t_kernel<VW, LPP, NI>, (32 / LPP) * NI * kWarps);
    } else {
      constexpr int U = Unroll<VW, NCH>::value;
      return run(svm_bwd_step_kernel<VW, LPP, NCH, U>, (32 / LPP) * U * kWarps);
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

struct SvmBwdArgLauncher {
  const BwdParams& p;
  cudaStream_t stream;
  int* grid_out;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    constexpr int U = Unroll<VW, NCH>::value;
    auto kern = svm_bwd_argmax_kernel<VW, LPP, NCH, U>;
    int grid = pass_grid(kern, 0, p.n, (32 / LPP) * U * kWarps);
    if (grid > p.ncand) grid = p.ncand;
    *grid_out = grid;
    kern<<<grid, kBlock, 0, stream>>>(p);
    return cudaGetLastError();
  }
};
}  // namespace

// SVM: the min/max pass and the seed (B = dL/dwbar^T, step T-1's bookkeeping).
cudaError_t launch_svm_bwd_seed(const BwdParams& p, bool vec, cudaStream_t stream) {
  int grid = 0;
  cudaError_t e = dispatch_shape<4>(p.d, vec, SvmBwdArgLauncher{p, stream, &grid});
  if (e != cudaSuccess) return e;
  BwdParams q = p;
  q.ncand = grid;
  svm_bwd_seed_kernel<0><<<1, 32, 0, stream>>>(q);
  return cudaGetLastError();
}

// SVM reverse step p.s (>= 0).
cudaError_t launch_svm_bwd_step(const BwdParams& p, bool vec, cudaStream_t stream, bool pdl) {
  return dispatch_shape<4>(p.d, vec, SvmBwdStepLauncher{p, stream, pdl});
}

// The argmax pass and the seed (B = dL/dubar^T, step T-1's bookkeeping).
cudaError_t launch_ses_bwd_seed(const BwdParams& p, bool vec, cudaStream_t stream) {
  int grid = 0;
  cudaError_t e = dispatch_shape<4>(p.d, vec, BwdArgmaxLauncher{p, stream, &grid});
  if (e != cudaSuccess) return e;
  BwdParams q = p;
  q.ncand = grid;
  ses_bwd_seed_kernel<0><<<1, 32, 0, stream>>>(q);
  return cudaGetLastError();
}

// Reverse step p.s (>= 1).
cudaError_t launch_ses_bwd_step(const BwdParams& p, bool vec, cudaStream_t stream, bool pdl) {
  return dispatch_shape<4>(p.d, vec, BwdStepLauncher{p, stream, pdl});
}

}  // namespace pdscp
