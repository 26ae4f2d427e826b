// Instances of the SVM iteration kernel (float32 and bfloat16 points).
#include "dispatch.cuh"
#include "svm_kernel.cuh"

namespace pdscp {

namespace {
template <typename T>
struct SvmLauncher {
  const SvmParams& p;
  cudaStream_t stream;
  bool pdl;
  // Dynamic shared memory: the per-warp partial sums of the pass, or in the
  // finishing CTA the column totals, the mean and (single-level
  // completion) every partial row, whichever is larger.
  template <typename Kern>
  cudaError_t launch(Kern kern, int points_per_lane_step, int lpp, int block, size_t ring_bytes = 0) {
    const int dp = dpad4(p.d);
    const int st = svm_partial_stride(p.d);
    size_t pass_smem = (size_t)(block / 32) * 2 * dp * sizeof(float);
    if (ring_bytes > pass_smem) pass_smem = ring_bytes;
    const size_t fin_base = (size_t)(st + 2 * dp) * sizeof(double);  // totals | mean | zbar
    size_t smem = pass_smem > fin_base ? pass_smem : fin_base;
    int grid = pass_grid(kern, smem, p.n, (32 / lpp) * points_per_lane_step * (block / 32), block);
    SvmParams q = p;
    q.wait_limit = wait_limit();
    // Rows that fit the staging area complete by one staged reduction in the
    // last CTA; wider rows that fit the workspace head's accumulators complete
    // through them (fixed point), the rest in two levels. Measured on GB300:
    // the staged reduction beats the accumulators for SES rows at d = 32
    // (35.5 against 37.5 us per iteration, n = 1e6), the accumulators beat
    // the two-level reduction for SVM rows at d = 128 (95.6 against 102.7 us).
    q.single = single_level(grid, st, block >= 512 ? kStageBytesOneCta : kStageBytesManyCta) ? 1 : 0;
    q.fx = (!q.single && st <= kFxMaxCols) ? 1 : 0;
    if (q.single) {
      const size_t fin = fin_base + (size_t)grid * st * sizeof(float);
      if (fin > smem) smem = fin;
      // the staging area may lower the CTAs per SM: keep the grid to one wave
      {
        cudaError_t e = allow_smem(kern, smem);
        if (e != cudaSuccess) return e;
      }
      const int g1 = pass_grid(kern, smem, p.n, (32 / lpp) * points_per_lane_step * (block / 32), block);
      if (g1 < grid) grid = g1;
    }
    {
      cudaError_t e = allow_smem(kern, smem);
      if (e != cudaSuccess) return e;
    }
    return launch_pass(kern, grid, block, smem, stream, pdl, q);
  }
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    if constexpr (VW > 1 && NCH == 1) {
      // vector rows of at most 32 chunks: the reduce-scatter form
      if constexpr (sizeof(T) == 2) {
        // bfloat16 rows: staged rounds of 8 points per lane group (4 KB per
        // slot), 512 threads (measured at n = 1e6, d = 128: 69.5 -> 56.4 us)
        constexpr int NI = StagedSlots<768>::kRoundPoints;
        constexpr int B = 512;
        constexpr int NS = StagedSlots<B>::value;
        return launch(svm_iter_t_kernel<T, VW, LPP, NI, B, NS>, NI, LPP, B,
                      (size_t)(B / 32) * NS * StagedSlots<B>::slot_bytes(VW * (int)sizeof(T), NI));
      } else {
        // float32 rows: rounds loaded into registers (staged at 512 threads
        // measured 91.6 against 88.3 us at n = 1e6, d = 128; at 768 threads
        // the staged kernel spills)
        constexpr int NI = RoundSize<VW, LPP>::value;
        constexpr int B = PassBlock<VW, NI>::value;
        return launch(svm_iter_t_kernel<T, VW, LPP, NI, B, 0>, NI, LPP, B);
      }
    } else {
      constexpr int U = Unroll<VW, NCH>::value;
      return launch(svm_iter_kernel<T, VW, LPP, NCH, U>, U, LPP, kBlock);
    }
  }
};
}  // namespace

cudaError_t launch_svm(const SvmParams& p, int dtype, bool vec, cudaStream_t stream, bool pdl) {
  if (dtype == PDSCP_F32) return dispatch_shape<4>(p.d, vec, SvmLauncher<float>{p, stream, pdl});
  return dispatch_shape<8>(p.d, vec, SvmLauncher<__nv_bfloat16>{p, stream, pdl});
}

cudaError_t launch_svm_merge(const SvmMergeParams& m, cudaStream_t stream) {
  const size_t smem = (size_t)(svm_partial_stride(m.d) + 2 * dpad4(m.d)) * sizeof(double);
  svm_merge_kernel<0><<<1, kSvmMergeBlock, smem, stream>>>(m);
  return cudaGetLastError();
}

}  // namespace pdscp
