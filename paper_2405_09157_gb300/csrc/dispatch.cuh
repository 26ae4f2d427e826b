// Shape dispatch shared by the point-pass kernels: picks lanes-per-point and
// chunks-per-lane for a dimension d (see the table in shape_for()).
#pragma once

#include "common.cuh"

namespace pdscp {

// Launch of a pass kernel; pdl: with programmatic stream serialization, so
// that it may start while the previous launch in the stream finishes (the
// kernel waits for that launch in pdl_wait before it reads its results).
template <typename Kern, typename P>
cudaError_t launch_pass(Kern kern, int grid, int block, size_t smem, cudaStream_t stream, bool pdl, const P& q) {
  if (!pdl) {
    kern<<<grid, block, smem, stream>>>(q);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned int)grid);
  cfg.blockDim = dim3((unsigned int)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, q);
}

// Launch configuration of one kernel instance on the current device.
struct LaunchCfg {
  int grid;
  size_t smem;
  cudaStream_t stream;
};

int device_sm_count();
pdscp_status report_error(pdscp_status s, const char* msg);  // sets pdscp_last_error()

// Calls L.template go<VW, LPP, NCH>() for the instance that serves d.
// vec: rows start on 16-byte boundaries and hold a whole number of 16-byte
// chunks of VWV elements (VWV = 4 for float32, 8 for bfloat16).
//   vector path: nch = d / VWV chunks per row; lanes per point = the next
//     power of two >= nch up to 32, then 2, 4 or 8 chunks per lane;
//   scalar path: one element per chunk; 2, 8 or 32 lanes per point, then up
//     to 32 elements per lane.
template <int VWV, typename L>
cudaError_t dispatch_shape(int d, bool vec, L&& l) {
  if (vec) {
    const int nch = d / VWV;
    if (nch <= 1) return l.template go<VWV, 1, 1>();
    if (nch <= 2) return l.template go<VWV, 2, 1>();
    if (nch <= 4) return l.template go<VWV, 4, 1>();
    if (nch <= 8) return l.template go<VWV, 8, 1>();
    if (nch <= 16) return l.template go<VWV, 16, 1>();
    if (nch <= 32) return l.template go<VWV, 32, 1>();
    if (nch <= 64) return l.template go<VWV, 32, 2>();
    if (nch <= 128) return l.template go<VWV, 32, 4>();
    if (nch <= 256) return l.template go<VWV, 32, 8>();
    return cudaErrorInvalidValue;
  }
  if (d <= 2) return l.template go<1, 2, 1>();
  if (d <= 8) return l.template go<1, 8, 1>();
  if (d <= 32) return l.template go<1, 32, 1>();
  if (d <= 64) return l.template go<1, 32, 2>();
  if (d <= 128) return l.template go<1, 32, 4>();
  if (d <= 256) return l.template go<1, 32, 8>();
  if (d <= 512) return l.template go<1, 32, 16>();
  if (d <= 1024) return l.template go<1, 32, 32>();
  return cudaErrorInvalidValue;
}

// Threads per CTA of the reduce-scatter kernels: one CTA per SM, as many
// warps as the register file allows at the instance's register use (rounds
// of up to 32 point floats per lane fit 85 registers, 64 floats 128).
template <int VW, int NI>
struct PassBlock {
  static constexpr int value = (VW * NI <= 32) ? 768 : 512;
};

// Staged pass kernels: rounds of kRoundPoints 16-byte chunks per lane (4 KB
// per warp), and as many slots per warp as fit 192 KB of shared memory beside
// the kernels' static shared memory (768 threads: 2, 512 threads: 3).
template <int BLOCK>
struct StagedSlots {
  static constexpr int kRoundPoints = 8;
  static constexpr int value = BLOCK >= 768 ? 2 : 3;
  static constexpr size_t slot_bytes(int chunk_bytes, int ni) { return (size_t)32 * ni * chunk_bytes; }
  static_assert((size_t)(BLOCK / 32) * value * 32 * kRoundPoints * 16 <= 192 * 1024, "ring exceeds 192 KB");
};

// Try limit of the staged kernels' waits for their bulk copies: kWaitLimit,
// or PDSCP_WAIT_LIMIT from the environment (read at each launch; a small
// value lets a test make the wait give up and check the reported status).
unsigned int wait_limit();

// Points in flight per lane group, by the number of floats a lane holds.
template <int VW, int NCH>
struct Unroll {
  static constexpr int value = (VW * NCH <= 8) ? 4 : ((VW * NCH <= 16) ? 2 : 1);
};

// Opts a kernel in to `dyn` bytes of dynamic shared memory when that, plus
// the kernel's static shared memory, exceeds the default per-block limit of
// 48 KB (the launch fails with an invalid argument otherwise).
template <typename KernelFn>
cudaError_t allow_smem(KernelFn kern, size_t dyn) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kern);
  if (e != cudaSuccess) return e;
  if (dyn + a.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

// Grid for a point pass: enough CTAs to fill every SM at the occupancy the
// instance allows (at most kMaxBlocksPerSM per SM), no more than the work needs.
template <typename KernelFn>
int pass_grid(KernelFn kern, size_t smem, int64_t n, int points_per_cta_step, int block = kBlock) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess || occ < 1) occ = 1;
  if (occ > kMaxBlocksPerSM) occ = kMaxBlocksPerSM;
  const int64_t full = (int64_t)device_sm_count() * occ;
  int64_t need = (n + points_per_cta_step - 1) / points_per_cta_step;
  if (need < 1) need = 1;
  return (int)(need < full ? need : full);
}

}  // namespace pdscp
