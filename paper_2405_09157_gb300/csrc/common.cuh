// Shared device helpers of the MWU kernels: point loaders, warp/group/block
// reductions, the device state header and the workspace layout.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/pdscp.h"

namespace pdscp {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr int kBlock = 256;           // threads per CTA of the point passes
constexpr int kWarps = kBlock / 32;
constexpr int kMaxBlocksPerSM = 8;    // upper bound used to size the workspace
constexpr size_t kHeadBytes = 256;    // workspace: completion counter + flags

// ---------------------------------------------------------------------------
// Device state of one alpha-FTP. 128-byte header, then the running mean in
// FP64 (master copy), its FP32 copy read by the point pass, and the best point.
// ---------------------------------------------------------------------------
struct StateHdr {
  int64_t t;        // completed ORACLE calls
  int32_t stopped;  // alpha-FTP ended (separation or a Sec. 5 rule)
  int32_t outcome;  // PDSCP_OUT_*
  int32_t status;   // pdscp_status of the device computation
  int32_t rules;    // PDSCP_RULES_*
  int32_t streak;   // consecutive |df|/f < delta (Sec. 5)
  int32_t patience;
  double delta;
  double hint;      // SES: max_{i>=2} dist_i + gamma_i at the mean read last;
                    // SVM: min_i margin_i at the mean read last
  double move;      // SES: ||ubar^t - ubar^{t-1}||; SVM: D||dw|| + max|ds|
  double f_prev;    // previous f (-1: none yet)
  double best_f;    // SES: smallest f seen; SVM: largest margin seen
  double lb_best;   // SES: best primal lower bound
  double ub_best;   // SVM: best Claim 10 upper bound
  double s1bar;     // SVM running means of s_1, s_2
  double s2bar;
  double last_value;
  double reserved[2];
};
static_assert(sizeof(StateHdr) == 128, "state header must be 128 bytes");

__host__ __device__ inline int dpad4(int d) { return (d + 3) & ~3; }

__host__ __device__ inline size_t state_bytes(int d) {
  // header | double mean[dp] | float mean32[dp] | float best[dp]
  const int dp = dpad4(d);
  return sizeof(StateHdr) + (size_t)dp * 8 + (size_t)dp * 4 * 2;
}
__host__ __device__ inline double* state_mean(void* s) {
  return reinterpret_cast<double*>(reinterpret_cast<char*>(s) + sizeof(StateHdr));
}
__host__ __device__ inline float* state_mean32(void* s, int d) {
  return reinterpret_cast<float*>(reinterpret_cast<char*>(s) + sizeof(StateHdr) + (size_t)dpad4(d) * 8);
}
__host__ __device__ inline float* state_best(void* s, int d) {
  return state_mean32(s, d) + dpad4(d);
}

// Per-CTA partial row width (floats).
__host__ __device__ inline int ses_partial_stride(int d) { return 4 + dpad4(d); }
__host__ __device__ inline int svm_partial_stride(int d) { return 4 + 2 * dpad4(d); }

// ---------------------------------------------------------------------------
// Point loaders: one "chunk" is VW consecutive elements of a row, converted
// to float. The 16-byte forms require an aligned row start.
// ---------------------------------------------------------------------------
template <typename T, int VW>
struct Chunk;

template <>
struct Chunk<float, 4> {
  static __device__ __forceinline__ void load(const float* row, int c, float* o) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(row) + c);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct Chunk<float, 1> {
  static __device__ __forceinline__ void load(const float* row, int c, float* o) { o[0] = __ldg(row + c); }
};
template <>
struct Chunk<__nv_bfloat16, 8> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* row, int c, float* o) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + c);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // bf16 -> fp32 is a 16-bit left shift of the bit pattern
      o[2 * j] = __uint_as_float(w[j] << 16);
      o[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
    }
  }
};
template <>
struct Chunk<__nv_bfloat16, 1> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* row, int c, float* o) {
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(row) + c);
    o[0] = __uint_as_float(((uint32_t)b) << 16);
  }
};

template <typename T>
__device__ __forceinline__ float elem_to_float(const T* p);
template <>
__device__ __forceinline__ float elem_to_float<float>(const float* p) { return *p; }
template <>
__device__ __forceinline__ float elem_to_float<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __uint_as_float(((uint32_t) * reinterpret_cast<const unsigned short*>(p)) << 16);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <int LPP>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = LPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one double per thread over the whole block; every thread gets the
// total. `red` is shared scratch of at least 32 doubles. Contains barriers:
// every thread of the block must call it.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];  // fixed order: deterministic
  return s;
}

// Completion counter: the CTA whose arrival is the last one runs the O(d)
// finalize. Returns true in every thread of that CTA. The writes of the
// partial row must precede the call.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, bool* flag_smem) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    *flag_smem = (prev == gridDim.x - 1);
  }
  __syncthreads();
  const bool last = *flag_smem;
  if (last) __threadfence();
  return last;
}

}  // namespace pdscp
