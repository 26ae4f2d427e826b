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
constexpr int kMaxBlock = 1024;       // largest CTA of any pass kernel
constexpr int kMaxBlocksPerSM = 8;    // upper bound used to size the workspace
// Completion stages every partial row in the last CTA's shared memory when
// they fit in this many bytes (kernels with one CTA per SM can spare much
// more shared memory than those with several; rows much wider than 128
// floats reduce faster through the two-level path); larger rows take the
// two-level completion.
constexpr size_t kStageBytesOneCta = 96 * 1024;
constexpr size_t kStageBytesManyCta = 48 * 1024;
// Workspace head (zeroed by mwu_state_init and left zeroed by every pass):
// [0, 1 KB) completion counters (top + per group) | [kFxFlagOff] overflow flag
// of the fixed-point completion | [kFxOff, kHeadBytes) its column accumulators.
constexpr size_t kHeadBytes = 16384;
constexpr size_t kFxFlagOff = 1024;
constexpr size_t kFxOff = 2048;
constexpr int kFxMaxCols = (int)((kHeadBytes - kFxOff) / 16);  // two 64-bit words per column
constexpr int kMaxGroups = 64;        // group rows reserved in the workspace

// ---------------------------------------------------------------------------
// Device state of one alpha-FTP. 128-byte header, then the running mean in
// FP64 (master copy), its FP32 copy read by the point pass, the best point,
// and the running average of the dual weights' d-vector (FP64: SES B-bar of
// the QP bound, SVM z-bar of the Claim 8 bound).
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
  double ub_best;   // SVM: best Claim 8 upper bound
  double s1bar;     // SVM running means of s_1, s_2
  double s2bar;
  double last_value;
  double dual_A;    // SES: running average A-bar of the QP bound
  double dual_w;    // sum of the averaging weights so far (iterate t has weight t^2)
};
static_assert(sizeof(StateHdr) == 128, "state header must be 128 bytes");

__host__ __device__ inline int dpad4(int d) { return (d + 3) & ~3; }

// k / sqrt2 = eta t / (rho sqrt2) of an SES pass, in FP32 (the pass kernels,
// the tape of the reverse sweep and the multi-candidate and batched passes use
// this one expression). Multiplies by 1/sqrt2 rather than dividing by sqrt2:
// FP64 division takes hundreds of cycles on this GPU, on every CTA's start.
constexpr double kRsqrt2 = 0.70710678118654752440;
__host__ __device__ inline float ses_kr(int64_t t, double eta_over_rho) {
  return (float)((double)t * eta_over_rho * kRsqrt2);
}

#ifdef __CUDACC__
// 8-byte global -> shared copy that holds no register while in flight (both
// addresses 8-byte aligned); completed by cp_async_wait_all() of the same thread.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned int)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// ---------------------------------------------------------------------------
// One-dimensional bulk copies (TMA, cp.async.bulk) global -> shared, completed
// on an mbarrier. Used by the staged pass kernels: each warp keeps a ring of
// slots in shared memory and copies its next rounds of points into it while it
// computes the current one. Addresses and sizes must be multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Makes initialised mbarriers visible to the async proxy (the bulk copies).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Orders this thread's earlier shared-memory accesses before later bulk copies
// into the same memory (a slot is refilled only after its data was read).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// L2 policy for data read once per pass: its lines are the first evicted, so
// a pass streaming more than L2 holds does not push out the lines the rest of
// the launch needs (the kernel's code, the state, the partial rows).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
// Copies `bytes` from global `src` to shared `dst`; the copy's completion
// flips the phase of `bar`, which expects exactly these bytes (one arrival).
// The source lines are read with the L2 evict-first policy (made here, at
// each copy: one instruction, and no register held across the caller's loop).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned int bytes, uint64_t* bar) {
  const uint64_t pol = l2_evict_first_policy();
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// Waits for the phase with parity `parity` of `bar` to complete, trying at
// most `limit` times (each try may suspend the thread for a short,
// hardware-chosen time). Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned int parity, unsigned int limit) {
  for (unsigned int it = 0; it < limit; ++it) {
    unsigned int done;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Default try limit of the staged kernels' waits (each try may suspend the
// thread for a hardware-chosen time; a copy of 4 KB completes within a few
// microseconds, so only a copy that never completes reaches the limit).
constexpr unsigned int kWaitLimit = 1u << 20;
// Workspace head word in which a staged pass records a wait that gave up
// (read and cleared by the finishing CTA, which then reports PDSCP_ERR_TIMEOUT).
constexpr size_t kTimeoutFlagOff = kFxFlagOff + 4;

// Device-scope acquire-release fence: the release half orders this CTA's
// earlier writes (made visible to this thread by the CTA barrier before it)
// before a following completion atomic, the acquire half orders the atomic
// before later reads of the other CTAs' writes. It is the weaker form of
// __threadfence(), which is sequentially consistent and costs more.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;\n" ::: "memory"); }
// Arrival on a completion counter in one instruction: an acquire-release
// atomic add (the release half orders this thread's earlier writes, and those
// the CTA barrier before it made visible to it, before the add; the acquire
// half orders the add before this thread's later reads). Returns the old value.
__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* a, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;\n" : "=r"(old) : "l"(a), "r"(v) : "memory");
  return old;
}
// Programmatic dependent launch: a pass kernel lets the next launch in the
// stream start early (pdl_trigger) and, in that next launch, waits for the
// previous grid's completion and memory (pdl_wait) before it reads anything
// the previous grid writes. Both are no-ops for a launch without the
// attribute. The wait is a hardware dependency, not a spin loop.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Paired FP32 arithmetic (two floats in one 64-bit register; one instruction
// for both lanes of the pair, each rounded as the scalar operation would be).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// a pair of bfloat16 values (low half first) widened to a pair of floats
__device__ __forceinline__ unsigned long long f2_from_bf16x2(uint32_t w) {
  return f2_pack(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
#endif

__host__ __device__ inline size_t state_bytes(int d) {
  // header | double mean[dp] | float mean32[dp] | float best[dp] | double dual[dp]
  const int dp = dpad4(d);
  return sizeof(StateHdr) + (size_t)dp * 8 * 2 + (size_t)dp * 4 * 2;
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
__host__ __device__ inline double* state_dual(void* s, int d) {
  return reinterpret_cast<double*>(state_best(s, d) + dpad4(d));
}

// Per-CTA partial row width (floats).
__host__ __device__ inline int ses_partial_stride(int d) { return 4 + dpad4(d); }
// One entry of the forward tape a reverse sweep reads (floats): S, |g|, k/sqrt2,
// the exponent shift, then the mean the pass read (dp) and g (dp).
__host__ __device__ inline int ses_tape_stride(int d) { return 4 + 2 * dpad4(d); }
// SVM tape entry (floats): S, |z|, k, the shift, s1bar, s2bar, 0, 0, then the
// mean the pass read (dp) and z (dp).
__host__ __device__ inline int svm_tape_stride(int d) { return 8 + 2 * dpad4(d); }

// Sink of the warm-up run of a finish (a scratch state, step record and tape
// entry that the run writes instead of the real ones): its size and parts.
__host__ __device__ inline size_t warm_sink_bytes(int d) {
  return ((state_bytes(d) + 255) & ~(size_t)255) + 256 + (size_t)svm_tape_stride(d) * sizeof(float);
}
__device__ __forceinline__ pdscp_step_out* warm_sink_out(unsigned char* sink, int d) {
  return reinterpret_cast<pdscp_step_out*>(sink + ((state_bytes(d) + 255) & ~(size_t)255));
}
__device__ __forceinline__ float* warm_sink_tape(unsigned char* sink, int d) {
  return reinterpret_cast<float*>(sink + ((state_bytes(d) + 255) & ~(size_t)255) + 256);
}

// Warp split of a pass: with warm-up warps (the last warp of each CTA, when a
// sink is given), the other warps take their share of the points.
struct WarpSplit {
  bool warm;
  int64_t gw, nwarps;
  __device__ WarpSplit(const void* sink, int nw, int warp) {
    const bool on = sink != nullptr && nw > 1;
    warm = on && warp == nw - 1;
    const int nws = on ? nw - 1 : nw;
    nwarps = (int64_t)gridDim.x * nws;
    gw = (int64_t)blockIdx.x * nws + warp;
  }
};
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

// Column operations of a partial row: 0 sum, 1 max, 2 min.
// Sums are carried as compensated FP32 pairs (s, c) (Neumaier's variant of
// Kahan summation): the error of a sum of m terms is about 2^-24 |sum| plus
// m 2^-48 sum|terms|, i.e. FP64-grade for these reductions, at FP32 speed
// (FP64 throughput on this GPU is ~1/64 of FP32).
__device__ __forceinline__ void neu_add(float& s, float& c, float v) {
  const float t = s + v;
  c += (fabsf(s) >= fabsf(v)) ? (s - t) + v : (v - t) + s;
  s = t;
}
__device__ __forceinline__ float2 col_init2(int op) {
  return make_float2(op == 0 ? 0.f : (op == 1 ? -INFINITY : INFINITY), 0.f);
}
__device__ __forceinline__ void col_comb2(int op, float2& a, float2 b) {
  if (op == 0) {
    neu_add(a.x, a.y, b.x);
    a.y += b.y;
  } else {
    a.x = op == 1 ? fmaxf(a.x, b.x) : fminf(a.x, b.x);
  }
}
__device__ __forceinline__ float2 as_pair(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ float2 as_pair(float2 v) { return v; }

// Column-wise reduction of rows [r0, r1) of a row-major (rows x stride)
// matrix of float or float2 pairs into out[0..stride) (float2 pairs), by
// every thread of the CTA. The rows are split R ways (R a power of two,
// R * stride <= blockDim) so each thread issues few loads, all independent;
// the R partial results are combined in a fixed order (deterministic).
// opof(pc) gives the operation of column pc. `scratch` holds blockDim
// float2. `ld` (> 0) is the row pitch when it differs from stride. The rows
// are read through L2 (other CTAs wrote them). Ends with a barrier; every
// thread must call it.

template <typename TIn, typename OpOf>
__device__ void reduce_rows(const TIn* m, int r0, int r1, int stride, float2* out, float2* scratch, OpOf opof,
                            int ld = 0) {
  const size_t pitch = ld > 0 ? (size_t)ld : (size_t)stride;  // row pitch; the first `stride` columns are reduced
  const int nt = blockDim.x;
  int R = 1;
  while (2 * R * stride <= nt && R < 32) R *= 2;
  if (R == 1) {
    for (int pc = threadIdx.x; pc < stride; pc += nt) {
      const int op = opof(pc);
      float2 acc = col_init2(op);
#pragma unroll 8
      for (int r = r0; r < r1; ++r) col_comb2(op, acc, as_pair(__ldcg(m + (size_t)r * pitch + pc)));
      out[pc] = acc;
    }
    __syncthreads();
    return;
  }
  const int t = threadIdx.x;
  if (t < R * stride) {
    const int pc = t % stride, q = t / stride;
    const int op = opof(pc);
    float2 acc = col_init2(op);
#pragma unroll 8
    for (int r = r0 + q; r < r1; r += R) col_comb2(op, acc, as_pair(__ldcg(m + (size_t)r * pitch + pc)));
    scratch[q * stride + pc] = acc;
  }
  __syncthreads();
  for (int pc = threadIdx.x; pc < stride; pc += nt) {
    const int op = opof(pc);
    float2 acc = scratch[pc];
    for (int q = 1; q < R; ++q) col_comb2(op, acc, scratch[q * stride + pc]);
    out[pc] = acc;
  }
  __syncthreads();
}

// Reciprocal and reciprocal square root in FP64 from the FP32 results
// refined by Newton's iteration (one step for 1/x: r <- r (2 - x r); one
// step for 1/sqrt(x): y <- y (3 - x y^2) / 2), each step squaring the
// relative error (2^-24 -> ~2^-47). Far cheaper than FP64 divide/sqrt on
// this GPU. x must be positive and within the FP32 range.
__device__ __forceinline__ double recip_d(double x) {
  const double r = (double)(1.0f / (float)x);
  return r * (2.0 - x * r);
}
__device__ __forceinline__ double rsqrt_d(double x) {
  const double y = (double)rsqrtf((float)x);
  return y * (1.5 - 0.5 * x * y * y);
}
__device__ __forceinline__ double sqrt_d(double x) { return x > 0.0 ? x * rsqrt_d(x) : 0.0; }

// CTAs per completion group for a grid of nb CTAs (about sqrt(nb)).
__host__ __device__ inline int group_size(int nb) {
  int g = 1;
  while (g * g < nb) ++g;
  return g;
}

// Two-level completion. Every CTA has written its partial row (stride
// floats) to rows[blockIdx.x]. CTA b belongs to group b / gs; the last CTA
// to arrive in a group reduces the group's rows into grows[group] (pairs),
// then arrives at the top counter. Returns true in exactly one CTA, the last
// group reducer to arrive, when every group row is complete. Counters are
// reset by their last arriver, so the workspace is ready for the next launch.
// No CTA waits for another: there is no spin anywhere.
template <typename OpOf>
__device__ bool arrive_two_level(const float* rows, int stride, float2* grows, unsigned int* counters,
                                 float2* scratch, bool* s_flag, OpOf opof) {
  const int nb = gridDim.x;
  const int gs = group_size(nb);
  const int g = blockIdx.x / gs;
  const int r0 = g * gs, r1 = min(nb, r0 + gs);
  // CTA barrier, then one thread's device-scope fence and atomic: the fence is
  // cumulative over the writes the barrier ordered before it.
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_acq_rel_gpu();
    const unsigned int prev = atomicAdd(&counters[1 + g], 1u);
    fence_acq_rel_gpu();
    *s_flag = (prev == (unsigned int)(r1 - r0 - 1));
  }
  __syncthreads();
  if (!*s_flag) return false;
  reduce_rows(rows, r0, r1, stride, grows + (size_t)g * stride, scratch, opof);  // ends with a barrier
  const int G = (nb + gs - 1) / gs;
  if (threadIdx.x == 0) {
    counters[1 + g] = 0u;
    fence_acq_rel_gpu();
    const unsigned int prev = atomicAdd(&counters[0], 1u);
    fence_acq_rel_gpu();
    *s_flag = (prev == (unsigned int)(G - 1));
  }
  __syncthreads();
  if (!*s_flag) return false;
  if (threadIdx.x == 0) counters[0] = 0u;
  return true;
}

// Two sums at once over the whole block (same barriers as block_sum_d).
__device__ __forceinline__ void block_sum2_d(double& a, double& b, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  __syncthreads();
  if (lane == 0) {
    red[warp] = a;
    red[16 + warp] = b;
  }
  __syncthreads();
  double sa = 0.0, sb = 0.0;
  for (int w = 0; w < nw; ++w) {
    sa += red[w];
    sb += red[16 + w];
  }
  a = sa;
  b = sb;
}

// Whether the completion of a grid of nb CTAs with partial rows of `stride`
// floats stages every row in shared memory (single level).
__host__ __device__ inline bool single_level(int nb, int stride, size_t limit) {
  return (size_t)nb * stride * sizeof(float) <= limit;
}

// Completion of one pass, in two calls. Every CTA has written its partial
// row (stride floats) to rows[blockIdx.x].
//   arrive_pass: returns true in exactly one CTA, the one that finishes;
//   final_reduce: in that CTA, the column totals of all rows into raw[0..stride)
//     as compensated pairs.
// Single level: the last CTA to arrive loads every row into shared memory
// `stage` with one round of independent 16-byte loads and reduces there.
// Two levels (rows too large to stage): arrive_two_level, then the group rows.
// Between the two calls the finishing CTA can issue its other loads so that
// their latency overlaps the staging. No CTA waits on another.
template <typename OpOf>
__device__ bool arrive_pass(const float* rows, int stride, float2* grows, unsigned int* counters, float2* scratch,
                            bool* s_flag, OpOf opof, bool single) {
  if (!single) return arrive_two_level(rows, stride, grows, counters, scratch, s_flag, opof);
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = (atom_add_acq_rel_gpu(&counters[0], 1u) == (unsigned int)(gridDim.x - 1));
  __syncthreads();
  return *s_flag;
}

// ---------------------------------------------------------------------------
// Fixed-point completion. Every CTA adds its partial row into per-column
// 64-bit integer accumulators in the workspace head (atomics, while the other
// CTAs still stream), so the finishing CTA reads one total per column instead
// of reducing every CTA's row. Integer addition is associative: the totals do
// not depend on the order in which CTAs arrive, and a run stays bit for bit
// reproducible. A column sum uses a scale 2^e fixed before the pass from a
// bound B on the column's absolute sum (identical in every CTA): a CTA's value
// v becomes X = v 2^e (exact in FP64), split into hi = floor(X) (signed) and
// lo = the next 32 bits of the fraction; with B 2^e < 2^51 the hi words of
// up to 2048 CTAs cannot overflow, and the total is exact to 2^-(e+32). A
// maximum (minimum) column takes an atomic maximum of an order-preserving
// integer image of v (of -v). A value outside its bound (or NaN) sets the
// overflow flag instead; the finishing CTA then reduces the CTAs' FP32 rows,
// which every CTA also writes, as before.
// ---------------------------------------------------------------------------
constexpr int kFxMaxBanks = 1;  // copies of the accumulators (see fx_cols)
struct FxCols {
  // bank b, column pc: acc[2 (b stride + pc)] = sum of hi (two's complement), acc[2 (b stride + pc) + 1] = sum of lo
  unsigned long long* acc;
  unsigned int* bad;
  int stride, banks;
};
// CTAs push into `banks` copies of the accumulators (CTA b into copy b mod
// banks; the finishing CTA adds the copies), so that fewer CTAs contend for
// one address: as many copies as the head holds, a power of two <= kFxMaxBanks.
__device__ __forceinline__ FxCols fx_cols(unsigned int* counter, int stride) {
  char* h = reinterpret_cast<char*>(counter);
  const int room = (int)((kHeadBytes - kFxOff) / (16 * (size_t)stride));
  int banks = 1;
  while (2 * banks <= room && 2 * banks <= kFxMaxBanks) banks *= 2;
  return FxCols{reinterpret_cast<unsigned long long*>(h + kFxOff), reinterpret_cast<unsigned int*>(h + kFxFlagOff),
                stride, banks};
}
// Scale exponent for a column whose absolute sum is at most `bound`.
__device__ __forceinline__ int fx_exp(double bound) {
  return 50 - ilogb(fmax(bound, 1e-30));
}
// Adds this CTA's value v of column pc (op 0 sum with scale 2^e, 1 max, 2 min).
// The split of X = v 2^e into hi and lo is integer work on the FP32 fields of
// v (FP64 arithmetic is slow on this GPU and would sit on every CTA's arrival):
// v = m 2^x with an integer m < 2^24, so |X| 2^32 = m 2^(x + e + 32) is a shift
// of m, truncated at 2^-32 (deterministic; a sign is applied to the 96-bit
// integer). rel: the column divides or is divided by, so a nonzero value must
// keep 30 bits of relative precision (|X| >= 1/4); a smaller one, a value of
// 2^52 or more, an Inf or a NaN sets the overflow flag instead.
static __device__ __noinline__ void fx_push(FxCols f, int pc, int op, int e, float v, bool rel = false) {
  unsigned long long* a = f.acc + 2 * ((blockIdx.x & (f.banks - 1)) * f.stride + pc);
  if (op == 0) {
    const unsigned int bits = __float_as_uint(v);
    const int be = (int)((bits >> 23) & 0xffu);
    if (be == 0xff) {  // Inf or NaN
      atomicOr(f.bad, 1u);
      return;
    }
    const unsigned long long m = be ? ((bits & 0x7fffffu) | 0x800000u) : (bits & 0x7fffffu);
    if (m == 0ull) return;                         // +-0 adds nothing
    const int sh = (be ? be - 150 : -149) + e;     // X = m 2^sh
    const int top = sh + 64 - __clzll((long long)m);  // bit length of m 2^sh; |X| < 2^top
    if (top > 52 || (rel && top < -1)) {
      atomicOr(f.bad, 1u);
      return;
    }
    unsigned long long hiw, low;  // |X| 2^32 = hiw 2^32 + low, low < 2^32
    const int s = sh + 32;
    if (s >= 32) {
      hiw = m << (s - 32);
      low = 0ull;
    } else if (s >= 0) {
      const unsigned long long w = m << s;  // < 2^56
      hiw = w >> 32;
      low = w & 0xffffffffull;
    } else {
      hiw = 0ull;
      low = s > -64 ? (m >> (-s)) : 0ull;
    }
    if (bits >> 31) {  // negate the 96-bit integer: (-hiw - [low != 0]) 2^32 + (2^32 - low)
      hiw = (unsigned long long)(-(long long)hiw) - (low != 0ull ? 1ull : 0ull);
      low = low != 0ull ? 4294967296ull - low : 0ull;
    }
    atomicAdd(a, hiw);
    if (low != 0ull) atomicAdd(a + 1, low);
  } else {
    const float u = op == 1 ? v : -v;
    if (u != u) {
      atomicOr(f.bad, 1u);
      return;
    }
    unsigned int b = __float_as_uint(u);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // larger float -> larger unsigned
    atomicMax(a, (unsigned long long)b);
  }
}
// Total of column pc as a compensated pair (s, c), s + c = total; resets the
// column's accumulators for the next launch.
__device__ __forceinline__ float2 fx_take(FxCols f, int pc, int op, int e) {
  unsigned long long hb[kFxMaxBanks], lb[kFxMaxBanks];
#pragma unroll
  for (int b = 0; b < kFxMaxBanks; ++b) {  // every load first, then the sums
    if (b < f.banks) {
      unsigned long long* a = f.acc + 2 * (b * f.stride + pc);
      hb[b] = __ldcg(a);
      lb[b] = __ldcg(a + 1);
    }
  }
  unsigned long long h = 0ull, l = 0ull;
#pragma unroll
  for (int b = 0; b < kFxMaxBanks; ++b) {
    if (b < f.banks) {
      unsigned long long* a = f.acc + 2 * (b * f.stride + pc);
      a[0] = 0ull;
      a[1] = 0ull;
      if (op == 0) {
        h += hb[b];  // two's complement: the wrapping sum is the signed sum
        l += lb[b];
      } else {
        h = hb[b] > h ? hb[b] : h;
      }
    }
  }
  if (op == 0) {
    const double T = ldexp((double)(long long)h + (double)l * (1.0 / 4294967296.0), -e);
    const float s = (float)T;
    return make_float2(s, (float)(T - (double)s));
  }
  if (h == 0ull) return col_init2(op);  // no CTA pushed a value
  unsigned int b = (unsigned int)h;
  b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
  const float u = __uint_as_float(b);
  return make_float2(op == 1 ? u : -u, 0.f);
}

// Arrival of a CTA for the fixed-point completion (after its pushes and its
// row): one device-scope fence and atomic per CTA, as arrive_pass. Returns
// true in the finishing CTA.
__device__ __forceinline__ bool fx_arrive(unsigned int* counters, bool* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = (atom_add_acq_rel_gpu(&counters[0], 1u) == (unsigned int)(gridDim.x - 1));
  __syncthreads();
  return *s_flag;
}

// In the finishing CTA: the column totals into raw[0..stride) (pairs), every
// accumulator and the counter reset. exp_of(pc) / opof(pc) give each column's
// scale and operation. When a CTA set the overflow flag, the FP32 rows (rows x
// stride) of all CTAs are reduced instead (compensated, fixed order). Ends
// with a barrier.
template <typename ExpOf, typename OpOf>
__device__ void fx_finish(unsigned int* counters, const float* rows, int stride, float2* raw, float2* scratch,
                          ExpOf exp_of, OpOf opof) {
  const FxCols f = fx_cols(counters, stride);
  const bool bad = __ldcg(f.bad) != 0u;
  __syncthreads();  // every thread has read the flag before thread 0 clears it
  for (int pc = threadIdx.x; pc < stride; pc += blockDim.x) {
    const float2 v = fx_take(f, pc, opof(pc), exp_of(pc));
    if (!bad) raw[pc] = v;
  }
  if (threadIdx.x == 0) {
    counters[0] = 0u;
    *f.bad = 0u;
  }
  __syncthreads();
  if (bad) reduce_rows(rows, 0, (int)gridDim.x, stride, raw, scratch, opof);  // ends with a barrier
}

// Column totals of an (nb x stride) float matrix in shared memory, L lanes
// per column (L a power of two dividing 32), every CTA thread on some column:
// each lane combines rows li, li + L, ... of its column (compensated FP32
// sums; column pc % period == max_col is a maximum, == min_col a minimum),
// then the L lanes combine in a fixed butterfly and lane 0 of the group
// writes the pair (a fixed order: the result is deterministic). Every warp
// runs the same number of passes (columns past `stride` take dummy values),
// so the shuffles never diverge. No barrier inside. With 16 lanes a CTA of
// 768 threads covers the 36 columns of a SES row at d = 32 in one pass,
// where one warp per column left half the warps two columns in a row.
// (Running this code in the warm-up warps as well, as a shared non-inlined
// function, did not shorten the reduction: measured 1.41 against 1.47 us.)
template <int L>
static __device__ __forceinline__ void group_columns(const float* m, int nb, int stride, float2* out, int period,
                                                     int max_col, int min_col) {
  const int li = threadIdx.x % L, g = threadIdx.x / L, ng = blockDim.x / L;
  const int passes = (stride + ng - 1) / ng;
  for (int k = 0; k < passes; ++k) {
    const int pc = g + k * ng;
    const bool on = pc < stride;
    const int q = on ? pc % period : -3;
    const int op = q == max_col ? 1 : (q == min_col ? 2 : 0);
    float2 acc = col_init2(op);
    if (on)
      for (int r = li; r < nb; r += L) col_comb2(op, acc, make_float2(m[(size_t)r * stride + pc], 0.f));
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
      float2 other;
      other.x = __shfl_xor_sync(0xffffffffu, acc.x, o);
      other.y = __shfl_xor_sync(0xffffffffu, acc.y, o);
      col_comb2(op, acc, other);
    }
    if (on && li == 0) out[pc] = acc;
  }
}

// max_col / min_col / period: the column operations for the single-level
// path (group_columns); opof gives the same for the two-level path.
template <typename OpOf>
__device__ void final_reduce(const float* rows, int stride, const float2* grows, unsigned int* counters,
                             float2* scratch, OpOf opof, float2* raw, float* stage, bool single, int max_col,
                             int min_col, int period) {
  const int nb = gridDim.x;
  if (!single) {
    const int G = (nb + group_size(nb) - 1) / group_size(nb);
    reduce_rows(grows, 0, G, stride, raw, scratch, opof);
    return;
  }
  // stride is a multiple of 4 and rows starts on a 256-byte boundary: copy
  // 16-byte pieces global -> shared with cp.async (L2 only, no registers),
  // all in flight at once, then wait for this thread's copies.
  const int n4 = nb * stride / 4;
  const float4* src = reinterpret_cast<const float4*>(rows);
  float4* dst = reinterpret_cast<float4*>(stage);
  for (int i = threadIdx.x; i < n4; i += blockDim.x) {
    const unsigned int saddr = (unsigned int)__cvta_generic_to_shared(dst + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(src + i) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // the rows are in shared memory: the next launch of the stream may start
  // now (a kernel that let it start earlier already has; then a no-op)
  pdl_trigger();
  if (threadIdx.x == 0) counters[0] = 0u;
  __syncthreads();
  group_columns<16>(stage, nb, stride, raw, period, max_col, min_col);
  __syncthreads();
}

// Sums of up to four doubles per thread over the whole block in one pass
// (fixed order, deterministic); every thread gets the totals. `red` holds
// 4 * 32 doubles. Contains barriers: every thread must call it.
template <int K>
__device__ __forceinline__ void block_sum_k(double (&v)[K], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[k * 32 + warp] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = red[k * 32];
    for (int w = 1; w < nw; ++w) s += red[k * 32 + w];
    v[k] = s;
  }
}

// Warp-wide sums of K doubles (fixed butterfly order: every lane gets the
// same, deterministic totals).
template <int K>
__device__ __forceinline__ void warp_sum_k(double (&v)[K]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

template <int K>
__device__ __forceinline__ void warp_sum_kf(float (&v)[K]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
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

namespace pdscp {

// Reduce-scatter across the LPP lanes of a lane group. On entry v[r] is this
// lane's partial sum for point r (r < NI). Stage s (xor-mask m = LPP >> (s+1))
// keeps the upper half of the remaining points in the lane whose bit m is set
// and adds the other half received from its partner.
//   NI >= LPP: after log2(LPP) stages v[k], k < NI/LPP, holds the full sum for
//              point r = (NI/LPP) * gl + k (gl = lane index in the group);
//   NI <  LPP: after log2(NI) stages a butterfly over the remaining masks
//              leaves in v[0] the full sum for point r = gl / (LPP/NI), held by
//              LPP/NI lanes.
template <int LPP, int NI>
struct GroupScatter {
  static_assert((NI & (NI - 1)) == 0 && (LPP & (LPP - 1)) == 0, "powers of two");
  static constexpr int OWN = NI >= LPP ? NI / LPP : 1;    // points owned per lane
  static constexpr int SHARE = NI >= LPP ? 1 : LPP / NI;  // lanes per owned point
  static constexpr int STAGES = (NI >= LPP ? LPP : NI) == 1 ? 0 : __builtin_ctz(NI >= LPP ? LPP : NI);

  static __device__ __forceinline__ void run(float (&v)[NI], int gl) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      const int m = LPP >> (s + 1);
      const int half = NI >> (s + 1);
      const bool upper = (gl & m) != 0;
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const float send = upper ? v[i] : v[i + half];
        const float keep = upper ? v[i + half] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
      }
    }
    if (NI < LPP) {
#pragma unroll
      for (int m = SHARE / 2; m > 0; m >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    }
  }
  // index (0..NI-1) of the k-th point owned by lane gl
  static __device__ __forceinline__ int owned(int gl, int k) { return NI >= LPP ? OWN * gl + k : gl / SHARE; }
  // lane (within the group) and slot holding point r's result
  static __device__ __forceinline__ int src_lane(int r) { return (r / OWN) * SHARE; }
};

// Points per round for the reduce-scatter kernels: enough 16-byte loads in
// flight per lane (>= 8) with at most 64 point values held in registers.
template <int VW, int LPP>
struct RoundSize {
  static constexpr int a = LPP > 8 ? LPP : 8;
  static constexpr int cap = 64 / VW;
  static constexpr int value = a < cap ? a : cap;
};

}  // namespace pdscp
