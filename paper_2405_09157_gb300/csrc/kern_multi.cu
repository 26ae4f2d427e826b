// Host side and instances of the multi-candidate SES iteration
// (multi_kernel.cuh): K alpha-FTPs advanced by one pass over float32 points.
#include <cmath>
#include <cstdio>

#include <atomic>

#include "dispatch.cuh"
#include "multi_kernel.cuh"
#include "multi_tc_kernel.cuh"

namespace pdscp {
namespace {

size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

pdscp_status merr(pdscp_status s, const char* fmt, long long a = 0, long long b = 0) {
  char buf[320];
  snprintf(buf, sizeof(buf), fmt, a, b);
  return report_error(s, buf);
}

// Workspace: [counters][per-CTA rows: K st floats][group rows: K st pairs]
struct MultiLayout {
  size_t partials, grows, total;
};
MultiLayout multi_layout(int d, int k) {
  const size_t wst = (size_t)k * ses_partial_stride(d);
  const size_t rows = (size_t)device_sm_count() * kMaxBlocksPerSM;
  MultiLayout L;
  L.partials = kHeadBytes;
  L.grows = L.partials + r256(rows * wst * sizeof(float));
  L.total = L.grows + r256((size_t)kMaxGroups * wst * sizeof(float2));
  return L;
}

template <int K>
struct MultiLauncher {
  const MultiParams& p;
  cudaStream_t stream;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    constexpr int U = K >= 8 ? 2 : Unroll<VW, NCH>::value;  // fewer points in flight, more warps (see the kernel)
    auto kern = ses_multi_kernel<float, VW, LPP, NCH, U, K>;
    const int dp = dpad4(p.d);
    const int wst = K * ses_partial_stride(p.d);
    const size_t pass_smem = (size_t)kWarps * K * dp * sizeof(float);
    const size_t fin_base = (size_t)(wst + K * dp + dp) * sizeof(double);
    size_t smem = pass_smem > fin_base ? pass_smem : fin_base;
    const int per_step = (32 / LPP) * U * kWarps;
    int grid = pass_grid(kern, smem, p.n, per_step);
    MultiParams q = p;
    q.single = single_level(grid, wst, kStageBytesManyCta) ? 1 : 0;
    if (q.single) {
      const size_t fin = fin_base + (size_t)grid * wst * sizeof(float);
      if (fin > smem) smem = fin;
    }
    cudaError_t e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBlock, smem, stream>>>(q);
    return cudaGetLastError();
  }
};

// Shapes for d <= 64 (float32): 16-byte chunks, or scalar lanes.
template <int K>
cudaError_t dispatch_multi(const MultiParams& p, bool vec, cudaStream_t s) {
  MultiLauncher<K> l{p, s};
  if (vec) {
    const int nch = p.d / 4;
    if (nch <= 1) return l.template go<4, 1, 1>();
    if (nch <= 2) return l.template go<4, 2, 1>();
    if (nch <= 4) return l.template go<4, 4, 1>();
    if (nch <= 8) return l.template go<4, 8, 1>();
    return l.template go<4, 16, 1>();
  }
  if (p.d <= 2) return l.template go<1, 2, 1>();
  if (p.d <= 8) return l.template go<1, 8, 1>();
  if (p.d <= 32) return l.template go<1, 32, 1>();
  return l.template go<1, 32, 2>();
}

// cuTensorMapEncodeTiled from the driver (found once; no link against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static std::atomic<EncodeTiledFn> fn{nullptr};
  EncodeTiledFn f = fn.load();
  if (!f) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = reinterpret_cast<EncodeTiledFn>(ptr);
    fn.store(f);
  }
  return f;
}

// Tensor-core pass (multi_tc_kernel.cuh): float32 points with d = 32, rows of
// 128 bytes from a 16-byte aligned base, streamed as tiles of 128 x 32 by a
// TMA load with the 128-byte swizzle; one CTA per SM.
template <int K>
pdscp_status launch_multi_tc(const MultiParams& p, cudaStream_t s) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return merr(PDSCP_ERR_CUDA, "multi: cuTensorMapEncodeTiled unavailable");
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)kTcD, (cuuint64_t)p.n};
  const cuuint64_t gstride[1] = {(cuuint64_t)kTcD * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcD, (cuuint32_t)kTcTile};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(p.pts), gdim, gstride, box,
                         estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return merr(PDSCP_ERR_CUDA, "multi: tensor map encoding failed (%lld)", (long long)r);
  const int64_t ntiles = (p.n + kTcTile - 1) / kTcTile;
  const int grid = (int)(ntiles < device_sm_count() ? ntiles : device_sm_count());
  MultiParams q = p;
  // single level: the finishing CTA stages the rows in chunks of whole
  // candidates in the pass's shared memory (else two levels)
  q.single = tc_stage_candidates(grid, K) >= 1 ? 1 : 0;
  auto kern = ses_multi_tc_kernel<K>;
  cudaError_t e = allow_smem(kern, kTcSmem);
  if (e == cudaSuccess) {
    kern<<<grid, kTcThreads, kTcSmem, s>>>(q, wait_limit(), map);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return merr(PDSCP_ERR_CUDA, "multi: tensor-core launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

}  // namespace
}  // namespace pdscp

using namespace pdscp;

extern "C" {

pdscp_status ses_multi_workspace_size(int32_t d, int32_t k, size_t* bytes_host) {
  if (d < 1 || d > kMultiMaxD) return merr(PDSCP_ERR_NOT_IMPLEMENTED, "multi: d = %lld outside [1, 64]", d);
  if (k != 1 && k != 2 && k != 4 && k != 8 && k != 16)
    return merr(PDSCP_ERR_NOT_IMPLEMENTED, "multi: k = %lld not in {1,2,4,8,16}", k);
  if (!bytes_host) return merr(PDSCP_ERR_INVALID_ARG, "multi: null output pointer");
  *bytes_host = multi_layout(d, k).total;
  return PDSCP_OK;
}

pdscp_status ses_multi_state_stride(int32_t d, size_t* bytes_host) {
  if (d < 1 || d > kMultiMaxD) return merr(PDSCP_ERR_NOT_IMPLEMENTED, "multi: d = %lld outside [1, 64]", d);
  if (!bytes_host) return merr(PDSCP_ERR_INVALID_ARG, "multi: null output pointer");
  *bytes_host = r256(state_bytes(d));
  return PDSCP_OK;
}

pdscp_status ses_multi_step(const float* pts, const float* radii, int64_t n, int32_t d, int32_t k,
                            const double* alpha_dev, const double* eta_over_rho_dev, void* states_dev,
                            void* ws_dev, size_t ws_bytes, pdscp_stream stream, pdscp_step_out* out_dev) {
  if (d < 1 || d > kMultiMaxD) return merr(PDSCP_ERR_NOT_IMPLEMENTED, "multi: d = %lld outside [1, 64]", d);
  if (k != 1 && k != 2 && k != 4 && k != 8 && k != 16)
    return merr(PDSCP_ERR_NOT_IMPLEMENTED, "multi: k = %lld not in {1,2,4,8,16}", k);
  if (n < 2) return merr(PDSCP_ERR_INVALID_ARG, "multi: SES needs n >= 2 (got %lld)", n);
  if (!pts || !alpha_dev || !eta_over_rho_dev || !states_dev || !ws_dev)
    return merr(PDSCP_ERR_INVALID_ARG, "multi: null pointer argument");
  if (((uintptr_t)pts % 4) || ((uintptr_t)states_dev % 256) || ((uintptr_t)ws_dev % 256) ||
      ((uintptr_t)alpha_dev % 8) || ((uintptr_t)eta_over_rho_dev % 8) || (out_dev && ((uintptr_t)out_dev % 8)))
    return merr(PDSCP_ERR_INVALID_ARG, "multi: misaligned pointer (points 4, states/workspace 256, values 8 bytes)");
  const MultiLayout L = multi_layout(d, k);
  if (ws_bytes < L.total) return merr(PDSCP_ERR_WORKSPACE, "multi: workspace %lld < %lld bytes", (long long)ws_bytes,
                                      (long long)L.total);
  unsigned char* ws = reinterpret_cast<unsigned char*>(ws_dev);
  MultiParams p{pts, radii, n, d, k, alpha_dev, eta_over_rho_dev, reinterpret_cast<unsigned char*>(states_dev),
                r256(state_bytes(d)), reinterpret_cast<float*>(ws + L.partials),
                reinterpret_cast<float2*>(ws + L.grows), reinterpret_cast<unsigned int*>(ws), 0, out_dev};
  const bool vec = ((uintptr_t)pts % 16) == 0 && d % 4 == 0;
  cudaStream_t s = (cudaStream_t)stream;
  // 16 candidates: the tensor-core pass (d = 32). Up to 8 the CUDA-core pass,
  // which measured faster at k = 8 (117 against 236 us per pass, n = 1e6)
  if (k == 16) {
    if (!(vec && d == kTcD))
      return merr(PDSCP_ERR_NOT_IMPLEMENTED, "multi: k = 16 needs d = 32 and 16-byte aligned points (got d = %lld)", d);
    return launch_multi_tc<16>(p, s);
  }
  cudaError_t e;
  switch (k) {
    case 1: e = dispatch_multi<1>(p, vec, s); break;
    case 2: e = dispatch_multi<2>(p, vec, s); break;
    case 4: e = dispatch_multi<4>(p, vec, s); break;
    default: e = dispatch_multi<8>(p, vec, s); break;
  }
  if (e != cudaSuccess) return merr(PDSCP_ERR_CUDA, "multi: launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

}  // extern "C"
