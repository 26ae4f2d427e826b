// Host side of the C ABI declared in include/pdscp.h: argument checks, the
// workspace layout, the bounds pre-pass, alpha-FTP state handling, one-step
// launches and the two search drivers (Sec. 3 "From feasibility to
// optimization", Sec. 4.1 and 4.2 constants, Sec. 5 stopping rules).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <string>
#include <vector>

#include "bounds_kernel.cuh"
#include "bwd_kernel.cuh"
#include "coreset.cuh"
#include "dispatch.cuh"
#include "ses_kernel.cuh"
#include "svm_kernel.cuh"

namespace pdscp {

cudaError_t launch_ses(const SesParams& p, int dtype, bool vec, cudaStream_t stream, bool pdl = false);
cudaError_t launch_svm(const SvmParams& p, int dtype, bool vec, cudaStream_t stream, bool pdl = false);
cudaError_t launch_ses_merge(const SesMergeParams& m, int dtype, cudaStream_t stream);
cudaError_t launch_svm_merge(const SvmMergeParams& m, cudaStream_t stream);
cudaError_t launch_ses_bwd_seed(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream);
cudaError_t launch_ses_bwd_step(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream, bool pdl);
cudaError_t launch_svm_bwd_seed(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream);
cudaError_t launch_svm_bwd_step(const BwdParams& p, bool bf16, bool vec, cudaStream_t stream, bool pdl);

namespace {

thread_local std::string g_err;

pdscp_status fail(pdscp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

pdscp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(PDSCP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int kRing = 4096;  // step records kept by the solves between polls

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t partials, grows, sink, state, ring, dval, total;
};

// Workspace: [counters][per-CTA partial rows (float)][per-group rows (double)]
//            [warm-up sink][solve state][step ring][D]
Layout layout(int problem, int d) {
  Layout L;
  const int st = problem == PDSCP_SES ? ses_partial_stride(d) : svm_partial_stride(d);
  const size_t rows = (size_t)device_sm_count() * kMaxBlocksPerSM;
  L.partials = kHeadBytes;
  L.grows = L.partials + round256(rows * (size_t)st * sizeof(float));
  L.sink = L.grows + round256((size_t)kMaxGroups * st * sizeof(float2));
  L.state = L.sink + round256(warm_sink_bytes(d));
  L.ring = L.state + round256(state_bytes(d));
  L.dval = L.ring + round256((size_t)kRing * sizeof(pdscp_step_out));
  L.total = L.dval + 256;
  return L;
}

// Reverse-sweep workspace: mwu_step's counters, per-CTA rows and group rows,
// then [state][tape: T entries][adjoint scratch][argmax candidates].
struct BwdLayout {
  size_t state, tape, bw, cval, cidx, total;
};
BwdLayout bwd_layout(int problem, int d, int64_t T) {
  const Layout L = layout(problem, d);
  const size_t rows = (size_t)device_sm_count() * kMaxBlocksPerSM;
  BwdLayout B;
  B.state = L.state;
  B.tape = B.state + round256(state_bytes(d));
  B.bw = B.tape + round256((size_t)T * svm_tape_stride(d) * sizeof(float));  // the larger of the two entries
  B.cval = B.bw + round256(bwd_scratch_bytes(d));
  B.cidx = B.cval + round256(2 * rows * sizeof(float));  // SVM: two candidates per CTA
  B.total = B.cidx + round256(2 * rows * sizeof(long long));
  return B;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t elem_size(int dtype) { return dtype == PDSCP_BF16 ? 2 : 4; }

pdscp_status check_common(int problem, const void* pts, int dtype, int64_t n, int d) {
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16) return fail(PDSCP_ERR_INVALID_ARG, "unknown dtype %d", dtype);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  if (problem == PDSCP_SES && n < 2) return fail(PDSCP_ERR_INVALID_ARG, "SES needs n >= 2 (got %lld)", (long long)n);
  if (problem == PDSCP_SVM && n < 2) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs n >= 2 (got %lld)", (long long)n);
  if (!pts) return fail(PDSCP_ERR_INVALID_ARG, "points pointer is null");
  if (!aligned(pts, elem_size(dtype))) return fail(PDSCP_ERR_INVALID_ARG, "points pointer not aligned to its element");
  return PDSCP_OK;
}

bool use_vec(const void* pts, int dtype, int d) {
  return aligned(pts, 16) && ((size_t)d * elem_size(dtype)) % 16 == 0;
}

// --- bounds launch (instances live here; the pass is a one-off per solve) ---
template <typename T>
struct BoundsLauncher {
  const BoundsParams& p;
  cudaStream_t stream;
  template <int VW, int LPP, int NCH>
  cudaError_t go() {
    constexpr int U = Unroll<VW, NCH>::value;
    auto kern = bounds_kernel<T, VW, LPP, NCH, U>;
    const int grid = pass_grid(kern, 0, p.n, (32 / LPP) * U * kWarps);
    kern<<<grid, kBlock, 0, stream>>>(p);
    return cudaGetLastError();
  }
};

cudaError_t launch_bounds(const BoundsParams& p, int dtype, bool vec, cudaStream_t s) {
  if (dtype == PDSCP_F32) return dispatch_shape<4>(p.d, vec, BoundsLauncher<float>{p, s});
  return dispatch_shape<8>(p.d, vec, BoundsLauncher<__nv_bfloat16>{p, s});
}

cudaError_t launch_state_init(int problem, const void* pts, int dtype, int d, int rules, double delta,
                              int patience, void* state, unsigned int* counter, cudaStream_t s) {
  if (dtype == PDSCP_F32)
    state_init_kernel<float><<<1, 256, 0, s>>>((const float*)pts, d, problem, rules, delta, patience, state, counter);
  else
    state_init_kernel<__nv_bfloat16>
        <<<1, 256, 0, s>>>((const __nv_bfloat16*)pts, d, problem, rules, delta, patience, state, counter);
  return cudaGetLastError();
}

pdscp_status do_step(int problem, const void* pts, int dtype, const float* radii, const int8_t* labels,
                     int64_t n, int d, double alpha, double eta_over_rho, double D, int eval_only,
                     void* state, void* ws, cudaStream_t stream, pdscp_step_out* out, float* tape = nullptr,
                     bool pdl = false) {
  const Layout L = layout(problem, d);
  const bool vec = use_vec(pts, dtype, d);
  unsigned int* counter = reinterpret_cast<unsigned int*>(ws);
  float* partials = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + L.partials);
  float2* grows = reinterpret_cast<float2*>(reinterpret_cast<char*>(ws) + L.grows);
  cudaError_t e;
  if (problem == PDSCP_SES) {
    SesParams p{pts, radii, n, d, eval_only, alpha, eta_over_rho, state, partials, grows, counter, 0, out, 1, nullptr,
                tape, reinterpret_cast<unsigned char*>(ws) + L.sink};
    e = launch_ses(p, dtype, vec, stream, pdl);
  } else {
    SvmParams p{pts, labels, n, d, eval_only, alpha, eta_over_rho, D, state, partials, grows, counter, 0, out, nullptr,
                reinterpret_cast<unsigned char*>(ws) + L.sink, tape};
    e = launch_svm(p, dtype, vec, stream, pdl);
  }
  if (e != cudaSuccess) return cuda_fail(e, "mwu_step launch");
  return PDSCP_OK;
}

}  // namespace

// Error reporting for the other translation units of the library.
pdscp_status report_error(pdscp_status s, const char* msg) {
  g_err = msg;
  return s;
}

unsigned int wait_limit() {
  const char* v = getenv("PDSCP_WAIT_LIMIT");
  if (!v || !*v) return kWaitLimit;
  char* end = nullptr;
  const unsigned long x = strtoul(v, &end, 10);
  return (end && *end == '\0' && x <= 0xffffffffUL) ? (unsigned int)x : kWaitLimit;
}

int device_sm_count() {
  // per-device cache, read and written by any host thread (relaxed atomics:
  // every thread that fills an entry stores the same value)
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

}  // namespace pdscp

using namespace pdscp;

extern "C" {

int32_t pdscp_version(void) { return 100; }

const char* pdscp_last_error(void) { return g_err.c_str(); }

pdscp_status pdscp_workspace_size(int32_t problem, int64_t n, int32_t d, size_t* bytes) {
  if (!bytes) return fail(PDSCP_ERR_INVALID_ARG, "bytes pointer is null");
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  if (n < 1) return fail(PDSCP_ERR_INVALID_ARG, "n must be >= 1");
  const size_t base = layout(problem, d).total;
  *bytes = round256(base) + coreset_bytes(n, d);  // (the core-set checks' region after the solve's)
  return PDSCP_OK;
}

pdscp_status pdscp_state_size(int32_t problem, int32_t d, size_t* bytes) {
  if (!bytes) return fail(PDSCP_ERR_INVALID_ARG, "bytes pointer is null");
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  *bytes = state_bytes(d);
  return PDSCP_OK;
}

pdscp_status pdscp_bounds(int32_t problem, const void* pts, int32_t dtype, const float* radii, int64_t n,
                          int32_t d, void* ws, size_t ws_bytes, pdscp_stream stream, double* D_dev) {
  pdscp_status st = check_common(problem, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if (!ws || !D_dev) return fail(PDSCP_ERR_INVALID_ARG, "workspace or output pointer is null");
  if (!aligned(ws, 16) || !aligned(D_dev, 8)) return fail(PDSCP_ERR_INVALID_ARG, "misaligned workspace/output");
  const Layout L = layout(problem, d);
  if (ws_bytes < L.state) return fail(PDSCP_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, L.state);
  BoundsParams p{pts, problem == PDSCP_SES ? radii : nullptr, n, d, problem,
                 reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + L.partials),
                 reinterpret_cast<unsigned int*>(ws), D_dev};
  cudaError_t e = launch_bounds(p, dtype, use_vec(pts, dtype, d), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "bounds launch");
  return PDSCP_OK;
}

pdscp_status mwu_state_init(int32_t problem, const void* pts, int32_t dtype, int64_t n, int32_t d, int32_t rules,
                            double delta, int32_t patience, void* state, void* ws, size_t ws_bytes,
                            pdscp_stream stream) {
  pdscp_status st = check_common(problem, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if (!state || !ws) return fail(PDSCP_ERR_INVALID_ARG, "state or workspace pointer is null");
  if (!aligned(state, 16) || !aligned(ws, 16)) return fail(PDSCP_ERR_INVALID_ARG, "state/workspace not 16-byte aligned");
  if (rules != PDSCP_RULES_NONE && rules != PDSCP_RULES_PRACTICAL) return fail(PDSCP_ERR_INVALID_ARG, "unknown rules %d", rules);
  if (!(delta >= 0.0) || patience < 1) return fail(PDSCP_ERR_INVALID_ARG, "delta must be >= 0 and patience >= 1");
  if (ws_bytes < layout(problem, d).state) return fail(PDSCP_ERR_WORKSPACE, "workspace too small");
  cudaError_t e = launch_state_init(problem, pts, dtype, d, rules, delta, patience, state,
                                    reinterpret_cast<unsigned int*>(ws), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "state init launch");
  return PDSCP_OK;
}

pdscp_status mwu_step(int32_t problem, const void* pts, int32_t dtype, const float* radii, const int8_t* labels,
                      int64_t n, int32_t d, double alpha, double eta_over_rho, double D, int32_t eval_only,
                      void* state, void* ws, size_t ws_bytes, pdscp_stream stream, pdscp_step_out* out) {
  pdscp_status st = check_common(problem, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if (!state || !ws) return fail(PDSCP_ERR_INVALID_ARG, "state or workspace pointer is null");
  if (!aligned(state, 16) || !aligned(ws, 16)) return fail(PDSCP_ERR_INVALID_ARG, "state/workspace not 16-byte aligned");
  if (out && !aligned(out, 8)) return fail(PDSCP_ERR_INVALID_ARG, "out pointer not 8-byte aligned");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(PDSCP_ERR_INVALID_ARG, "alpha must be finite and > 0");
  if (!(eta_over_rho >= 0.0) || !std::isfinite(eta_over_rho)) return fail(PDSCP_ERR_INVALID_ARG, "eta/rho must be finite and >= 0");
  if (problem == PDSCP_SVM) {
    if (!labels) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs labels");
    if (!(D > 0.0) || !std::isfinite(D)) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs D > 0 (the largest point norm)");
  }
  if (ws_bytes < layout(problem, d).state) return fail(PDSCP_ERR_WORKSPACE, "workspace too small");
  return do_step(problem, pts, dtype, problem == PDSCP_SES ? radii : nullptr, labels, n, d, alpha, eta_over_rho, D,
                 eval_only, state, ws, (cudaStream_t)stream, out);
}

pdscp_status mwu_run(int32_t problem, const void* pts, int32_t dtype, const float* radii, const int8_t* labels,
                     int64_t n, int32_t d, double alpha, double eta_over_rho, double D, int64_t k, void* state, void* ws,
                     size_t ws_bytes, pdscp_stream stream, pdscp_step_out* out) {
  if (k < 0) return fail(PDSCP_ERR_INVALID_ARG, "mwu_run: k = %lld < 0", (long long)k);
  pdscp_status st = check_common(problem, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if (!state || !ws) return fail(PDSCP_ERR_INVALID_ARG, "state or workspace pointer is null");
  if (!aligned(state, 16) || !aligned(ws, 16)) return fail(PDSCP_ERR_INVALID_ARG, "state/workspace not 16-byte aligned");
  if (out && !aligned(out, 8)) return fail(PDSCP_ERR_INVALID_ARG, "out pointer not 8-byte aligned");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(PDSCP_ERR_INVALID_ARG, "alpha must be finite and > 0");
  if (!(eta_over_rho >= 0.0) || !std::isfinite(eta_over_rho)) return fail(PDSCP_ERR_INVALID_ARG, "eta/rho must be finite and >= 0");
  if (problem == PDSCP_SVM) {
    if (!labels) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs labels");
    if (!(D > 0.0) || !std::isfinite(D)) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs D > 0 (the largest point norm)");
  }
  if (ws_bytes < layout(problem, d).state) return fail(PDSCP_ERR_WORKSPACE, "workspace too small");
  for (int64_t j = 0; j < k; ++j) {
    st = do_step(problem, pts, dtype, problem == PDSCP_SES ? radii : nullptr, labels, n, d, alpha, eta_over_rho, D, 0,
                 state, ws, (cudaStream_t)stream, out ? out + j : nullptr, nullptr, true);
    if (st != PDSCP_OK) return st;
  }
  return PDSCP_OK;
}

pdscp_status mwu_state_read(int32_t problem, int32_t d, const void* state, float* mean_dev, float* best_dev,
                            pdscp_stream stream) {
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d outside range");
  if (!state) return fail(PDSCP_ERR_INVALID_ARG, "state pointer is null");
  state_read_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(d, problem, state, mean_dev, best_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "state read launch");
  return PDSCP_OK;
}

pdscp_status mwu_state_set(int32_t problem, const void* pts, int32_t dtype, const float* radii,
                           const int8_t* labels, int64_t n, int32_t d, int64_t t, const double* mean_dev, double D,
                           void* state, void* ws, size_t ws_bytes, pdscp_stream stream) {
  pdscp_status st = check_common(problem, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if (!state || !ws || !mean_dev) return fail(PDSCP_ERR_INVALID_ARG, "state, workspace or mean pointer is null");
  if (!aligned(state, 16) || !aligned(ws, 16) || !aligned(mean_dev, 8))
    return fail(PDSCP_ERR_INVALID_ARG, "misaligned state/workspace/mean");
  if (t < 0) return fail(PDSCP_ERR_INVALID_ARG, "t must be >= 0");
  if (problem == PDSCP_SVM && (!labels || !(D > 0.0))) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs labels and D > 0");
  if (ws_bytes < layout(problem, d).state) return fail(PDSCP_ERR_WORKSPACE, "workspace too small");
  state_set_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(d, problem, t, mean_dev, state, reinterpret_cast<unsigned int*>(ws));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "state set launch");
  // evaluation pass at the mean: sets the shift bound (hint) and f
  return do_step(problem, pts, dtype, problem == PDSCP_SES ? radii : nullptr, labels, n, d, 1.0, 0.0,
                 problem == PDSCP_SVM ? D : 0.0, 1, state, ws, (cudaStream_t)stream, nullptr);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Built-in scratch for mwu_step_noalloc. Some callers cannot allocate device
// memory at all (for example code running inside a host program that owns
// every byte of GPU memory through its own pool and forbids cudaMalloc, or
// plug-ins that must not trigger the implicit synchronisation an allocation
// can cause). For them the workspace of mwu_step lives in this file-scope
// array instead. Every GPU that loads the library reserves it until the
// process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = 2u << 20;  // 2 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device. In host code
// the array's name is only a stand-in, so the address is looked up with the
// device current through cudaGetSymbolAddress. The lookup is host-side work
// (no device call once the library's device code is loaded on the device)
// and is repeated on every call rather than cached: a cached address would
// go stale after cudaDeviceReset or when the device's primary context is
// destroyed and created again.
pdscp_status static_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) return cuda_fail(e, "mwu_step_noalloc: cudaGetSymbolAddress");
  *out = p;
  return PDSCP_OK;
}

}  // namespace

extern "C" {

pdscp_status mwu_step_noalloc(int32_t problem, const void* pts, int32_t dtype, const float* radii,
                              const int8_t* labels, int64_t n, int32_t d, double alpha, double eta_over_rho,
                              double D, int32_t eval_only, void* state, pdscp_stream stream, pdscp_step_out* out) {
  pdscp_status st = check_common(problem, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if (!state) return fail(PDSCP_ERR_INVALID_ARG, "state pointer is null");
  if (!aligned(state, 16)) return fail(PDSCP_ERR_INVALID_ARG, "state not 16-byte aligned");
  if (out && !aligned(out, 8)) return fail(PDSCP_ERR_INVALID_ARG, "out pointer not 8-byte aligned");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(PDSCP_ERR_INVALID_ARG, "alpha must be finite and > 0");
  if (!(eta_over_rho >= 0.0) || !std::isfinite(eta_over_rho)) return fail(PDSCP_ERR_INVALID_ARG, "eta/rho must be finite and >= 0");
  if (problem == PDSCP_SVM) {
    if (!labels) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs labels");
    if (!(D > 0.0) || !std::isfinite(D)) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs D > 0 (the largest point norm)");
  }
  const size_t need = layout(problem, d).state;  // counters + partial rows + group rows
  if (need > kStaticScratchBytes)
    return fail(PDSCP_ERR_WORKSPACE,
                "mwu_step_noalloc: this problem needs %zu bytes of scratch but the built-in scratch holds %zu "
                "bytes (d=%d is too large for it); call mwu_step with a caller-provided workspace instead",
                need, kStaticScratchBytes, d);
  void* ws = nullptr;
  if ((st = static_scratch(&ws)) != PDSCP_OK) return st;
  // The completion counters must start at zero; the scratch keeps whatever
  // the previous call left, so clear them on the caller's stream first.
  cudaError_t e = cudaMemsetAsync(ws, 0, kHeadBytes, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "mwu_step_noalloc: clearing counters");
  return do_step(problem, pts, dtype, problem == PDSCP_SES ? radii : nullptr, labels, n, d, alpha, eta_over_rho, D,
                 eval_only, state, ws, (cudaStream_t)stream, out);
}

// --- row-sharded iteration (one shard of the rows per GPU) -----------------

pdscp_status mwu_shard_row_width(int32_t problem, int32_t d, int32_t* width) {
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  if (!width) return fail(PDSCP_ERR_INVALID_ARG, "width pointer is null");
  *width = problem == PDSCP_SES ? ses_partial_stride(d) : svm_partial_stride(d);
  return PDSCP_OK;
}

pdscp_status mwu_shard_init(int32_t problem, const void* first, int32_t dtype, int32_t d, int32_t rules, double delta,
                            int32_t patience, void* state, void* ws, size_t ws_bytes, pdscp_stream stream) {
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16) return fail(PDSCP_ERR_INVALID_ARG, "unknown dtype %d", dtype);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  if (problem == PDSCP_SES && (!first || !aligned(first, elem_size(dtype))))
    return fail(PDSCP_ERR_INVALID_ARG, "SES shards need v_1 (first), aligned to its element");
  if (!state || !ws) return fail(PDSCP_ERR_INVALID_ARG, "state or workspace pointer is null");
  if (!aligned(state, 16) || !aligned(ws, 16)) return fail(PDSCP_ERR_INVALID_ARG, "state/workspace not 16-byte aligned");
  if (rules != PDSCP_RULES_NONE && rules != PDSCP_RULES_PRACTICAL) return fail(PDSCP_ERR_INVALID_ARG, "unknown rules %d", rules);
  if (!(delta >= 0.0) || patience < 1) return fail(PDSCP_ERR_INVALID_ARG, "delta must be >= 0 and patience >= 1");
  if (ws_bytes < layout(problem, d).state) return fail(PDSCP_ERR_WORKSPACE, "workspace too small");
  cudaError_t e = launch_state_init(problem, first, dtype, d, rules, delta, patience, state,
                                    reinterpret_cast<unsigned int*>(ws), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "state init launch");
  return PDSCP_OK;
}

pdscp_status mwu_shard_partial(int32_t problem, const void* pts, int32_t dtype, const float* radii,
                               const int8_t* labels, int64_t n, int32_t d, int32_t holds_first, double alpha,
                               double eta_over_rho, double D, int32_t eval_only, const void* state, void* ws,
                               size_t ws_bytes, pdscp_stream stream, float* row_out) {
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16) return fail(PDSCP_ERR_INVALID_ARG, "unknown dtype %d", dtype);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  if (n < 1) return fail(PDSCP_ERR_INVALID_ARG, "a shard needs n >= 1 (got %lld)", (long long)n);
  if (!pts || !aligned(pts, elem_size(dtype))) return fail(PDSCP_ERR_INVALID_ARG, "points pointer null or misaligned");
  if (!state || !ws || !row_out) return fail(PDSCP_ERR_INVALID_ARG, "state, workspace or row pointer is null");
  if (!aligned(state, 16) || !aligned(ws, 16)) return fail(PDSCP_ERR_INVALID_ARG, "state/workspace not 16-byte aligned");
  if (!aligned(row_out, 8)) return fail(PDSCP_ERR_INVALID_ARG, "row pointer not 8-byte aligned");
  if (holds_first != 0 && holds_first != 1) return fail(PDSCP_ERR_INVALID_ARG, "holds_first must be 0 or 1");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(PDSCP_ERR_INVALID_ARG, "alpha must be finite and > 0");
  if (!(eta_over_rho >= 0.0) || !std::isfinite(eta_over_rho)) return fail(PDSCP_ERR_INVALID_ARG, "eta/rho must be finite and >= 0");
  if (problem == PDSCP_SVM) {
    if (!labels) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs labels");
    if (!(D > 0.0) || !std::isfinite(D)) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs D > 0 (the largest point norm)");
  }
  if (ws_bytes < layout(problem, d).state) return fail(PDSCP_ERR_WORKSPACE, "workspace too small");
  const Layout L = layout(problem, d);
  const bool vec = use_vec(pts, dtype, d);
  unsigned int* counter = reinterpret_cast<unsigned int*>(ws);
  float* partials = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + L.partials);
  float2* grows = reinterpret_cast<float2*>(reinterpret_cast<char*>(ws) + L.grows);
  void* st_rw = const_cast<void*>(state);  // the pass only reads the state
  float2* row = reinterpret_cast<float2*>(row_out);
  cudaError_t e;
  if (problem == PDSCP_SES) {
    // the same warp split as mwu_step (its warm-up warps streaming nothing), so that one shard reproduces
    // the unsharded iteration bit for bit
    SesParams p{pts, radii, n, d, eval_only, alpha, eta_over_rho, st_rw, partials, grows, counter, 0, nullptr,
                holds_first ? 1 : 0, row, nullptr, reinterpret_cast<unsigned char*>(ws) + L.sink};
    e = launch_ses(p, dtype, vec, (cudaStream_t)stream);
  } else {
    SvmParams p{pts, labels, n, d, eval_only, alpha, eta_over_rho, D, st_rw, partials, grows, counter, 0, nullptr, row,
                reinterpret_cast<unsigned char*>(ws) + L.sink, nullptr};
    e = launch_svm(p, dtype, vec, (cudaStream_t)stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "mwu_shard_partial launch");
  return PDSCP_OK;
}

pdscp_status mwu_shard_finish(int32_t problem, const float* rows, int32_t ranks, const void* first, int32_t dtype,
                              const float* first_radius, int32_t d, double alpha, double eta_over_rho, double D,
                              int32_t eval_only, void* state, pdscp_stream stream, pdscp_step_out* out) {
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16) return fail(PDSCP_ERR_INVALID_ARG, "unknown dtype %d", dtype);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  if (ranks < 1) return fail(PDSCP_ERR_INVALID_ARG, "ranks must be >= 1 (got %d)", ranks);
  if (!rows || !aligned(rows, 8)) return fail(PDSCP_ERR_INVALID_ARG, "rows pointer null or not 8-byte aligned");
  if (!state || !aligned(state, 16)) return fail(PDSCP_ERR_INVALID_ARG, "state pointer null or not 16-byte aligned");
  if (out && !aligned(out, 8)) return fail(PDSCP_ERR_INVALID_ARG, "out pointer not 8-byte aligned");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(PDSCP_ERR_INVALID_ARG, "alpha must be finite and > 0");
  if (!(eta_over_rho >= 0.0) || !std::isfinite(eta_over_rho)) return fail(PDSCP_ERR_INVALID_ARG, "eta/rho must be finite and >= 0");
  cudaError_t e;
  if (problem == PDSCP_SES) {
    if (!first || !aligned(first, elem_size(dtype))) return fail(PDSCP_ERR_INVALID_ARG, "SES needs v_1 (first), aligned to its element");
    SesMergeParams m{reinterpret_cast<const float2*>(rows), ranks, first, first_radius, d, eval_only, alpha,
                     eta_over_rho, state, out};
    e = launch_ses_merge(m, dtype, (cudaStream_t)stream);
  } else {
    if (!(D > 0.0) || !std::isfinite(D)) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs D > 0 (the largest point norm)");
    SvmMergeParams m{reinterpret_cast<const float2*>(rows), ranks, d, eval_only, alpha, eta_over_rho, D, state, out};
    e = launch_svm_merge(m, (cudaStream_t)stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "mwu_shard_finish launch");
  return PDSCP_OK;
}

// --- reverse sweep (SES) -------------------------------------------------------

pdscp_status mwu_backward_workspace_size(int32_t problem, int64_t n, int32_t d, int64_t T, size_t* bytes) {
  if (problem != PDSCP_SES && problem != PDSCP_SVM) return fail(PDSCP_ERR_INVALID_ARG, "unknown problem %d", problem);
  if (d < 1 || d > PDSCP_MAX_D) return fail(PDSCP_ERR_NOT_IMPLEMENTED, "d=%d outside [1, %d]", d, PDSCP_MAX_D);
  if (n < 2 || T < 1) return fail(PDSCP_ERR_INVALID_ARG, "need n >= 2 and T >= 1");
  if (!bytes) return fail(PDSCP_ERR_INVALID_ARG, "bytes pointer is null");
  *bytes = bwd_layout(problem, d, T).total;
  return PDSCP_OK;
}

pdscp_status mwu_backward(int32_t problem, const void* pts, int32_t dtype, const float* radii, const int8_t* labels,
                          int64_t n, int32_t d, double alpha, double eta_over_rho, double D, int64_t T,
                          const double* seed, void* ws, size_t ws_bytes, pdscp_stream stream, float* grad,
                          pdscp_step_out* out) {
  pdscp_status st = check_common(problem, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if (T < 1) return fail(PDSCP_ERR_INVALID_ARG, "T must be >= 1");
  if (!ws || !grad) return fail(PDSCP_ERR_INVALID_ARG, "workspace or gradient pointer is null");
  if (!aligned(ws, 256)) return fail(PDSCP_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (!aligned(grad, 4)) return fail(PDSCP_ERR_INVALID_ARG, "gradient pointer not 4-byte aligned");
  if (out && !aligned(out, 8)) return fail(PDSCP_ERR_INVALID_ARG, "out pointer not 8-byte aligned");
  if (seed && !aligned(seed, 8)) return fail(PDSCP_ERR_INVALID_ARG, "seed pointer not 8-byte aligned");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(PDSCP_ERR_INVALID_ARG, "alpha must be finite and > 0");
  if (!(eta_over_rho >= 0.0) || !std::isfinite(eta_over_rho)) return fail(PDSCP_ERR_INVALID_ARG, "eta/rho must be finite and >= 0");
  if (problem == PDSCP_SVM) {
    if (!labels) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs labels");
    if (!(D > 0.0) || !std::isfinite(D)) return fail(PDSCP_ERR_INVALID_ARG, "SVM needs D > 0 (the largest point norm)");
  }
  const BwdLayout B = bwd_layout(problem, d, T);
  if (ws_bytes < B.total) return fail(PDSCP_ERR_WORKSPACE, "workspace too small for the reverse sweep");
  cudaStream_t s = (cudaStream_t)stream;
  char* w = reinterpret_cast<char*>(ws);
  void* state = w + B.state;
  float* tape = reinterpret_cast<float*>(w + B.tape);
  unsigned int* counter = reinterpret_cast<unsigned int*>(ws);
  cudaError_t e = launch_state_init(problem, pts, dtype, d, PDSCP_RULES_NONE, 1e-4, 10, state, counter, s);
  if (e != cudaSuccess) return cuda_fail(e, "state init launch");
  e = cudaMemsetAsync(grad, 0, (size_t)n * d * sizeof(float), s);
  if (e != cudaSuccess) return cuda_fail(e, "gradient clear");
  // forward, recording the tape (a stopped alpha-FTP leaves the later launches idle)
  const float* rad = problem == PDSCP_SES ? radii : nullptr;
  const int8_t* lab = problem == PDSCP_SVM ? labels : nullptr;
  for (int64_t t = 0; t < T; ++t) {
    st = do_step(problem, pts, dtype, rad, lab, n, d, alpha, eta_over_rho, D, 0, state, ws, s, nullptr, tape, true);
    if (st != PDSCP_OK) return st;
  }
  const Layout L = layout(problem, d);
  BwdParams bp{};
  bp.pts = pts;
  bp.radii = rad;
  bp.labels = lab;
  bp.n = n;
  bp.d = d;
  bp.alpha = alpha;
  bp.s = T - 1;
  bp.state = state;
  bp.tape = tape;
  bp.bw = reinterpret_cast<unsigned char*>(w + B.bw);
  bp.grad = grad;
  bp.partials = reinterpret_cast<float*>(w + L.partials);
  bp.grows = reinterpret_cast<float2*>(w + L.grows);
  bp.counter = counter;
  bp.cand_val = reinterpret_cast<float*>(w + B.cval);
  bp.cand_idx = reinterpret_cast<long long*>(w + B.cidx);
  bp.ncand = device_sm_count() * kMaxBlocksPerSM;
  bp.seed = seed;
  bp.out = out;
  // the reverse passes read 4-element chunks of either point type next to float4 gradient chunks
  const bool bf16 = dtype == PDSCP_BF16;
  const bool vec = d % 4 == 0 && aligned(pts, 4 * elem_size(dtype)) && aligned(grad, 16);
  if (problem == PDSCP_SES) {
    e = launch_ses_bwd_seed(bp, bf16, vec, s);
    if (e != cudaSuccess) return cuda_fail(e, "reverse-sweep seed launch");
    for (int64_t k = T - 1; k >= 1; --k) {  // step 0 only hands dL/dubar^1 to v_1 (done by step 1's bookkeeping)
      bp.s = k;
      e = launch_ses_bwd_step(bp, bf16, vec, s, true);  // consecutive reverse steps overlap (dependent launch)
      if (e != cudaSuccess) return cuda_fail(e, "reverse-step launch");
    }
  } else {
    e = launch_svm_bwd_seed(bp, bf16, vec, s);
    if (e != cudaSuccess) return cuda_fail(e, "reverse-sweep seed launch");
    for (int64_t k = T - 1; k >= 0; --k) {
      bp.s = k;
      e = launch_svm_bwd_step(bp, bf16, vec, s, true);
      if (e != cudaSuccess) return cuda_fail(e, "reverse-step launch");
    }
  }
  return PDSCP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Search drivers
// ---------------------------------------------------------------------------
namespace {

struct FtpResult {
  StateHdr hdr;
  int64_t iters;
  bool certified;  // stopped at a poll because the certificates closed
  bool stuck;      // stopped at a poll because the FTP's own gap stopped shrinking
};

// CERTIFIED mode: first progress check of an alpha-FTP at eta = 1 (1024/eta in
// general; then 2x, 4x, ...), the factor the FTP's own gap must shrink by
// while t doubles, and the eta below which it is not halved any more.
constexpr double kCertFirstCheck = 1024.0;
constexpr double kCertShrink = 0.8;
constexpr double kCertMinEta = 1.0 / 64.0;

// Certificate test of the CERTIFIED mode, made at every poll: the best bounds
// known before this alpha-FTP (lb, ub) combined with the FTP's own (SES: the
// smallest f and the best lower bound; SVM: the largest margin and the best
// Claim 8 value) close to within a factor 1 + eps.
struct CertCheck {
  bool on;
  double lb, ub, eps, eta;
};
bool cert_closed(int problem, const CertCheck& c, const StateHdr& h) {
  if (!c.on) return false;
  const double lo = problem == PDSCP_SES ? std::max(c.lb, h.lb_best) : std::max(c.lb, h.best_f);
  const double hi = problem == PDSCP_SES ? std::min(c.ub, h.best_f) : std::min(c.ub, h.ub_best);
  return hi <= (1.0 + c.eps) * lo;
}
// The FTP's own certificate gap (upper over lower bound, minus 1; inf before a
// lower bound exists), the measure of its progress.
double own_gap(int problem, const StateHdr& h) {
  if (problem == PDSCP_SES) return h.lb_best > 0.0 ? h.best_f / h.lb_best - 1.0 : INFINITY;
  return h.best_f > 0.0 ? h.ub_best / h.best_f - 1.0 : INFINITY;
}

// Core-set certificates of the certified searches (PDSCP_MODE_CORESET).
// next: the search's iteration count of the next check (256, then doubling,
// kept across FTPs); base: the search's count when this FTP began; lb, ub:
// the best bounds this FTP's checks found; w: SVM, the unit direction of lb;
// SES, the centre of the ball of radius ub.
struct CoresetHook {
  int64_t next = kCoresetFirst, base = 0;
  double lb = 0.0, ub = INFINITY;
  std::vector<double> w;
  void* ws = nullptr;  // coreset_bytes(n, d) bytes of the solve's workspace
};

pdscp_status check_opts(const pdscp_options* o) {
  if (!o) return fail(PDSCP_ERR_INVALID_ARG, "options pointer is null");
  if (!(o->eps > 0.0) || !std::isfinite(o->eps)) return fail(PDSCP_ERR_INVALID_ARG, "eps must be > 0");
  if (!(o->delta >= 0.0)) return fail(PDSCP_ERR_INVALID_ARG, "delta must be >= 0");
  if (o->patience < 1) return fail(PDSCP_ERR_INVALID_ARG, "patience must be >= 1");
  if (o->mode != PDSCP_MODE_PRACTICAL && o->mode != PDSCP_MODE_THEORY && o->mode != PDSCP_MODE_CERTIFIED &&
      o->mode != PDSCP_MODE_CORESET)
    return fail(PDSCP_ERR_INVALID_ARG, "unknown mode");
  if (o->max_iters < 1) return fail(PDSCP_ERR_INVALID_ARG, "max_iters must be >= 1");
  if (o->poll_every < 1 || o->poll_every > kRing) return fail(PDSCP_ERR_INVALID_ARG, "poll_every outside [1, %d]", kRing);
  if (o->max_steps < 1) return fail(PDSCP_ERR_INVALID_ARG, "max_steps must be >= 1");
  if (!(o->eta >= 0.0) || o->eta > 1.0) return fail(PDSCP_ERR_INVALID_ARG, "eta must be 0 (theorem) or in (0, 1]");
  return PDSCP_OK;
}

// Runs one alpha-FTP on the device: T (capped by budget) iterations, polling
// the state every poll_every launches; evaluates f at the final mean when the
// loop ended without a stop (as the oracle's end-of-FTP evaluation does).
// cert.on (CERTIFIED mode): the stall rule is off (delta = 0); the FTP also
// ends at the first poll where the certificates close, or, as stuck, at the
// first poll with t >= c, 2c, 4c, ... (c = 1024/eta; none once eta <= 1/64)
// where its own gap has not shrunk by the factor 0.8 since the previous one.
pdscp_status run_ftp(int problem, const void* pts, int dtype, const float* radii, const int8_t* labels, int64_t n,
                     int d, double alpha, double eta_over_rho, double D, int rules, const pdscp_options* o,
                     int64_t budget, void* ws, size_t ws_bytes, cudaStream_t s, FtpResult* res,
                     const CertCheck& cert = CertCheck{false, 0.0, 0.0, 0.0, 1.0}, CoresetHook* cs = nullptr) {
  const Layout L = layout(problem, d);
  void* state = reinterpret_cast<char*>(ws) + L.state;
  pdscp_step_out* ring = reinterpret_cast<pdscp_step_out*>(reinterpret_cast<char*>(ws) + L.ring);
  res->certified = false;
  pdscp_status st = mwu_state_init(problem, pts, dtype, n, d, rules, cert.on ? 0.0 : o->delta, o->patience, state,
                                   ws, ws_bytes, (pdscp_stream)s);
  if (st != PDSCP_OK) return st;
  int64_t ran = 0;
  StateHdr h;
  bool stopped = false;
  res->stuck = false;
  double last_gap = INFINITY;
  double next_check = (cert.on && cert.eta > kCertMinEta) ? std::ceil(kCertFirstCheck / cert.eta) : INFINITY;
  while (ran < budget) {
    const int64_t chunk = std::min<int64_t>(o->poll_every, budget - ran);
    for (int64_t j = 0; j < chunk; ++j) {
      // consecutive iterations of the solve overlap by programmatic dependent launch
      st = do_step(problem, pts, dtype, radii, labels, n, d, alpha, eta_over_rho, D, 0, state, ws, s, ring + j, nullptr,
                   true);
      if (st != PDSCP_OK) return st;
    }
    ran += chunk;
    cudaError_t e = cudaMemcpyAsync(&h, state, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ftp poll");
    if (h.status != PDSCP_OK) return fail((pdscp_status)h.status, "device status %d in alpha-FTP", h.status);
    if (h.stopped) {
      stopped = true;
      break;
    }
    if (cs && problem == PDSCP_SES && cs->base + h.t >= cs->next) {
      // SES: from the current mean
      float* tmp = reinterpret_cast<float*>(cs->ws);
      std::vector<float> cf(d);
      st = mwu_state_read(problem, d, state, tmp, nullptr, (pdscp_stream)s);
      if (st != PDSCP_OK) return st;
      e = cudaMemcpyAsync(cf.data(), tmp, (size_t)d * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "core-set centre read");
      std::vector<double> c0(cf.begin(), cf.end()), cc;
      double lbc = 0.0, ubc = INFINITY;
      st = ses_coreset_check(pts, dtype, n, d, c0.data(), cert.eps, cs->ws, s, &lbc, &ubc, cc);
      if (st != PDSCP_OK) return st;
      cs->lb = std::max(cs->lb, lbc);
      if (ubc < cs->ub) {
        cs->ub = ubc;
        cs->w = cc;
      }
      cs->next *= 2;
    } else if (cs && cs->base + h.t >= cs->next) {
      // the check starts from the FTP's best direction so far: a core-set
      // direction of this FTP, else the device's best, else the mean
      std::vector<double> w0(d);
      if (cs->lb > 0.0 && cs->lb >= h.best_f) {
        w0 = cs->w;
      } else {
        float* tmp = reinterpret_cast<float*>(cs->ws);
        std::vector<float> wf(d);
        st = mwu_state_read(problem, d, state, h.best_f > 0.0 ? nullptr : tmp, h.best_f > 0.0 ? tmp : nullptr,
                            (pdscp_stream)s);
        if (st != PDSCP_OK) return st;
        e = cudaMemcpyAsync(wf.data(), tmp, (size_t)d * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "core-set direction read");
        for (int j = 0; j < d; ++j) w0[j] = wf[j];
      }
      double lbc = 0.0, ubc = INFINITY;
      std::vector<double> wc;
      st = svm_coreset_check(pts, dtype, labels, n, d, w0.data(), cert.eps, cs->ws, s, &lbc, &ubc, wc);
      if (st != PDSCP_OK) return st;
      if (lbc > cs->lb) {
        cs->lb = lbc;
        cs->w = wc;
      }
      cs->ub = std::min(cs->ub, ubc);
      cs->next *= 2;
    }
    StateHdr hc = h;  // the core-set bounds join the FTP's own
    if (cs && problem == PDSCP_SES) {
      hc.lb_best = std::max(hc.lb_best, cs->lb);
      hc.best_f = std::min(hc.best_f, cs->ub);
    } else if (cs) {
      hc.best_f = std::max(hc.best_f, cs->lb);
      hc.ub_best = std::min(hc.ub_best, cs->ub);
    }
    if (cert_closed(problem, cert, hc)) {
      res->certified = true;
      break;
    }
    if (cert.on && (double)h.t >= next_check) {
      const double gap = own_gap(problem, hc);
      if (gap > kCertShrink * last_gap) {
        res->stuck = true;
        break;
      }
      last_gap = gap;
      next_check *= 2;
    }
  }
  if (!stopped) {
    st = do_step(problem, pts, dtype, radii, labels, n, d, alpha, eta_over_rho, D, 1, state, ws, s, nullptr);
    if (st != PDSCP_OK) return st;
    cudaError_t e = cudaMemcpyAsync(&h, state, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ftp final read");
  }
  res->hdr = h;
  res->iters = h.t;
  return PDSCP_OK;
}

int64_t theorem_T(double c, double D, double logr, double eps_i, double alpha) {
  const double T = std::ceil(c * D * D * logr / (eps_i * eps_i * alpha * alpha));
  return T > 4.0e18 ? (int64_t)4e18 : (int64_t)T;
}

}  // namespace

extern "C" {

pdscp_status ses_solve(const void* pts, int32_t dtype, const float* radii, int64_t n, int32_t d,
                       const pdscp_options* o, void* ws, size_t ws_bytes, pdscp_stream stream, float* center,
                       pdscp_report* rep) {
  pdscp_status st = check_common(PDSCP_SES, pts, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if ((st = check_opts(o)) != PDSCP_OK) return st;
  if (!ws || !center || !rep) return fail(PDSCP_ERR_INVALID_ARG, "null workspace/center/report pointer");
  if (!aligned(ws, 256)) return fail(PDSCP_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  const Layout L = layout(PDSCP_SES, d);
  // core-set certificates for points (with radii the mode is CERTIFIED)
  const bool use_cs = o->mode == PDSCP_MODE_CORESET && !radii;
  const size_t need = use_cs ? round256(L.total) + coreset_bytes(n, d) : L.total;
  if (ws_bytes < need) return fail(PDSCP_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
  CoresetHook cs;
  cs.ws = reinterpret_cast<char*>(ws) + round256(L.total);
  cudaStream_t s = (cudaStream_t)stream;
  memset(rep, 0, sizeof(*rep));
  double* Ddev = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + L.dval);
  if ((st = mwu_state_init(PDSCP_SES, pts, dtype, n, d, 0, 0.0, 1, reinterpret_cast<char*>(ws) + L.state, ws,
                           ws_bytes, stream)) != PDSCP_OK)
    return st;
  if ((st = pdscp_bounds(PDSCP_SES, pts, dtype, radii, n, d, ws, ws_bytes, stream, Ddev)) != PDSCP_OK) return st;
  double D = 0.0;
  cudaError_t e = cudaMemcpyAsync(&D, Ddev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "bounds read");
  if (!std::isfinite(D)) return fail(PDSCP_ERR_NUMERIC, "bounds pass produced a non-finite D");
  rep->D = D;
  const size_t esz = elem_size(dtype);
  float gam1 = 0.f;
  if (radii) {
    e = cudaMemcpyAsync(&gam1, radii, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "radius read");
  }
  // centre fallback: v_1 with radius D encloses every sphere
  auto copy_v1 = [&]() -> pdscp_status {
    void* st0 = reinterpret_cast<char*>(ws) + L.state;
    if (mwu_state_init(PDSCP_SES, pts, dtype, n, d, 0, 0.0, 1, st0, ws, ws_bytes, stream) != PDSCP_OK) return PDSCP_ERR_CUDA;
    return mwu_state_read(PDSCP_SES, d, st0, center, nullptr, stream);
  };
  (void)esz;
  if (D <= 0.0) {  // all spheres share a centre and have radius 0
    if ((st = copy_v1()) != PDSCP_OK) return st;
    rep->value = rep->lower_bound = rep->upper_bound = 0.0;
    rep->status = PDSCP_OK;
    return PDSCP_OK;
  }
  const double rho = 3.0 * D / std::sqrt(2.0);
  const double logr = std::log(2.0 * (double)(n - 1));
  double Lo = D / 2.0, Up = D, lb = 0.0, ub = INFINITY;
  int64_t total = 0;
  int steps = 0;
  bool have_center = false;
  const double eps = o->eps;
  const bool certified = o->mode == PDSCP_MODE_CERTIFIED || o->mode == PDSCP_MODE_CORESET;
  const int rules = o->mode == PDSCP_MODE_THEORY ? PDSCP_RULES_NONE : PDSCP_RULES_PRACTICAL;
  // CERTIFIED: only proven conclusions move the range (separation: OPT > alpha;
  // f < alpha: OPT < alpha), every FTP also ends when the certificates close,
  // and the loop ends on ub <= (1+eps) max(lb, L); eta defaults to 1.
  double eta_c = o->eta > 0.0 ? o->eta : 1.0;
  while (certified && ub > (1.0 + eps) * std::max(lb, Lo) && total < o->max_iters && steps < o->max_steps) {
    const double alpha = Lo + (Up - Lo) / 3.0;
    const double eta = eta_c;
    FtpResult r;
    const CertCheck c{true, std::max(lb, Lo), ub, eps, eta};
    cs.base = total;
    cs.lb = 0.0;
    cs.ub = INFINITY;
    if ((st = run_ftp(PDSCP_SES, pts, dtype, radii, nullptr, n, d, alpha, eta / rho, 0.0, rules, o, o->max_iters - total,
                      ws, ws_bytes, s, &r, c, use_cs ? &cs : nullptr)) != PDSCP_OK)
      return st;
    total += r.iters;
    if (r.hdr.best_f < ub) {
      ub = r.hdr.best_f;
      if ((st = mwu_state_read(PDSCP_SES, d, reinterpret_cast<char*>(ws) + L.state, nullptr, center, stream)) != PDSCP_OK)
        return st;
      have_center = true;
    }
    if (r.hdr.lb_best > lb) lb = r.hdr.lb_best;
    if (cs.ub < ub) {  // a core-set centre gives the smallest enclosing ball
      ub = cs.ub;
      std::vector<float> cf(cs.w.begin(), cs.w.end());
      e = cudaMemcpyAsync(center, cf.data(), (size_t)d * sizeof(float), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "core-set centre write");
      have_center = true;
    }
    if (cs.lb > lb) lb = cs.lb;
    const int oc = r.hdr.stopped ? r.hdr.outcome : PDSCP_OUT_RUNNING;
    if (oc == PDSCP_OUT_SEPARATED) Lo = std::max(Lo, alpha);
    if (r.stuck) eta_c *= 0.5;  // smaller steps resolve alpha closer to OPT
    Up = std::min(Up, ub);
    Lo = std::max(Lo, lb);
    ++steps;
    if (oc == PDSCP_OUT_RUNNING && !r.certified && !r.stuck) break;  // budget spent inside the step
  }
  while (!certified && Up > (1.0 + eps) * Lo && ub > (1.0 + eps) * lb && total < o->max_iters &&
         steps < o->max_steps) {
    const double alpha = Lo + (Up - Lo) / 3.0;
    const double eps_i = (Up - Lo) / (3.0 * alpha);
    const int64_t T = theorem_T(36.0, D, logr, eps_i, alpha);
    const double eta = o->eta > 0.0 ? o->eta : std::sqrt(logr / (double)T);
    const int64_t budget = std::min<int64_t>(T, o->max_iters - total);
    FtpResult r;
    if ((st = run_ftp(PDSCP_SES, pts, dtype, radii, nullptr, n, d, alpha, eta / rho, 0.0, rules, o, budget, ws,
                      ws_bytes, s, &r)) != PDSCP_OK)
      return st;
    total += r.iters;
    if (r.hdr.best_f < ub) {
      ub = r.hdr.best_f;
      if ((st = mwu_state_read(PDSCP_SES, d, reinterpret_cast<char*>(ws) + L.state, nullptr, center, stream)) != PDSCP_OK)
        return st;
      have_center = true;
    }
    if (r.hdr.lb_best > lb) lb = r.hdr.lb_best;
    const int oc = r.hdr.stopped ? r.hdr.outcome : PDSCP_OUT_RUNNING;
    if (oc == PDSCP_OUT_SEPARATED) {
      Lo = std::max(Lo, alpha);
    } else if (r.iters >= T || oc == PDSCP_OUT_STALLED || oc == PDSCP_OUT_BEAT_ALPHA) {
      Up = std::min(std::min(Up, (1.0 + eps_i) * alpha), ub);
    }
    Lo = std::max(Lo, lb);
    ++steps;
    if (oc == PDSCP_OUT_RUNNING && r.iters < T) break;  // budget spent inside the step
  }
  if (!have_center) {
    if ((st = copy_v1()) != PDSCP_OK) return st;
    ub = D;
  }
  (void)gam1;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "ses_solve final sync");
  if (certified) lb = std::max(lb, Lo);  // a separation is a proof too
  rep->value = ub;
  rep->lower_bound = lb;
  rep->upper_bound = ub;
  rep->search_L = Lo;
  rep->search_U = Up;
  rep->iters = total;
  rep->search_steps = steps;
  const bool done = certified ? ub <= (1.0 + eps) * lb : (Up <= (1.0 + eps) * Lo || ub <= (1.0 + eps) * lb);
  rep->status = done ? PDSCP_OK : PDSCP_ERR_NOT_CONVERGED;
  if (!done) fail(PDSCP_ERR_NOT_CONVERGED, "iteration budget spent (range [%g, %g], certificate [%g, %g])", Lo, Up, lb, ub);
  return (pdscp_status)rep->status;
}

pdscp_status svm_solve(const void* X, int32_t dtype, const int8_t* labels, int64_t n, int32_t d,
                       const pdscp_options* o, void* ws, size_t ws_bytes, pdscp_stream stream, float* w_out,
                       pdscp_report* rep) {
  pdscp_status st = check_common(PDSCP_SVM, X, dtype, n, d);
  if (st != PDSCP_OK) return st;
  if ((st = check_opts(o)) != PDSCP_OK) return st;
  if (!labels || !ws || !w_out || !rep) return fail(PDSCP_ERR_INVALID_ARG, "null labels/workspace/w/report pointer");
  if (!aligned(ws, 256)) return fail(PDSCP_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  const Layout L = layout(PDSCP_SVM, d);
  const bool use_cs = o->mode == PDSCP_MODE_CORESET;
  const size_t need = use_cs ? round256(L.total) + coreset_bytes(n, d) : L.total;
  if (ws_bytes < need) return fail(PDSCP_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  memset(rep, 0, sizeof(*rep));
  CoresetHook cs;
  cs.ws = reinterpret_cast<char*>(ws) + round256(L.total);
  double* Ddev = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + L.dval);
  if ((st = mwu_state_init(PDSCP_SVM, X, dtype, n, d, 0, 0.0, 1, reinterpret_cast<char*>(ws) + L.state, ws, ws_bytes,
                           stream)) != PDSCP_OK)
    return st;
  if ((st = pdscp_bounds(PDSCP_SVM, X, dtype, nullptr, n, d, ws, ws_bytes, stream, Ddev)) != PDSCP_OK) return st;
  double D = 0.0;
  cudaError_t e = cudaMemcpyAsync(&D, Ddev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "bounds read");
  if (!(D > 0.0) || !std::isfinite(D)) return fail(PDSCP_ERR_NUMERIC, "largest point norm D=%g is not positive", D);
  rep->D = D;
  const double rho = 2.0 * D;
  const double logr = std::log((double)n);
  double Lo = 0.0, Up = 2.0 * D, lb = 0.0, ub = INFINITY;
  int64_t total = 0;
  int steps = 0;
  bool have_w = false;
  const double eps = o->eps;
  const bool certified = o->mode == PDSCP_MODE_CERTIFIED || o->mode == PDSCP_MODE_CORESET;
  const int rules = o->mode == PDSCP_MODE_THEORY ? PDSCP_RULES_NONE : PDSCP_RULES_PRACTICAL;
  // CERTIFIED (as in ses_solve): separation gives U = alpha, f > alpha gives
  // L = f; the loop ends on min(ub, U) <= (1+eps) lb.
  double eta_c = o->eta > 0.0 ? o->eta : 1.0;
  while (certified && std::min(ub, Up) > (1.0 + eps) * lb && total < o->max_iters && steps < o->max_steps) {
    const double alpha = Up - (Up - Lo) / 3.0;
    const double eta = eta_c;
    FtpResult r;
    const CertCheck c{true, lb, std::min(ub, Up), eps, eta};
    cs.base = total;
    cs.lb = 0.0;
    cs.ub = INFINITY;
    if ((st = run_ftp(PDSCP_SVM, X, dtype, nullptr, labels, n, d, alpha, eta / rho, D, rules, o, o->max_iters - total,
                      ws, ws_bytes, s, &r, c, use_cs ? &cs : nullptr)) != PDSCP_OK)
      return st;
    total += r.iters;
    if (cs.lb > lb && cs.lb > r.hdr.best_f) {  // a core-set direction has the best margin
      lb = cs.lb;
      std::vector<float> wf(cs.w.begin(), cs.w.end());
      e = cudaMemcpyAsync(w_out, wf.data(), sizeof(float) * d, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // wf is pageable and about to go
      if (e != cudaSuccess) return cuda_fail(e, "core-set direction write");
      have_w = true;
    } else if (r.hdr.best_f > lb) {
      lb = r.hdr.best_f;
      if ((st = mwu_state_read(PDSCP_SVM, d, reinterpret_cast<char*>(ws) + L.state, nullptr, w_out, stream)) != PDSCP_OK)
        return st;
      have_w = true;
    }
    if (r.hdr.ub_best < ub) ub = r.hdr.ub_best;
    if (cs.ub < ub) ub = cs.ub;
    const int oc = r.hdr.stopped ? r.hdr.outcome : PDSCP_OUT_RUNNING;
    if (oc == PDSCP_OUT_SEPARATED) Up = std::min(Up, alpha);
    if (r.stuck) eta_c *= 0.5;
    Up = std::min(Up, ub);
    Lo = std::max(Lo, lb);
    ++steps;
    if (oc == PDSCP_OUT_RUNNING && !r.certified && !r.stuck) break;
  }
  while (!certified && Up > (1.0 + eps) * Lo && ub > (1.0 + eps) * lb && total < o->max_iters &&
         steps < o->max_steps) {
    const double alpha = Up - (Up - Lo) / 3.0;
    const double eps_i = (Up - Lo) / (3.0 * alpha);
    const int64_t T = theorem_T(64.0, D, logr, eps_i, alpha);
    const double eta = o->eta > 0.0 ? o->eta : std::sqrt(logr / (double)T);
    const int64_t budget = std::min<int64_t>(T, o->max_iters - total);
    FtpResult r;
    if ((st = run_ftp(PDSCP_SVM, X, dtype, nullptr, labels, n, d, alpha, eta / rho, D, rules, o, budget, ws, ws_bytes,
                      s, &r)) != PDSCP_OK)
      return st;
    total += r.iters;
    if (r.hdr.best_f > lb) {
      lb = r.hdr.best_f;
      if ((st = mwu_state_read(PDSCP_SVM, d, reinterpret_cast<char*>(ws) + L.state, nullptr, w_out, stream)) != PDSCP_OK)
        return st;
      have_w = true;
    }
    if (r.hdr.ub_best < ub) ub = r.hdr.ub_best;
    const int oc = r.hdr.stopped ? r.hdr.outcome : PDSCP_OUT_RUNNING;
    if (oc == PDSCP_OUT_SEPARATED) {
      Up = std::min(Up, alpha);
    } else if (r.iters >= T || oc == PDSCP_OUT_STALLED || oc == PDSCP_OUT_BEAT_ALPHA) {
      Lo = std::max(std::max(Lo, (1.0 - eps_i) * alpha), lb);
    }
    Up = std::min(Up, ub);
    Lo = std::max(Lo, lb);
    ++steps;
    if (oc == PDSCP_OUT_RUNNING && r.iters < T) break;
  }
  if (!have_w) {
    e = cudaMemsetAsync(w_out, 0, sizeof(float) * d, s);
    if (e != cudaSuccess) return cuda_fail(e, "w reset");
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "svm_solve final sync");
  if (certified) ub = std::min(ub, Up);  // a separation is a proof too
  rep->value = lb;
  rep->lower_bound = lb;
  rep->upper_bound = ub;
  rep->search_L = Lo;
  rep->search_U = Up;
  rep->iters = total;
  rep->search_steps = steps;
  const bool done = certified ? ub <= (1.0 + eps) * lb : (Up <= (1.0 + eps) * Lo || ub <= (1.0 + eps) * lb);
  rep->status = done ? PDSCP_OK : PDSCP_ERR_NOT_CONVERGED;
  if (!done) fail(PDSCP_ERR_NOT_CONVERGED, "iteration budget spent (range [%g, %g], certificate [%g, %g])", Lo, Up, lb, ub);
  return (pdscp_status)rep->status;
}

}  // extern "C"
