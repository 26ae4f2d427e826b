// Host side of the batched SVM iteration and search (svm_batch_kernel.cuh):
// workspace layout (the SES batch's regions plus label offsets and D per
// instance), per-instance tables, the largest point norms, one-iteration
// launches and the device-side search, for float32 or bfloat16 points.
#include <cstring>
#include <vector>

#include "batch_host.cuh"
#include "svm_batch_kernel.cuh"

namespace pdscp {
namespace {
using namespace batchhost;

struct SvmBatchLayout {
  BatchLayout b;
  size_t lab_off, dval_off, total;
};

pdscp_status svm_layout(int num, const int64_t* n, const int32_t* d, int tile_rows, SvmBatchLayout* L,
                        std::vector<BatchInst>* insts, std::vector<BatchTile>* tiles, const int64_t* offs) {
  pdscp_status st = batch_layout(num, n, d, tile_rows, &L->b, insts, tiles, offs, kSvmBatchStride);
  if (st != PDSCP_OK) return st;
  L->lab_off = L->b.total;
  L->dval_off = L->lab_off + r256((size_t)num * sizeof(int64_t));
  L->total = L->dval_off + r256((size_t)num * sizeof(double));
  return PDSCP_OK;
}

// Tables, header, fresh states and D of every instance. Synchronises the
// stream (the host tables are local).
pdscp_status svm_setup(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len, const int64_t* offset_host,
                       const int64_t* n_host, const int32_t* d_host, const int8_t* labels_dev, int64_t labels_len,
                       const int64_t* label_offset_host, int32_t tile_rows, void* ws_dev, size_t ws_bytes,
                       cudaStream_t s) {
  if (!pts_dev || !offset_host || !ws_dev || !n_host || !d_host || !labels_dev || !label_offset_host)
    return err(PDSCP_ERR_INVALID_ARG, "svm batch: null pointer argument");
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16)
    return err(PDSCP_ERR_INVALID_ARG, "svm batch: unknown dtype %lld", dtype);
  const size_t es = batch_elem(dtype);
  if (((uintptr_t)pts_dev % es) != 0 || ((uintptr_t)ws_dev % 256) != 0)
    return err(PDSCP_ERR_INVALID_ARG, "svm batch: points must be aligned to their element and workspace to 256 bytes");
  for (int i = 0; i < num; ++i) {
    if (offset_host[i] < 0 || label_offset_host[i] < 0)
      return err(PDSCP_ERR_INVALID_ARG, "svm batch: negative offset for instance %lld", i);
    if (n_host[i] < 0 || d_host[i] < 0 || offset_host[i] + n_host[i] * (int64_t)d_host[i] > pts_len)
      return err(PDSCP_ERR_INVALID_ARG, "svm batch: instance %lld extends past the %lld point elements", i, pts_len);
    if (label_offset_host[i] + n_host[i] > labels_len)
      return err(PDSCP_ERR_INVALID_ARG, "svm batch: instance %lld's labels extend past the %lld labels", i,
                 labels_len);
  }
  SvmBatchLayout L;
  std::vector<BatchInst> insts;
  std::vector<BatchTile> tiles;
  insts.reserve(num);
  pdscp_status st = svm_layout(num, n_host, d_host, tile_rows, &L, &insts, &tiles, offset_host);
  if (st != PDSCP_OK) return st;
  if (ws_bytes < L.total)
    return err(PDSCP_ERR_WORKSPACE, "svm batch: workspace %lld < %lld bytes", (long long)ws_bytes, (long long)L.total);
  for (auto& in : insts)
    if (in.shape <= 4 && ((uintptr_t)pts_dev + (uintptr_t)in.pt_off * es) % (4 * es) != 0)
      in.shape = batch_shape(in.d, false);
  unsigned char* ws = reinterpret_cast<unsigned char*>(ws_dev);
  SvmBatchHeader sh;
  memset(&sh, 0, sizeof(sh));
  sh.b = BatchHeader{num, L.b.ntiles, (int64_t)L.b.inst_off, (int64_t)L.b.instcnt_off, (int64_t)L.b.tile_off,
                     (int64_t)L.b.partial_off, (int64_t)L.b.search_off, dtype, 0};
  sh.lab_off = (int64_t)L.lab_off;
  sh.dval_off = (int64_t)L.dval_off;
  cudaError_t e = cudaMemsetAsync(ws, 0, 1024, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + 256, &sh, sizeof(sh), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.b.inst_off, insts.data(), insts.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.b.tile_off, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.b.search_off, 0, (size_t)num * sizeof(BatchSearch), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.lab_off, label_offset_host, (size_t)num * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.dval_off, 0, (size_t)num * sizeof(double), s);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: table upload failed (%lld)", (long long)e);
  const BatchInst* inst_dev = reinterpret_cast<const BatchInst*>(ws + L.b.inst_off);
  const BatchTile* tile_dev = reinterpret_cast<const BatchTile*>(ws + L.b.tile_off);
  unsigned int* cnt_dev = reinterpret_cast<unsigned int*>(ws + L.b.instcnt_off);
  unsigned long long* Dbits = reinterpret_cast<unsigned long long*>(ws + L.dval_off);
  svm_batch_init_kernel<<<num, 64, 0, s>>>(inst_dev, ws, cnt_dev);
  const int grid = device_sm_count() * 4;
  if (dtype == PDSCP_BF16)
    svm_batch_norm_kernel<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(pts_dev), inst_dev, tile_dev,
                                               L.b.ntiles, Dbits);
  else
    svm_batch_norm_kernel<<<grid, 256, 0, s>>>(static_cast<const float*>(pts_dev), inst_dev, tile_dev, L.b.ntiles,
                                               Dbits);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host tables go out of scope
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: init launches failed (%lld)", (long long)e);
  return PDSCP_OK;
}

template <typename T>
cudaError_t launch_svm_batch_t(const T* pts, const int8_t* labels, const double* alpha, const double* eor,
                               unsigned char* ws, pdscp_step_out* out, BatchSearch* search, cudaStream_t s, int num) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, svm_batch_kernel<T>, kBatchBlock, 0) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const int grid = device_sm_count() * occ;
  SvmBatchParams p{pts, labels, alpha, eor, ws, out, search};
  svm_batch_kernel<T><<<grid, kBatchBlock, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !search) return e;
  svm_batch_search_kernel<<<(num + 7) / 8, 256, 0, s>>>(ws, num);
  return cudaGetLastError();
}
cudaError_t launch_svm_batch(const void* pts, int32_t dtype, const int8_t* labels, const double* alpha,
                             const double* eor, unsigned char* ws, pdscp_step_out* out, BatchSearch* search,
                             cudaStream_t s, int num = 0) {
  if (dtype == PDSCP_BF16)
    return launch_svm_batch_t(static_cast<const __nv_bfloat16*>(pts), labels, alpha, eor, ws, out, search, s, num);
  return launch_svm_batch_t(static_cast<const float*>(pts), labels, alpha, eor, ws, out, search, s, num);
}

pdscp_status svm_read_header(const void* ws_dev, cudaStream_t s, SvmBatchHeader* sh) {
  cudaError_t e = cudaMemcpyAsync(sh, reinterpret_cast<const unsigned char*>(ws_dev) + 256, sizeof(*sh),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: header read failed (%lld)", (long long)e);
  if (sh->b.search_off <= 0 || sh->dval_off <= 0)
    return err(PDSCP_ERR_INVALID_ARG, "svm batch: workspace was not set up by svm_batch_*init");
  return PDSCP_OK;
}

}  // namespace
}  // namespace pdscp

using namespace pdscp;
using namespace pdscp::batchhost;

extern "C" {

pdscp_status svm_batch_workspace_size(int32_t num, const int64_t* n_host, const int32_t* d_host, int32_t tile_rows,
                                      size_t* bytes_host) {
  if (!bytes_host) return err(PDSCP_ERR_INVALID_ARG, "svm batch: null output pointer");
  SvmBatchLayout L;
  pdscp_status st = svm_layout(num, n_host, d_host, tile_rows, &L, nullptr, nullptr, nullptr);
  if (st != PDSCP_OK) return st;
  *bytes_host = L.total;
  return PDSCP_OK;
}

pdscp_status svm_batch_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                            const int64_t* offset_host, const int64_t* n_host, const int32_t* d_host,
                            const int8_t* labels_dev, int64_t labels_len, const int64_t* label_offset_host,
                            int32_t tile_rows, void* ws_dev, size_t ws_bytes, pdscp_stream stream) {
  return svm_setup(num, pts_dev, dtype, pts_len, offset_host, n_host, d_host, labels_dev, labels_len,
                   label_offset_host, tile_rows, ws_dev, ws_bytes, (cudaStream_t)stream);
}

pdscp_status svm_batch_step(int32_t num, const void* pts_dev, int32_t dtype, const int8_t* labels_dev,
                            const double* alpha_dev, const double* eta_over_rho_dev, void* ws_dev, size_t ws_bytes,
                            pdscp_stream stream, pdscp_step_out* out_dev) {
  if (num < 1 || !pts_dev || !labels_dev || !alpha_dev || !eta_over_rho_dev || !ws_dev)
    return err(PDSCP_ERR_INVALID_ARG, "svm batch: bad argument to svm_batch_step");
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16)
    return err(PDSCP_ERR_INVALID_ARG, "svm batch: unknown dtype %lld", dtype);
  if (ws_bytes < 1024) return err(PDSCP_ERR_WORKSPACE, "svm batch: workspace too small");
  cudaError_t e = launch_svm_batch(pts_dev, dtype, labels_dev, alpha_dev, eta_over_rho_dev,
                                   reinterpret_cast<unsigned char*>(ws_dev), out_dev, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: step launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

pdscp_status svm_batch_read(int32_t num, const void* ws_dev, float* mean_dev, float* best_dev, double* D_dev,
                            pdscp_stream stream) {
  if (num < 1 || !ws_dev) return err(PDSCP_ERR_INVALID_ARG, "svm batch: bad argument to svm_batch_read");
  cudaStream_t s = (cudaStream_t)stream;
  SvmBatchHeader sh;
  pdscp_status st = svm_read_header(ws_dev, s, &sh);
  if (st != PDSCP_OK) return st;
  unsigned char* ws = reinterpret_cast<unsigned char*>(const_cast<void*>(ws_dev));
  svm_batch_read_kernel<<<num, 64, 0, s>>>(reinterpret_cast<const BatchInst*>(ws + sh.b.inst_off), ws,
                                           reinterpret_cast<const double*>(ws + sh.dval_off), mean_dev, best_dev,
                                           D_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: read launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

pdscp_status svm_batch_solve_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                                  const int64_t* offset_host, const int64_t* n_host, const int32_t* d_host,
                                  const int8_t* labels_dev, int64_t labels_len, const int64_t* label_offset_host,
                                  int32_t tile_rows, const pdscp_options* opts, void* ws_dev, size_t ws_bytes,
                                  pdscp_stream stream) {
  BatchSolveOpts bo;
  pdscp_status st = solve_opts(opts, &bo);
  if (st != PDSCP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = svm_setup(num, pts_dev, dtype, pts_len, offset_host, n_host, d_host, labels_dev, labels_len, label_offset_host,
                 tile_rows, ws_dev, ws_bytes, s);
  if (st != PDSCP_OK) return st;
  cudaError_t e = cudaMemcpyAsync(reinterpret_cast<unsigned char*>(ws_dev) + kBatchOptsOff, &bo, sizeof(bo),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: options upload failed (%lld)", (long long)e);
  return PDSCP_OK;
}

pdscp_status svm_batch_solve_run(int32_t num, const void* pts_dev, const int8_t* labels_dev, void* ws_dev,
                                 size_t ws_bytes, int32_t launches_per_poll, int64_t max_launches,
                                 pdscp_stream stream, int64_t* launches_host, int32_t* done_host) {
  if (num < 1 || !pts_dev || !labels_dev || !ws_dev || launches_per_poll < 1 || max_launches < 1)
    return err(PDSCP_ERR_INVALID_ARG, "svm batch: bad argument to svm_batch_solve_run");
  if (ws_bytes < 1024) return err(PDSCP_ERR_WORKSPACE, "svm batch: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* ws = reinterpret_cast<unsigned char*>(ws_dev);
  SvmBatchHeader sh;
  pdscp_status st = svm_read_header(ws_dev, s, &sh);
  if (st != PDSCP_OK) return st;
  const int32_t dtype = sh.b.dtype;  // the point type given to svm_batch_solve_init
  BatchSearch* search = reinterpret_cast<BatchSearch*>(ws + sh.b.search_off);
  const unsigned int* done = reinterpret_cast<const unsigned int*>(ws) + 2;
  // a CUDA graph of launches_per_poll iterations, captured on a private
  // stream and replayed on `stream` (as ses_batch_solve_run)
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < launches_per_poll && e == cudaSuccess; ++k)
      e = launch_svm_batch(pts_dev, dtype, labels_dev, nullptr, nullptr, ws, nullptr, search, cs, num);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  int64_t launches = 0;
  unsigned int done_h = 0;
  while (e == cudaSuccess && launches < max_launches) {
    e = cudaGraphLaunch(exec, s);
    launches += launches_per_poll;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&done_h, done, sizeof(done_h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (done_h >= (unsigned int)num) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: search launches failed (%lld)", (long long)e);
  if (launches_host) *launches_host = launches;
  if (done_host) *done_host = (int32_t)done_h;
  return PDSCP_OK;
}

pdscp_status svm_batch_solve_read(int32_t num, const void* ws_dev, double eps, pdscp_report* reports_dev,
                                  float* w_dev, pdscp_stream stream) {
  if (num < 1 || !ws_dev) return err(PDSCP_ERR_INVALID_ARG, "svm batch: bad argument to svm_batch_solve_read");
  cudaStream_t s = (cudaStream_t)stream;
  SvmBatchHeader sh;
  pdscp_status st = svm_read_header(ws_dev, s, &sh);
  if (st != PDSCP_OK) return st;
  const unsigned char* ws = reinterpret_cast<const unsigned char*>(ws_dev);
  svm_batch_solve_read_kernel<<<num, 64, 0, s>>>(reinterpret_cast<const BatchInst*>(ws + sh.b.inst_off),
                                                 reinterpret_cast<const BatchSearch*>(ws + sh.b.search_off), eps,
                                                 reports_dev, w_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "svm batch: read launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

}  // extern "C"
