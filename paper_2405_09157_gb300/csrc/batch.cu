// Host side of the batched SES iteration (batch_kernel.cuh): workspace
// layout, per-instance tables and states, one-iteration launches, for
// float32 or bfloat16 points (one instantiation of the kernels per type).
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "batch_host.cuh"

namespace pdscp {
namespace {
using namespace batchhost;

// Tables, header and fresh states of a batch (shared by the plain and the
// search entry points). Synchronises the stream (the host tables are local).
pdscp_status batch_setup(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len, const int64_t* offset_host,
                         const int64_t* n_host, const int32_t* d_host, int32_t tile_rows, void* ws_dev,
                         size_t ws_bytes, cudaStream_t s, BatchLayout* Lout) {
  if (!pts_dev || !offset_host || !ws_dev || !n_host || !d_host)
    return err(PDSCP_ERR_INVALID_ARG, "batch: null pointer argument");
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16) return err(PDSCP_ERR_INVALID_ARG, "batch: unknown dtype %lld", dtype);
  const size_t es = batch_elem(dtype);
  if (((uintptr_t)pts_dev % es) != 0 || ((uintptr_t)ws_dev % 256) != 0)
    return err(PDSCP_ERR_INVALID_ARG, "batch: points must be aligned to their element and workspace to 256 bytes");
  for (int i = 0; i < num; ++i) {
    if (offset_host[i] < 0) return err(PDSCP_ERR_INVALID_ARG, "batch: negative offset for instance %lld", i);
    if (n_host[i] < 0 || d_host[i] < 0 || offset_host[i] + n_host[i] * (int64_t)d_host[i] > pts_len)
      return err(PDSCP_ERR_INVALID_ARG, "batch: instance %lld extends past the %lld point elements", i, pts_len);
  }
  BatchLayout L;
  std::vector<BatchInst> insts;
  std::vector<BatchTile> tiles;
  insts.reserve(num);
  pdscp_status st = batch_layout(num, n_host, d_host, tile_rows, &L, &insts, &tiles, offset_host);
  if (st != PDSCP_OK) return st;
  if (ws_bytes < L.total) return err(PDSCP_ERR_WORKSPACE, "batch: workspace %lld < %lld bytes", (long long)ws_bytes,
                                     (long long)L.total);
  // chunk loads (16 bytes for float32, 8 for bfloat16) need each instance's rows to start on a
  // 4-element boundary of the address space
  for (auto& in : insts)
    if (in.shape <= 4 && ((uintptr_t)pts_dev + (uintptr_t)in.pt_off * es) % (4 * es) != 0)
      in.shape = batch_shape(in.d, false);
  unsigned char* ws = reinterpret_cast<unsigned char*>(ws_dev);
  BatchHeader bh{num, L.ntiles, (int64_t)L.inst_off, (int64_t)L.instcnt_off, (int64_t)L.tile_off,
                 (int64_t)L.partial_off, (int64_t)L.search_off, dtype, 0};
  cudaError_t e = cudaMemsetAsync(ws, 0, 1024, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + 256, &bh, sizeof(bh), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.inst_off, insts.data(), insts.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.tile_off, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.search_off, 0, (size_t)num * sizeof(BatchSearch), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host tables go out of scope
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: table upload failed (%lld)", (long long)e);
  const BatchInst* inst_dev = reinterpret_cast<const BatchInst*>(ws + L.inst_off);
  unsigned int* cnt_dev = reinterpret_cast<unsigned int*>(ws + L.instcnt_off);
  if (dtype == PDSCP_BF16)
    ses_batch_init_kernel<<<num, 64, 0, s>>>(static_cast<const __nv_bfloat16*>(pts_dev), inst_dev, ws, cnt_dev);
  else
    ses_batch_init_kernel<<<num, 64, 0, s>>>(static_cast<const float*>(pts_dev), inst_dev, ws, cnt_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: init launch failed (%lld)", (long long)e);
  if (Lout) *Lout = L;
  return PDSCP_OK;
}

// One iteration of every instance; with a search, then every instance's search step.
template <typename T>
cudaError_t launch_batch_t(const T* pts, const double* alpha, const double* eor, unsigned char* ws,
                           pdscp_step_out* out, BatchSearch* search, cudaStream_t s, int num, int ctas) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ses_batch_kernel<T>, kBatchBlock, 0) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const int grid = device_sm_count() * (ctas > 0 && ctas < occ ? ctas : occ);
  BatchParams p{pts, alpha, eor, ws, out, search};
  ses_batch_kernel<T><<<grid, kBatchBlock, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !search) return e;
  ses_batch_search_kernel<T><<<(num + 7) / 8, 256, 0, s>>>(pts, ws, num);
  return cudaGetLastError();
}
// ctas: CTAs per SM of the persistent grid (0: as many as fit)
cudaError_t launch_batch(const void* pts, int32_t dtype, const double* alpha, const double* eor, unsigned char* ws,
                         pdscp_step_out* out, BatchSearch* search, cudaStream_t s, int num = 0, int ctas = 0) {
  if (dtype == PDSCP_BF16)
    return launch_batch_t(static_cast<const __nv_bfloat16*>(pts), alpha, eor, ws, out, search, s, num, ctas);
  return launch_batch_t(static_cast<const float*>(pts), alpha, eor, ws, out, search, s, num, ctas);
}

// Records the grid of the search launches and rewrites the instances' lane
// layouts (batch_layout_kernel) in a set-up workspace.
pdscp_status set_launch(int32_t num, const void* pts_dev, void* ws_dev, const BatchHeader& bh, int ctas, int layout,
                        cudaStream_t s) {
  unsigned char* ws = reinterpret_cast<unsigned char*>(ws_dev);
  cudaError_t e = cudaMemcpyAsync(ws + 256 + offsetof(BatchHeader, ctas_per_sm), &ctas, sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    batch_layout_kernel<<<(num + 127) / 128, 128, 0, s>>>(reinterpret_cast<BatchInst*>(ws + bh.inst_off), num,
                                                          pts_dev, (int)batch_elem(bh.dtype), layout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `ctas` is a host local
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: launch settings failed (%lld)", (long long)e);
  return PDSCP_OK;
}

pdscp_status solve_setup(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len, const int64_t* offset_host,
                         const int64_t* n_host, const int32_t* d_host, int32_t tile_rows, const pdscp_options* o,
                         void* ws_dev, size_t ws_bytes, cudaStream_t s) {
  BatchSolveOpts bo;
  pdscp_status st = solve_opts(o, &bo);
  if (st != PDSCP_OK) return st;
  st = batch_setup(num, pts_dev, dtype, pts_len, offset_host, n_host, d_host, tile_rows, ws_dev, ws_bytes, s,
                   nullptr);
  if (st != PDSCP_OK) return st;
  cudaError_t e = cudaMemcpyAsync(reinterpret_cast<unsigned char*>(ws_dev) + kBatchOptsOff, &bo, sizeof(bo),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: options upload failed (%lld)", (long long)e);
  return PDSCP_OK;
}

pdscp_status read_header(const void* ws_dev, cudaStream_t s, BatchHeader* bh) {
  cudaError_t e = cudaMemcpyAsync(bh, reinterpret_cast<const unsigned char*>(ws_dev) + 256, sizeof(*bh),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: header read failed (%lld)", (long long)e);
  if (bh->search_off <= 0) return err(PDSCP_ERR_INVALID_ARG, "batch: workspace was not set up by ses_batch_*init");
  return PDSCP_OK;
}

}  // namespace
}  // namespace pdscp

using namespace pdscp;
using namespace pdscp::batchhost;

extern "C" {

pdscp_status ses_batch_workspace_size(int32_t num, const int64_t* n_host, const int32_t* d_host, int32_t tile_rows,
                                      size_t* bytes_host) {
  if (!bytes_host) return err(PDSCP_ERR_INVALID_ARG, "batch: null output pointer");
  BatchLayout L;
  pdscp_status st = batch_layout(num, n_host, d_host, tile_rows, &L, nullptr, nullptr, nullptr);
  if (st != PDSCP_OK) return st;
  *bytes_host = L.total;
  return PDSCP_OK;
}

pdscp_status ses_batch_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                            const int64_t* offset_host, const int64_t* n_host, const int32_t* d_host,
                            int32_t tile_rows, void* ws_dev, size_t ws_bytes, pdscp_stream stream) {
  return batch_setup(num, pts_dev, dtype, pts_len, offset_host, n_host, d_host, tile_rows, ws_dev, ws_bytes,
                     (cudaStream_t)stream, nullptr);
}

pdscp_status ses_batch_step(int32_t num, const void* pts_dev, int32_t dtype, const double* alpha_dev,
                            const double* eta_over_rho_dev, void* ws_dev, size_t ws_bytes, pdscp_stream stream,
                            pdscp_step_out* out_dev) {
  if (num < 1 || !pts_dev || !alpha_dev || !eta_over_rho_dev || !ws_dev)
    return err(PDSCP_ERR_INVALID_ARG, "batch: bad argument to ses_batch_step");
  if (dtype != PDSCP_F32 && dtype != PDSCP_BF16) return err(PDSCP_ERR_INVALID_ARG, "batch: unknown dtype %lld", dtype);
  if (ws_bytes < 1024) return err(PDSCP_ERR_WORKSPACE, "batch: workspace too small");
  cudaError_t e = launch_batch(pts_dev, dtype, alpha_dev, eta_over_rho_dev, reinterpret_cast<unsigned char*>(ws_dev),
                               out_dev, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: step launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

pdscp_status ses_batch_solve_init(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                                  const int64_t* offset_host, const int64_t* n_host, const int32_t* d_host,
                                  int32_t tile_rows, const pdscp_options* opts, void* ws_dev, size_t ws_bytes,
                                  pdscp_stream stream) {
  return solve_setup(num, pts_dev, dtype, pts_len, offset_host, n_host, d_host, tile_rows, opts, ws_dev, ws_bytes,
                     (cudaStream_t)stream);
}

pdscp_status ses_batch_solve_run(int32_t num, const void* pts_dev, void* ws_dev, size_t ws_bytes,
                                 int32_t launches_per_poll, int64_t max_launches, pdscp_stream stream,
                                 int64_t* launches_host, int32_t* done_host) {
  if (num < 1 || !pts_dev || !ws_dev || launches_per_poll < 1 || max_launches < 1)
    return err(PDSCP_ERR_INVALID_ARG, "batch: bad argument to ses_batch_solve_run");
  if (ws_bytes < 1024) return err(PDSCP_ERR_WORKSPACE, "batch: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* ws = reinterpret_cast<unsigned char*>(ws_dev);
  BatchHeader bh;
  pdscp_status st = read_header(ws_dev, s, &bh);
  if (st != PDSCP_OK) return st;
  const int32_t dtype = bh.dtype;  // the point type given to ses_batch_solve_init
  BatchSearch* search = reinterpret_cast<BatchSearch*>(ws + bh.search_off);
  const unsigned int* done = reinterpret_cast<const unsigned int*>(ws) + 2;
  // a CUDA graph of launches_per_poll iterations, captured on a private stream
  // (the legacy default stream cannot be captured) and replayed on `stream`
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < launches_per_poll && e == cudaSuccess; ++k)
      e = launch_batch(pts_dev, dtype, nullptr, nullptr, ws, nullptr, search, cs, num, bh.ctas_per_sm);
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
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: search launches failed (%lld)", (long long)e);
  if (launches_host) *launches_host = launches;
  if (done_host) *done_host = (int32_t)done_h;
  return PDSCP_OK;
}

pdscp_status ses_batch_solve_read(int32_t num, const void* ws_dev, double eps, pdscp_report* reports_dev,
                                  float* centers_dev, pdscp_stream stream) {
  if (num < 1 || !ws_dev) return err(PDSCP_ERR_INVALID_ARG, "batch: bad argument to ses_batch_solve_read");
  cudaStream_t s = (cudaStream_t)stream;
  BatchHeader bh;
  pdscp_status st = read_header(ws_dev, s, &bh);
  if (st != PDSCP_OK) return st;
  const unsigned char* ws = reinterpret_cast<const unsigned char*>(ws_dev);
  ses_batch_solve_read_kernel<<<num, 64, 0, s>>>(reinterpret_cast<const BatchInst*>(ws + bh.inst_off),
                                                 reinterpret_cast<const BatchSearch*>(ws + bh.search_off), eps,
                                                 reports_dev, centers_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: read launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

pdscp_status ses_batch_autotune(int32_t num, const void* pts_dev, int32_t dtype, int64_t pts_len,
                                const int64_t* offset_host,
                                const int64_t* n_host, const int32_t* d_host, const pdscp_options* opts,
                                void* ws_dev, size_t ws_bytes, pdscp_stream stream, int32_t* tile_rows_host,
                                float* ms_per_launch_host, int32_t* ctas_per_sm_host, int32_t* layout_host) {
  if (!tile_rows_host) return err(PDSCP_ERR_INVALID_ARG, "batch: null output pointer");
  static const int32_t cand[] = {512, 1024, 2048, 4096, 8192, 16384, 32768};
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: event create failed (%lld)", (long long)e);
  int32_t best = 0, best_ctas = 0, best_layout = 0;
  float best_ms = INFINITY;
  pdscp_status st = PDSCP_OK;
  // every tile size that fits, with 1, 2 or 3 CTAs per SM and either layout policy
  for (int32_t tr : cand) {
    BatchLayout L;
    if (batch_layout(num, n_host, d_host, tr, &L, nullptr, nullptr, nullptr) != PDSCP_OK || L.total > ws_bytes) continue;
    for (int layout = 0; layout < 2 && st == PDSCP_OK && e == cudaSuccess; ++layout) {
      for (int ctas = 1; ctas <= 3 && st == PDSCP_OK && e == cudaSuccess; ++ctas) {
        st = solve_setup(num, pts_dev, dtype, pts_len, offset_host, n_host, d_host, tr, opts, ws_dev, ws_bytes, s);
        BatchHeader bh;
        if (st == PDSCP_OK) st = read_header(ws_dev, s, &bh);
        if (st == PDSCP_OK) st = set_launch(num, pts_dev, ws_dev, bh, ctas, layout, s);
        if (st != PDSCP_OK) break;
        unsigned char* ws = reinterpret_cast<unsigned char*>(ws_dev);
        BatchSearch* search = reinterpret_cast<BatchSearch*>(ws + bh.search_off);
        // the bounds pass and one iteration untimed, then four timed iterations
        for (int k = 0; k < 2 && e == cudaSuccess; ++k)
          e = launch_batch(pts_dev, dtype, nullptr, nullptr, ws, nullptr, search, s, num, ctas);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
          e = launch_batch(pts_dev, dtype, nullptr, nullptr, ws, nullptr, search, s, num, ctas);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        if (ms / 4.f < best_ms) {
          best_ms = ms / 4.f;
          best = tr;
          best_ctas = ctas;
          best_layout = layout;
        }
      }
    }
    if (st != PDSCP_OK || e != cudaSuccess) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: autotune launches failed (%lld)", (long long)e);
  if (st != PDSCP_OK) return st;
  if (best == 0) return err(PDSCP_ERR_WORKSPACE, "batch: workspace too small for every tile size");
  *tile_rows_host = best;
  if (ms_per_launch_host) *ms_per_launch_host = best_ms;
  if (ctas_per_sm_host) *ctas_per_sm_host = best_ctas;
  if (layout_host) *layout_host = best_layout;
  return PDSCP_OK;
}

pdscp_status ses_batch_set_launch(int32_t num, const void* pts_dev, void* ws_dev, int32_t ctas_per_sm,
                                  int32_t layout, pdscp_stream stream) {
  if (num < 1 || !pts_dev || !ws_dev) return err(PDSCP_ERR_INVALID_ARG, "batch: bad argument to ses_batch_set_launch");
  if (ctas_per_sm < 0 || ctas_per_sm > 3 || layout < 0 || layout > 1)
    return err(PDSCP_ERR_INVALID_ARG, "batch: ctas_per_sm must be in [0, 3] and layout 0 or 1");
  cudaStream_t s = (cudaStream_t)stream;
  BatchHeader bh;
  pdscp_status st = read_header(ws_dev, s, &bh);
  if (st != PDSCP_OK) return st;
  if (bh.num != num) return err(PDSCP_ERR_INVALID_ARG, "batch: the workspace holds %lld instances, not %lld", bh.num, num);
  return set_launch(num, pts_dev, ws_dev, bh, ctas_per_sm, layout, s);
}

pdscp_status ses_batch_read(int32_t num, const void* ws_dev, float* mean_dev, float* best_dev, pdscp_stream stream) {
  if (num < 1 || !ws_dev) return err(PDSCP_ERR_INVALID_ARG, "batch: bad argument to ses_batch_read");
  unsigned char* ws = reinterpret_cast<unsigned char*>(const_cast<void*>(ws_dev));
  ses_batch_read_kernel<<<num, 64, 0, (cudaStream_t)stream>>>(reinterpret_cast<const BatchInst*>(ws + 1024), ws,
                                                              mean_dev, best_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return err(PDSCP_ERR_CUDA, "batch: read launch failed (%lld)", (long long)e);
  return PDSCP_OK;
}

}  // extern "C"
