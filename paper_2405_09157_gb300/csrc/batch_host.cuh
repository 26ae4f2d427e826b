// Host helpers shared by the batched SES and SVM entry points (batch.cu,
// svm_batch.cu): the workspace layout of a batch (instance and tile tables,
// partial rows, states, search records), error reporting and the search
// options.
#pragma once

#include <cstdio>
#include <vector>

#include "batch_kernel.cuh"
#include "dispatch.cuh"

namespace pdscp {
namespace batchhost {

inline size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

inline pdscp_status err(pdscp_status s, const char* fmt, long long a = 0, long long b = 0) {
  char buf[320];
  snprintf(buf, sizeof(buf), fmt, a, b);
  return report_error(s, buf);
}

struct BatchLayout {
  int64_t ntiles;
  size_t inst_off, instcnt_off, tile_off, partial_off, state_off, search_off, total;
};

// row_floats: floats per tile partial row (kBatchStride for SES, kSvmBatchStride for SVM)
inline pdscp_status batch_layout(int num, const int64_t* n, const int32_t* d, int tile_rows, BatchLayout* L,
                                 std::vector<BatchInst>* insts, std::vector<BatchTile>* tiles, const int64_t* offs,
                                 int row_floats = kBatchStride) {
  if (num < 1) return err(PDSCP_ERR_INVALID_ARG, "batch: num must be >= 1 (got %lld)", num);
  if (!n || !d) return err(PDSCP_ERR_INVALID_ARG, "batch: null size arrays");
  if (tile_rows < 32) return err(PDSCP_ERR_INVALID_ARG, "batch: tile_rows must be >= 32 (got %lld)", tile_rows);
  int64_t T = 0;
  for (int i = 0; i < num; ++i) {
    if (n[i] < 2) return err(PDSCP_ERR_INVALID_ARG, "batch: instance %lld has n = %lld < 2", i, n[i]);
    if (d[i] < 1 || d[i] > kBatchMaxD)
      return err(PDSCP_ERR_NOT_IMPLEMENTED, "batch: instance %lld has d = %lld outside [1, 64]", i, d[i]);
    T += (n[i] + tile_rows - 1) / tile_rows;
  }
  L->ntiles = T;
  L->inst_off = 1024;
  L->instcnt_off = L->inst_off + r256((size_t)num * sizeof(BatchInst));
  L->tile_off = L->instcnt_off + r256((size_t)num * sizeof(unsigned int));
  L->partial_off = L->tile_off + r256((size_t)T * sizeof(BatchTile));
  L->state_off = L->partial_off + r256((size_t)T * row_floats * sizeof(float));
  size_t so = L->state_off;
  int64_t t0 = 0, moff = 0;
  for (int i = 0; i < num; ++i) {
    const int64_t nt = (n[i] + tile_rows - 1) / tile_rows;
    if (insts) {
      BatchInst in;
      in.pt_off = offs ? offs[i] : 0;
      in.n = n[i];
      in.state_off = (int64_t)so;
      in.tile0 = t0;
      in.mean_off = moff;
      in.ntiles = (int32_t)nt;
      in.d = d[i];
      in.shape = batch_shape(d[i], offs ? (offs[i] % 4 == 0) : false);
      in.pad = 0;
      insts->push_back(in);
      for (int64_t k = 0; k < nt; ++k) {
        BatchTile tl;
        tl.inst = i;
        tl.pad = 0;
        tl.r0 = k * tile_rows;
        tl.r1 = (k + 1) * tile_rows < n[i] ? (k + 1) * tile_rows : n[i];
        tiles->push_back(tl);
      }
    }
    so += r256(state_bytes(d[i]));
    t0 += nt;
    moff += d[i];
  }
  L->search_off = r256(so);
  L->total = L->search_off + r256((size_t)num * sizeof(BatchSearch));
  return PDSCP_OK;
}


inline size_t batch_elem(int dtype) { return dtype == PDSCP_BF16 ? 2 : 4; }

// The search options of a batched solve (shared by SES and SVM).
inline pdscp_status solve_opts(const pdscp_options* o, BatchSolveOpts* b) {
  if (!o) return err(PDSCP_ERR_INVALID_ARG, "batch: options pointer is null");
  if (!(o->eps > 0.0) || !(o->delta >= 0.0) || o->patience < 1 || o->max_iters < 1 || o->max_steps < 1 ||
      (o->mode != PDSCP_MODE_PRACTICAL && o->mode != PDSCP_MODE_THEORY && o->mode != PDSCP_MODE_CERTIFIED) ||
      !(o->eta >= 0.0) || o->eta > 1.0 || (o->mode == PDSCP_MODE_CERTIFIED && o->poll_every < 1))
    return err(PDSCP_ERR_INVALID_ARG, "batch: invalid search options");
  const bool cert = o->mode == PDSCP_MODE_CERTIFIED;
  b->eps = o->eps;
  b->delta = cert ? 0.0 : o->delta;  // CERTIFIED: no stall rule
  b->eta = o->eta;
  b->max_iters = o->max_iters;
  b->patience = o->patience;
  b->rules = o->mode == PDSCP_MODE_THEORY ? PDSCP_RULES_NONE : PDSCP_RULES_PRACTICAL;
  b->max_steps = o->max_steps;
  b->mode = o->mode;
  b->poll = cert ? o->poll_every : 1;
  b->pad = 0;
  return PDSCP_OK;
}


}  // namespace batchhost
}  // namespace pdscp
