// Bounds pre-pass (one streaming pass, max reduction):
//   SES (Sec. 4.1):  D = max_{i>=2} ||v_1 - v_i|| + gamma_1 + gamma_i
//   SVM (Lemma 6):   D = max_i ||x_i||
// plus the small state-initialisation and state-read kernels.
#pragma once

#include "common.cuh"

namespace pdscp {

struct BoundsParams {
  const void* pts;
  const float* radii;  // SES, may be null
  int64_t n;
  int d;
  int problem;
  float* partials;  // one float per CTA
  unsigned int* counter;
  double* D_out;
};

template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) bounds_kernel(BoundsParams p) {
  __shared__ float s_m[kWarps];
  __shared__ bool s_last;
  const int d = p.d;
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  const bool ses = p.problem == PDSCP_SES;
  const T* pts = reinterpret_cast<const T*>(p.pts);

  float ref[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
    if (ses && c < nch) {
      Chunk<T, VW>::load(pts, c, ref[j]);
    } else {
#pragma unroll
      for (int e = 0; e < VW; ++e) ref[j][e] = 0.f;
    }
  }
  const float gam1 = (ses && p.radii) ? __ldg(p.radii) : 0.f;
  float m = -INFINITY;
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  for (int64_t base = gw * (PPW * U); base < p.n; base += nwarps * (PPW * U)) {
    float x[U][NCH][VW];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      const T* row = pts + i * d;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        if (i < p.n && c < nch) {
          Chunk<T, VW>::load(row, c, x[u][j]);
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e) x[u][j][e] = 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      float part = 0.f;
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const float v = x[u][j][e] - ref[j][e];
          part = fmaf(v, v, part);
        }
      const float r = sqrtf(group_sum<LPP>(part));
      if (i < p.n && (!ses || i >= 1)) {
        const float val = ses ? r + gam1 + (p.radii ? __ldg(p.radii + i) : 0.f) : r;
        m = fmaxf(m, val);
      }
    }
  }
  m = warp_max(m);
  if (lane == 0) s_m[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = -INFINITY;
    for (int w = 0; w < kWarps; ++w) b = fmaxf(b, s_m[w]);
    p.partials[blockIdx.x] = b;
  }
  if (!arrive_last(p.counter, &s_last)) return;
  if (threadIdx.x < 32) {  // one warp: lanes stride over the CTAs' maxima
    float D = -INFINITY;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) D = fmaxf(D, __ldcg(p.partials + b));
    D = warp_max(D);
    if (threadIdx.x == 0) {
      *p.D_out = (double)D;
      *p.counter = 0u;
    }
  }
}

// Fresh alpha-FTP state (Sec. 3): t = 0; SES mean = v_1, SVM (w, s1, s2) = 0.
template <typename T>
__global__ void state_init_kernel(const T* pts, int d, int problem, int rules, double delta,
                                  int patience, void* state, unsigned int* counter) {
  StateHdr* hdr = reinterpret_cast<StateHdr*>(state);
  double* mean = state_mean(state);
  float* mean32 = state_mean32(state, d);
  float* best = state_best(state, d);
  double* dual = state_dual(state, d);
  const int dp = dpad4(d);
  for (int j = threadIdx.x; j < dp; j += blockDim.x) {
    const double v = (problem == PDSCP_SES && j < d) ? (double)elem_to_float<T>(pts + j) : 0.0;
    mean[j] = v;
    mean32[j] = (float)v;
    best[j] = (float)v;
    dual[j] = 0.0;
  }
  if (threadIdx.x == 0) {
    StateHdr h;
    h.t = 0;
    h.stopped = 0;
    h.outcome = PDSCP_OUT_RUNNING;
    h.status = PDSCP_OK;
    h.rules = rules;
    h.streak = 0;
    h.patience = patience;
    h.delta = delta;
    h.hint = 0.0;
    h.move = 0.0;
    h.f_prev = -1.0;
    h.best_f = (problem == PDSCP_SES) ? INFINITY : 0.0;
    h.lb_best = 0.0;
    h.ub_best = INFINITY;
    h.s1bar = 0.0;
    h.s2bar = 0.0;
    h.last_value = 0.0;
    h.dual_A = 0.0;
    h.dual_w = 0.0;
    *hdr = h;
  }
  if (counter)
    for (int j = threadIdx.x; j < (int)(kHeadBytes / sizeof(unsigned int)); j += blockDim.x) counter[j] = 0u;
}

// Resume from a checkpoint: t and the running mean (FP64; SVM: wbar, then
// s1bar, s2bar) are set; the shift bound is recomputed by an evaluation pass.
template <int kUnused = 0>
__global__ void state_set_kernel(int d, int problem, int64_t t, const double* mean_in, void* state,
                                 unsigned int* counter) {
  StateHdr* hdr = reinterpret_cast<StateHdr*>(state);
  double* mean = state_mean(state);
  float* mean32 = state_mean32(state, d);
  float* best = state_best(state, d);
  double* dual = state_dual(state, d);
  const int dp = dpad4(d);
  for (int j = threadIdx.x; j < dp; j += blockDim.x) {
    const double v = j < d ? mean_in[j] : 0.0;
    mean[j] = v;
    mean32[j] = (float)v;
    best[j] = (float)v;
    dual[j] = 0.0;
  }
  if (threadIdx.x == 0) {
    StateHdr h;
    h.t = t;
    h.stopped = 0;
    h.outcome = PDSCP_OUT_RUNNING;
    h.status = PDSCP_OK;
    h.rules = PDSCP_RULES_NONE;
    h.streak = 0;
    h.patience = 1;
    h.delta = 0.0;
    h.hint = 0.0;
    h.move = 0.0;
    h.f_prev = -1.0;
    h.best_f = (problem == PDSCP_SES) ? INFINITY : 0.0;
    h.lb_best = 0.0;
    h.ub_best = INFINITY;
    h.s1bar = problem == PDSCP_SVM ? mean_in[d] : 0.0;
    h.s2bar = problem == PDSCP_SVM ? mean_in[d + 1] : 0.0;
    h.last_value = 0.0;
    h.dual_A = 0.0;
    h.dual_w = 0.0;
    *hdr = h;
  }
  if (counter)
    for (int j = threadIdx.x; j < (int)(kHeadBytes / sizeof(unsigned int)); j += blockDim.x) counter[j] = 0u;
}

template <int kUnused = 0>
__global__ void state_read_kernel(int d, int problem, const void* state, float* mean_out,
                                  float* best_out) {
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(state);
  const float* mean32 = state_mean32(const_cast<void*>(state), d);
  const float* best = state_best(const_cast<void*>(state), d);
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    if (mean_out) mean_out[j] = mean32[j];
    if (best_out) best_out[j] = best[j];
  }
  if (threadIdx.x == 0 && mean_out && problem == PDSCP_SVM) {
    mean_out[d] = (float)hdr->s1bar;
    mean_out[d + 1] = (float)hdr->s2bar;
  }
}

}  // namespace pdscp
