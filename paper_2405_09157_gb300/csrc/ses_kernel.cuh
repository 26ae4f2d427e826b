// SES iteration kernel: one streaming pass over the points per MWU iteration
// (Sec. 4.1 with the update of Eq. implement and the ORACLE of Eq. ses_oracle),
// finished in FP64 by the last CTA to complete.
//
// Per cone i >= 2 the exponent is X_i = -k (ubar - v_i; alpha - gamma_i) with
// k = eta t / rho. Its SOC spectrum (Sec. 2.1) is
//   lambda_1 = k (dist_i - a_i)/sqrt2,  lambda_2 = -k (dist_i + a_i)/sqrt2,
//   dist_i = ||ubar - v_i||, a_i = alpha - gamma_i,
// with frame q_{1,2} = (1/sqrt2)(+-(v_i - ubar)/dist_i; 1), so
//   exp(X_i) = (1/sqrt2) ((E1 - E2)(v_i - ubar)/dist_i ; E1 + E2),  E_j = e^{lambda_j}.
// The trace normaliser is C = sum_i (E1 + E2) and p_i = exp(X_i)/C = (w_i; s_i).
// Nothing per point is stored: the pass accumulates
//   S  = sum (E1 + E2)                       (C up to the shift)
//   G' = sum c_i (v_i - ubar),  c_i = (E1 - E2)/dist_i    (so g = G'/(sqrt2 S))
//   Wt = sum [a_i (E1 + E2) - dist_i (E1 - E2)]
//   maxd = max_i dist_i + gamma_i                          (f^t, Sec. 5)
// and the ORACLE value of Eq. (ses_oracle) is rewritten around ubar:
//   g^T u + alpha/sqrt2 - sum v_i^T w_i - sum gamma_i s_i
//     = g^T (u - ubar) + Wt / (sqrt2 S)        (uses sum_i s_i = 1/sqrt2).
//
// Scaling. Every exponent is shifted by a bound M^ >= max_i lambda_1,i known
// before the pass: dist_i(ubar^t) + gamma_i <= hint + move, where hint is the
// maximum at ubar^{t-1} (found by the previous pass) and move = ||ubar^t -
// ubar^{t-1}||. The shift cancels in p; the largest shifted exponent is at
// least -2 k move/sqrt2 >= -4 eta/3, so nothing overflows or underflows
// where it matters. E1 - E2 is formed as E1 * (-expm1(-2 k dist/sqrt2)) so no
// cancellation occurs when dist -> 0 (limit c_i = E1 * sqrt2 k).
#pragma once

#include "common.cuh"

namespace pdscp {

struct SesParams {
  const void* pts;
  const float* radii;  // may be null
  int64_t n;
  int d;
  int eval_only;
  double alpha;
  double eta_over_rho;
  void* state;
  float* partials;
  unsigned int* counter;
  pdscp_step_out* out;  // may be null
};

template <typename T>
__device__ void ses_finalize(const SesParams& p, double* sD, double* s_red, double* s_bc);

// T: element type of the points; VW: elements per chunk; LPP: lanes per point
// (power of two); NCH: chunks per lane; U: points in flight per lane group.
template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) ses_iter_kernel(SesParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_sc[kWarps][3];
  __shared__ double s_red[32];
  __shared__ double s_bc[8];
  __shared__ bool s_last;

  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  if (hdr->stopped && !p.eval_only) return;

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;

  // k/sqrt2; an evaluation pass needs only distances, so it uses k = 0
  const float kr = p.eval_only ? 0.f : (float)((double)hdr->t * p.eta_over_rho / kSqrt2);
  const float H = (float)(hdr->hint + hdr->move);
  const float alpha = (float)p.alpha;
  const float* mean32 = state_mean32(p.state, d);

  float ub[NCH][VW], G[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      ub[j][e] = (c < nch) ? mean32[c * VW + e] : 0.f;
      G[j][e] = 0.f;
    }
  }
  float S = 0.f, W = 0.f, maxd = -INFINITY;

  const T* pts = reinterpret_cast<const T*>(p.pts);
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
          x[u][j][e] -= ub[j][e];
          part = fmaf(x[u][j][e], x[u][j][e], part);
        }
      const float dist2 = group_sum<LPP>(part);
      float c = 0.f;
      if (i >= 1 && i < p.n) {
        const float dist = sqrtf(dist2);
        const float gam = p.radii ? __ldg(p.radii + i) : 0.f;
        const float a = alpha - gam;
        const float E1 = expf(kr * ((dist + gam) - H));
        const float em = -expm1f(-2.f * kr * dist);  // 1 - e^{lambda_2 - lambda_1}
        const float dif = E1 * em;                   // E1 - E2 (shifted)
        const float sum = E1 * (2.f - em);           // E1 + E2 (shifted)
        c = dist > 0.f ? dif / dist : 2.f * kr * E1;
        if (gl == 0) {
          S += sum;
          W += a * sum - dist * dif;
          maxd = fmaxf(maxd, dist + gam);
        }
      }
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) G[j][e] = fmaf(c, x[u][j][e], G[j][e]);
    }
  }

  // ---- CTA reduction: across the lane groups of a warp, then across warps.
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
      for (int e = 0; e < VW; ++e) G[j][e] += __shfl_xor_sync(0xffffffffu, G[j][e], o);
  S = warp_sum(S);
  W = warp_sum(W);
  maxd = warp_max(maxd);
  float* sG = reinterpret_cast<float*>(smem_raw);  // [kWarps][dp]
  if (grp == 0) {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int c = gl + j * LPP;
      if (c < nch)
#pragma unroll
        for (int e = 0; e < VW; ++e) sG[warp * dp + c * VW + e] = G[j][e];
    }
  }
  if (lane == 0) {
    s_sc[warp][0] = S;
    s_sc[warp][1] = W;
    s_sc[warp][2] = maxd;
  }
  __syncthreads();
  float* prow = p.partials + (size_t)blockIdx.x * ses_partial_stride(d);
  for (int j = threadIdx.x; j < d; j += kBlock) {
    float s = 0.f;
    for (int w = 0; w < kWarps; ++w) s += sG[w * dp + j];
    prow[4 + j] = s;
  }
  if (threadIdx.x == 0) {
    float s0 = 0.f, s1 = 0.f, m = -INFINITY;
    for (int w = 0; w < kWarps; ++w) {
      s0 += s_sc[w][0];
      s1 += s_sc[w][1];
      m = fmaxf(m, s_sc[w][2]);
    }
    prow[0] = s0;
    prow[1] = s1;
    prow[2] = m;
    prow[3] = 0.f;
  }
  if (!arrive_last(p.counter, &s_last)) return;
  ses_finalize<T>(p, reinterpret_cast<double*>(smem_raw), s_red, s_bc);
}

// O(d) finish of one SES iteration, run by every thread of the last CTA.
template <typename T>
__device__ void ses_finalize(const SesParams& p, double* sD, double* s_red, double* s_bc) {
  const int d = p.d;
  const int nb = gridDim.x;
  const int st = ses_partial_stride(d);
  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  double* mean = state_mean(p.state);
  float* mean32 = state_mean32(p.state, d);
  float* best = state_best(p.state, d);
  const T* pts = reinterpret_cast<const T*>(p.pts);

  // column sums of the per-CTA partials, in FP64, fixed order
  for (int col = threadIdx.x; col < 3 + d; col += blockDim.x) {
    if (col == 2) {
      double m = -INFINITY;
      for (int b = 0; b < nb; ++b) m = fmax(m, (double)__ldcg(p.partials + (size_t)b * st + 2));
      sD[2] = m;
    } else {
      const int pc = col < 2 ? col : col + 1;
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += (double)__ldcg(p.partials + (size_t)b * st + pc);
      sD[col] = s;
    }
  }
  __syncthreads();
  const double S = sD[0], Wt = sD[1], maxd = sD[2];
  const double alpha = p.alpha;
  const double gam1 = p.radii ? (double)p.radii[0] : 0.0;
  const double inv = 1.0 / (kSqrt2 * S);  // g = G' / (sqrt2 S)

  double ng2 = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double g = sD[3 + j] * inv;
    ng2 += g * g;
  }
  ng2 = block_sum_d(ng2, s_red);
  const double ng = sqrt(ng2);
  const double rad = alpha - gam1;
  double gu = 0.0, d1 = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double g = sD[3 + j] * inv;
    const double v1 = (double)elem_to_float<T>(pts + j);
    const double u = ng > 0.0 ? v1 + rad * g / ng : v1;
    const double m = mean[j];
    gu += g * (u - m);
    d1 += (m - v1) * (m - v1);
  }
  gu = block_sum_d(gu, s_red);
  d1 = block_sum_d(d1, s_red);
  const double V = gu + Wt * inv;                                // Eq. (ses_oracle) value
  const double LB = fmax(gam1, alpha - V / (ng + 1.0 / kSqrt2));  // Eq. (primal_construction)
  const double f = fmax(maxd, sqrt(d1) + gam1);                   // f at the mean read (Sec. 5)
  const int64_t t = hdr->t;

  if (threadIdx.x == 0) {
    int status = PDSCP_OK;
    if (!(S > 0.0) || !isfinite(S) || !isfinite(V) || !isfinite(f)) status = PDSCP_ERR_NUMERIC;
    bool stop = false, failed = false;
    int outcome = PDSCP_OUT_RUNNING;
    const bool better = (t > 0 && f < hdr->best_f);
    if (!p.eval_only) {
      if (LB > hdr->lb_best) hdr->lb_best = LB;
      failed = V < 0.0;
      if (status != PDSCP_OK) {
        stop = true;
      } else if (failed) {
        stop = true;
        outcome = PDSCP_OUT_SEPARATED;
      } else if (hdr->rules == PDSCP_RULES_PRACTICAL && t > 0) {
        if (f < alpha) {
          stop = true;
          outcome = PDSCP_OUT_BEAT_ALPHA;
        } else {
          if (hdr->f_prev > 0.0) {
            hdr->streak = (fabs(f - hdr->f_prev) / hdr->f_prev < hdr->delta) ? hdr->streak + 1 : 0;
            if (hdr->streak >= hdr->patience) {
              stop = true;
              outcome = PDSCP_OUT_STALLED;
            }
          }
          if (!stop) hdr->f_prev = f;
        }
      }
    }
    s_bc[0] = better ? 1.0 : 0.0;
    s_bc[1] = (!p.eval_only && !stop) ? 1.0 : 0.0;
    s_bc[2] = stop ? 1.0 : 0.0;
    s_bc[3] = (double)outcome;
    s_bc[4] = (double)status;
    s_bc[5] = failed ? 1.0 : 0.0;
  }
  __syncthreads();
  const bool better = s_bc[0] != 0.0, advance = s_bc[1] != 0.0;
  double mv = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double m = mean[j];
    if (better) best[j] = (float)m;
    if (advance) {
      const double g = sD[3 + j] * inv;
      const double v1 = (double)elem_to_float<T>(pts + j);
      const double u = ng > 0.0 ? v1 + rad * g / ng : v1;
      const double nm = m + (u - m) / (double)(t + 1);
      mean[j] = nm;
      mean32[j] = (float)nm;
      mv += (nm - m) * (nm - m);
    }
  }
  mv = block_sum_d(mv, s_red);
  if (threadIdx.x == 0) {
    if (better) hdr->best_f = f;
    hdr->hint = maxd;
    hdr->move = advance ? sqrt(mv) : 0.0;
    if (advance) hdr->t = t + 1;
    if (s_bc[2] != 0.0) {
      hdr->stopped = 1;
      hdr->outcome = (int)s_bc[3];
    }
    if ((int)s_bc[4] != PDSCP_OK) hdr->status = (int)s_bc[4];
    hdr->last_value = V;
    if (p.out) {
      pdscp_step_out o;
      o.oracle_value = V;
      o.objective = f;
      o.lower_bound = LB;
      o.upper_bound = f;
      o.t = hdr->t;
      o.failed = s_bc[5] != 0.0;
      o.stopped = hdr->stopped;
      o.status = (int)s_bc[4];
      o.outcome = (int)s_bc[3];
      o.k = (double)t * p.eta_over_rho;
      *p.out = o;
    }
    *p.counter = 0u;
  }
}

}  // namespace pdscp
