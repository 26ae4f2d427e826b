// SVM iteration kernel: one streaming pass over the labelled points per MWU
// iteration of the minimisation variant (Sec. 3, Eq. min_implement) for the
// data of Eq. (svm_dual_scp), K = R^n_+ (Sec. 4.2), finished in FP64 by the
// last CTA to complete.
//
// Point i (label y_i = +1 for P, -1 for Q) has margin
//   m_i = y_i x_i^T wbar - sbar_{class i}      (c - sum_j a_j ybar_j, Sec. 4.2)
// and weight p_i = e^{-k m_i} / sum_l e^{-k m_l}, k = eta t / rho (Sec. 2.1:
// exp on R^n_+ is componentwise). The pass accumulates, per class,
//   S_P = sum_P e^{-k m_i},  Z_P = sum_P e^{-k m_i} x_i   (same for Q)
// and min_P x^T wbar, max_Q x^T wbar. Then Tr(mu) = S_P/S, Tr(gamma) = S_Q/S,
// z = P mu - Q gamma = (Z_P - Z_Q)/S, and the ORACLE of Eq. (svm_oracle) is
// w = z/||z||, s_1 = D if Tr(mu) <= Tr(gamma) else alpha - D, s_2 = alpha - s_1,
// value ||z|| - Tr(mu) s_1 - Tr(gamma) s_2. Claim 10's PD value is
// ||Z_P/S_P - Z_Q/S_Q||; the margin f^t of Sec. 5 is
// max{(min_P x^T wbar - max_Q x^T wbar)/||wbar||, 0}.
//
// Scaling: exponents are shifted by a bound known before the pass. With
// hint = min_i m_i at the previous mean and move = D||dw|| + max|ds| the
// change of the means, every margin at the current mean is >= hint - move,
// so -k (m_i - (hint - move)) <= 0 for all i, and the largest term is at
// least e^{-2 k move}.
#pragma once

#include "common.cuh"

namespace pdscp {

struct SvmParams {
  const void* pts;
  const int8_t* labels;
  int64_t n;
  int d;
  int eval_only;
  double alpha;
  double eta_over_rho;
  double D;
  void* state;
  float* partials;
  unsigned int* counter;
  pdscp_step_out* out;
};

template <typename T>
__device__ void svm_finalize(const SvmParams& p, double* sD, double* s_red, double* s_bc);

template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) svm_iter_kernel(SvmParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_sc[kWarps][4];
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

  const float k = p.eval_only ? 0.f : (float)((double)hdr->t * p.eta_over_rho);
  const float Hm = (float)(hdr->hint - hdr->move);
  const float s1 = (float)hdr->s1bar, s2 = (float)hdr->s2bar;
  const float* mean32 = state_mean32(p.state, d);

  float wb[NCH][VW], ZP[NCH][VW], ZQ[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      wb[j][e] = (c < nch) ? mean32[c * VW + e] : 0.f;
      ZP[j][e] = 0.f;
      ZQ[j][e] = 0.f;
    }
  }
  float SP = 0.f, SQ = 0.f, minP = INFINITY, maxQ = -INFINITY;

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
        for (int e = 0; e < VW; ++e) part = fmaf(x[u][j][e], wb[j][e], part);
      const float dot = group_sum<LPP>(part);
      float qp = 0.f, qq = 0.f;
      if (i < p.n) {
        const bool pos = __ldg(p.labels + i) > 0;
        const float margin = pos ? dot - s1 : -dot - s2;
        const float pt = expf(-k * (margin - Hm));
        qp = pos ? pt : 0.f;
        qq = pos ? 0.f : pt;
        if (gl == 0) {
          SP += qp;
          SQ += qq;
          if (pos) minP = fminf(minP, dot);
          else maxQ = fmaxf(maxQ, dot);
        }
      }
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          ZP[j][e] = fmaf(qp, x[u][j][e], ZP[j][e]);
          ZQ[j][e] = fmaf(qq, x[u][j][e], ZQ[j][e]);
        }
    }
  }

#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        ZP[j][e] += __shfl_xor_sync(0xffffffffu, ZP[j][e], o);
        ZQ[j][e] += __shfl_xor_sync(0xffffffffu, ZQ[j][e], o);
      }
  SP = warp_sum(SP);
  SQ = warp_sum(SQ);
  minP = warp_min(minP);
  maxQ = warp_max(maxQ);
  float* sZ = reinterpret_cast<float*>(smem_raw);  // [kWarps][2 dp]
  if (grp == 0) {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int c = gl + j * LPP;
      if (c < nch)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          sZ[warp * 2 * dp + c * VW + e] = ZP[j][e];
          sZ[warp * 2 * dp + dp + c * VW + e] = ZQ[j][e];
        }
    }
  }
  if (lane == 0) {
    s_sc[warp][0] = SP;
    s_sc[warp][1] = SQ;
    s_sc[warp][2] = minP;
    s_sc[warp][3] = maxQ;
  }
  __syncthreads();
  float* prow = p.partials + (size_t)blockIdx.x * svm_partial_stride(d);
  for (int j = threadIdx.x; j < d; j += kBlock) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < kWarps; ++w) {
      a += sZ[w * 2 * dp + j];
      b += sZ[w * 2 * dp + dp + j];
    }
    prow[4 + j] = a;
    prow[4 + dp + j] = b;
  }
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, mn = INFINITY, mx = -INFINITY;
    for (int w = 0; w < kWarps; ++w) {
      a += s_sc[w][0];
      b += s_sc[w][1];
      mn = fminf(mn, s_sc[w][2]);
      mx = fmaxf(mx, s_sc[w][3]);
    }
    prow[0] = a;
    prow[1] = b;
    prow[2] = mn;
    prow[3] = mx;
  }
  if (!arrive_last(p.counter, &s_last)) return;
  svm_finalize<T>(p, reinterpret_cast<double*>(smem_raw), s_red, s_bc);
}

template <typename T>
__device__ void svm_finalize(const SvmParams& p, double* sD, double* s_red, double* s_bc) {
  const int d = p.d;
  const int dp = dpad4(d);
  const int nb = gridDim.x;
  const int st = svm_partial_stride(d);
  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  double* mean = state_mean(p.state);
  float* mean32 = state_mean32(p.state, d);
  float* best = state_best(p.state, d);

  // sD layout: [0]=S_P [1]=S_Q [2]=minP [3]=maxQ [4..4+d)=Z_P [4+d..4+2d)=Z_Q
  for (int col = threadIdx.x; col < 4 + 2 * d; col += blockDim.x) {
    int pc;
    if (col < 4) pc = col;
    else if (col < 4 + d) pc = col;
    else pc = 4 + dp + (col - 4 - d);
    double acc;
    if (col == 2) {
      acc = INFINITY;
      for (int b = 0; b < nb; ++b) acc = fmin(acc, (double)__ldcg(p.partials + (size_t)b * st + pc));
    } else if (col == 3) {
      acc = -INFINITY;
      for (int b = 0; b < nb; ++b) acc = fmax(acc, (double)__ldcg(p.partials + (size_t)b * st + pc));
    } else {
      acc = 0.0;
      for (int b = 0; b < nb; ++b) acc += (double)__ldcg(p.partials + (size_t)b * st + pc);
    }
    sD[col] = acc;
  }
  __syncthreads();
  const double SP = sD[0], SQ = sD[1], minP = sD[2], maxQ = sD[3];
  const double S = SP + SQ;
  const double trmu = SP / S, trga = SQ / S;
  const double alpha = p.alpha, D = p.D;

  double nz2 = 0.0, ub2 = 0.0, nw2 = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double zp = sD[4 + j], zq = sD[4 + d + j];
    const double z = (zp - zq) / S;
    nz2 += z * z;
    const double df = zp / SP - zq / SQ;
    ub2 += df * df;
    nw2 += mean[j] * mean[j];
  }
  nz2 = block_sum_d(nz2, s_red);
  ub2 = block_sum_d(ub2, s_red);
  nw2 = block_sum_d(nw2, s_red);
  const double nz = sqrt(nz2);
  const double s1 = (trmu <= trga) ? D : alpha - D;
  const double s2 = alpha - s1;
  const double V = nz - trmu * s1 - trga * s2;                       // Eq. (svm_oracle)
  const double UB = (SP > 0.0 && SQ > 0.0) ? sqrt(ub2) : INFINITY;   // Claim 10
  const double nw = sqrt(nw2);
  const double f = nw > 0.0 ? fmax((minP - maxQ) / nw, 0.0) : 0.0;   // Sec. 5
  const int64_t t = hdr->t;
  const double s1b = hdr->s1bar, s2b = hdr->s2bar;

  if (threadIdx.x == 0) {
    int status = PDSCP_OK;
    if (!(S > 0.0) || !isfinite(S) || !isfinite(V)) status = PDSCP_ERR_NUMERIC;
    bool stop = false, failed = false;
    int outcome = PDSCP_OUT_RUNNING;
    const bool better = f > hdr->best_f;
    if (!p.eval_only) {
      if (UB < hdr->ub_best) hdr->ub_best = UB;
      failed = V < 0.0;
      if (status != PDSCP_OK) {
        stop = true;
      } else if (failed) {
        stop = true;
        outcome = PDSCP_OUT_SEPARATED;
      } else if (hdr->rules == PDSCP_RULES_PRACTICAL && t > 0) {
        if (f > alpha) {
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
  const double tp1 = (double)(t + 1);
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double m = mean[j];
    if (better) best[j] = (float)m;
    if (advance) {
      const double z = (sD[4 + j] - sD[4 + d + j]) / S;
      const double w = nz > 0.0 ? z / nz : 0.0;
      const double nm = m + (w - m) / tp1;
      mean[j] = nm;
      mean32[j] = (float)nm;
      mv += (nm - m) * (nm - m);
    }
  }
  mv = block_sum_d(mv, s_red);
  if (threadIdx.x == 0) {
    if (better) hdr->best_f = f;
    hdr->hint = fmin(minP - s1b, -maxQ - s2b);
    if (advance) {
      const double n1 = s1b + (s1 - s1b) / tp1, n2 = s2b + (s2 - s2b) / tp1;
      hdr->move = D * sqrt(mv) + fmax(fabs(n1 - s1b), fabs(n2 - s2b));
      hdr->s1bar = n1;
      hdr->s2bar = n2;
      hdr->t = t + 1;
    } else {
      hdr->move = 0.0;
    }
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
      o.lower_bound = f;
      o.upper_bound = UB;
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
