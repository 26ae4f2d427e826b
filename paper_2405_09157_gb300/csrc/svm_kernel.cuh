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
// value ||z|| - Tr(mu) s_1 - Tr(gamma) s_2. Claim 8's PD value is
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
  float* partials;       // one row of svm_partial_stride(d) floats per CTA
  float2* grows;         // one compensated-FP32 row per completion group
  unsigned int* counter; // completion counters: [0] top, [1 + g] group g
  pdscp_step_out* out;
};

template <typename T>
__device__ void svm_finish(const SvmParams& p, unsigned char* smem_raw);

template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) svm_iter_kernel(SvmParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_sc[kWarps][4];

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
  svm_finish<T>(p, smem_raw);
}

// O(d) finish of one SVM iteration. Every CTA calls it after writing its
// partial row [S_P, S_Q, minP, maxQ, Z_P (dp), Z_Q (dp)]; the two-level
// completion elects one CTA, which reduces the group rows in FP64 and does
// the rest.
template <typename T>
__device__ void svm_finish(const SvmParams& p, unsigned char* smem_raw) {
  __shared__ float2 s_scr[kBlock];
  __shared__ __align__(16) double s_hdr[sizeof(StateHdr) / 8];
  __shared__ bool s_flag;
  const int d = p.d;
  const int dp = dpad4(d);
  const int st = svm_partial_stride(d);
  auto opof = [](int pc) { return pc == 2 ? 2 : (pc == 3 ? 1 : 0); };  // minP min, maxQ max
  if (!arrive_two_level(p.partials, st, p.grows, p.counter, s_scr, &s_flag, opof)) return;

  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  double* mean = state_mean(p.state);
  float* mean32 = state_mean32(p.state, d);
  float* best = state_best(p.state, d);
  const int tid = threadIdx.x;
  // dynamic shared memory: column totals as (s, c) pairs | mean
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  double* s_mean = reinterpret_cast<double*>(smem_raw) + st;
  constexpr int HW = (int)(sizeof(StateHdr) / 8);
  const double hw = tid < HW ? reinterpret_cast<const double*>(hdr)[tid] : 0.0;
  const double m0 = tid < d ? mean[tid] : 0.0;
  const int nb = gridDim.x;
  const int G = (nb + group_size(nb) - 1) / group_size(nb);
  reduce_rows(p.grows, 0, G, st, raw, s_scr, opof);
  if (tid < HW) s_hdr[tid] = hw;
  if (tid < d) s_mean[tid] = m0;
  for (int j = tid + blockDim.x; j < d; j += blockDim.x) s_mean[j] = mean[j];
  __syncthreads();
  // The O(d) math runs in warp 0 alone (see ses_finish).
  if (tid >= 32) return;
  const int lane = tid;
  const StateHdr& h = *reinterpret_cast<const StateHdr*>(s_hdr);
  auto tot = [&](int pc) { return (double)raw[pc].x + (double)raw[pc].y; };
  const double SP = tot(0), SQ = tot(1), minP = (double)raw[2].x, maxQ = (double)raw[3].x;
  const double S = SP + SQ;
  const double rS = recip_d(S);
  const double rSP = SP > 0.0 ? recip_d(SP) : 0.0, rSQ = SQ > 0.0 ? recip_d(SQ) : 0.0;
  const double trmu = SP * rS, trga = SQ * rS;
  const double alpha = p.alpha, D = p.D;
  const double s1b = h.s1bar, s2b = h.s2bar;
  // |z|^2, Claim 8 |P mu/Tr mu - Q gamma/Tr gamma|^2, |wbar|^2, z . wbar
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = lane; j < d; j += 32) {
    const double zp = tot(4 + j), zq = tot(4 + dp + j);
    const double z = (zp - zq) * rS;
    const double df = zp * rSP - zq * rSQ;
    const double m = s_mean[j];
    acc[0] += z * z;
    acc[1] += df * df;
    acc[2] += m * m;
    acc[3] += z * m;
  }
  warp_sum_k<4>(acc);
  const double rnz = acc[0] > 0.0 ? rsqrt_d(acc[0]) : 0.0;
  const double nz = acc[0] * rnz;
  const double s1 = (trmu <= trga) ? D : alpha - D;
  const double s2 = alpha - s1;
  const double V = nz - trmu * s1 - trga * s2;                           // Eq. (svm_oracle)
  const double UB = (SP > 0.0 && SQ > 0.0) ? sqrt_d(acc[1]) : INFINITY;  // Claim 8
  const double rnw = acc[2] > 0.0 ? rsqrt_d(acc[2]) : 0.0;
  const double f = acc[2] > 0.0 ? fmax((minP - maxQ) * rnw, 0.0) : 0.0;  // Sec. 5
  const double wscale = rS * rnz;                                        // w = (Z_P - Z_Q) wscale

  const int64_t t = h.t;
  int status = PDSCP_OK;
  if (!(S > 0.0) || !isfinite(S) || !isfinite(V)) status = PDSCP_ERR_NUMERIC;
  bool stop = false, failed = false;
  int outcome = PDSCP_OUT_RUNNING;
  const bool better = f > h.best_f;
  int streak = h.streak;
  bool set_fprev = false;
  if (!p.eval_only) {
    failed = V < 0.0;
    if (status != PDSCP_OK) {
      stop = true;
    } else if (failed) {
      stop = true;
      outcome = PDSCP_OUT_SEPARATED;
    } else if (h.rules == PDSCP_RULES_PRACTICAL && t > 0) {
      if (f > alpha) {
        stop = true;
        outcome = PDSCP_OUT_BEAT_ALPHA;
      } else {
        const double fp = h.f_prev;
        if (fp > 0.0) {
          streak = (fabs(f - fp) / fp < h.delta) ? streak + 1 : 0;
          if (streak >= h.patience) {
            stop = true;
            outcome = PDSCP_OUT_STALLED;
          }
        }
        set_fprev = !stop;
      }
    }
  }
  const bool advance = !p.eval_only && !stop;
  const double rtp1 = recip_d((double)t + 1.0);
  for (int j = lane; j < d; j += 32) {
    const double m = s_mean[j];
    if (better) best[j] = (float)m;
    if (advance) {
      const double w = (tot(4 + j) - tot(4 + dp + j)) * wscale;
      const double nm = m + (w - m) * rtp1;
      mean[j] = nm;
      mean32[j] = (float)nm;
    }
  }
  if (lane == 0) {
    if (!p.eval_only && UB < h.ub_best) hdr->ub_best = UB;
    if (streak != h.streak) hdr->streak = streak;
    if (set_fprev) hdr->f_prev = f;
    if (better) hdr->best_f = f;
    hdr->hint = fmin(minP - s1b, -maxQ - s2b);
    const int64_t tn = t + (advance ? 1 : 0);
    if (advance) {
      // ||w - wbar||^2 = |w|^2 - 2 w.wbar + |wbar|^2, |w| = 1 (or w = 0)
      const double ww = acc[0] > 0.0 ? 1.0 : 0.0;
      const double mv2 = ww - 2.0 * acc[3] * rnz + acc[2];
      const double n1 = s1b + (s1 - s1b) * rtp1, n2 = s2b + (s2 - s2b) * rtp1;
      hdr->move = (D * rtp1 * sqrt_d(fmax(mv2, 0.0)) + fmax(fabs(n1 - s1b), fabs(n2 - s2b))) * (1.0 + 1e-6);
      hdr->s1bar = n1;
      hdr->s2bar = n2;
    } else {
      hdr->move = 0.0;
    }
    hdr->t = tn;
    if (stop) {
      hdr->stopped = 1;
      hdr->outcome = outcome;
    }
    if (status != PDSCP_OK) hdr->status = status;
    hdr->last_value = V;
    if (p.out) {
      pdscp_step_out o;
      o.oracle_value = V;
      o.objective = f;
      o.lower_bound = f;
      o.upper_bound = UB;
      o.t = tn;
      o.failed = failed ? 1 : 0;
      o.stopped = (stop || h.stopped) ? 1 : 0;
      o.status = status;
      o.outcome = outcome;
      o.k = (double)t * p.eta_over_rho;
      *p.out = o;
    }
  }
}

}  // namespace pdscp

namespace pdscp {

// Vector-path form of svm_iter_kernel for rows of at most 32 chunks (see
// ses_iter_t_kernel): the partial dot products x_i^T wbar are
// reduce-scattered so that one lane per point forms the margin, the label
// test and the exponential; the signed weight y_i e^{...} is broadcast back
// for the per-class weighted sums Z_P, Z_Q.
template <typename T, int VW, int LPP, int NI>
__global__ void __launch_bounds__(kBlock) svm_iter_t_kernel(SvmParams p) {
  using GS = GroupScatter<LPP, NI>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_sc[kWarps][4];

  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  if (hdr->stopped && !p.eval_only) return;

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = d / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  const bool owner = (gl % GS::SHARE) == 0;
  const bool has_chunk = gl < nch;

  const float k = p.eval_only ? 0.f : (float)((double)hdr->t * p.eta_over_rho);
  const float Hm = (float)(hdr->hint - hdr->move);
  const float s1 = (float)hdr->s1bar, s2 = (float)hdr->s2bar;
  const float* mean32 = state_mean32(p.state, d);

  float wb[VW], ZP[VW], ZQ[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    wb[e] = has_chunk ? mean32[gl * VW + e] : 0.f;
    ZP[e] = 0.f;
    ZQ[e] = 0.f;
  }
  float SP = 0.f, SQ = 0.f, minP = INFINITY, maxQ = -INFINITY;

  const T* pts = reinterpret_cast<const T*>(p.pts);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  constexpr int ROUND = PPW * NI;
  for (int64_t base = gw * ROUND; base < p.n; base += nwarps * ROUND) {
    float x[NI][VW];
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int64_t i = base + r * PPW + grp;
      if (i < p.n && has_chunk) {
        Chunk<T, VW>::load(pts + i * d, gl, x[r]);
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) x[r][e] = 0.f;
      }
    }
    float part[NI];
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      float a = 0.f;
#pragma unroll
      for (int e = 0; e < VW; ++e) a = fmaf(x[r][e], wb[e], a);
      part[r] = a;
    }
    GS::run(part, gl);
    float q[GS::OWN];  // y_i e^{-k (m_i - Hm)}, signed by the label
#pragma unroll
    for (int kk = 0; kk < GS::OWN; ++kk) {
      const int64_t i = base + GS::owned(gl, kk) * PPW + grp;
      q[kk] = 0.f;
      if (i < p.n) {
        const float dot = part[kk];
        const bool pos = __ldg(p.labels + i) > 0;
        const float margin = pos ? dot - s1 : -dot - s2;
        const float pt = expf(-k * (margin - Hm));
        q[kk] = pos ? pt : -pt;
        if (owner) {
          if (pos) {
            SP += pt;
            minP = fminf(minP, dot);
          } else {
            SQ += pt;
            maxQ = fmaxf(maxQ, dot);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const float qr = __shfl_sync(0xffffffffu, q[r % GS::OWN], grp * LPP + GS::src_lane(r));
      const float qp = fmaxf(qr, 0.f), qq = fmaxf(-qr, 0.f);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        ZP[e] = fmaf(qp, x[r][e], ZP[e]);
        ZQ[e] = fmaf(qq, x[r][e], ZQ[e]);
      }
    }
  }

#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      ZP[e] += __shfl_xor_sync(0xffffffffu, ZP[e], o);
      ZQ[e] += __shfl_xor_sync(0xffffffffu, ZQ[e], o);
    }
  SP = warp_sum(SP);
  SQ = warp_sum(SQ);
  minP = warp_min(minP);
  maxQ = warp_max(maxQ);
  float* sZ = reinterpret_cast<float*>(smem_raw);
  if (grp == 0 && has_chunk)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      sZ[warp * 2 * dp + gl * VW + e] = ZP[e];
      sZ[warp * 2 * dp + dp + gl * VW + e] = ZQ[e];
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
  svm_finish<T>(p, smem_raw);
}

}  // namespace pdscp
