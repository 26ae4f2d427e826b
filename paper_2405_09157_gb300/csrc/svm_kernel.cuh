// SVM iteration kernel: one streaming pass over the labelled points per MWU
// iteration of the minimisation variant (Sec. 3, Eq. min_implement) for the
// data of Eq. (svm_dual_scp), K = R^n_+ (Sec. 4.2), finished by the last CTA
// to complete (compensated FP32 column totals, an FP32 O(d) finish in one
// warp, the running means kept in FP64).
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
  int single;            // completion stages all partial rows in shared memory (single_level)
  pdscp_step_out* out;
  float2* row_out;       // non-null: a shard's pass; write the column totals here, no finish
  unsigned char* sink;   // non-null: warm-up warps run the finish's code early, writing here
  float* tape;           // non-null: the finish records entry t (svm_tape_stride floats) for a reverse sweep
  int fx;                // completion through the fixed-point column accumulators (fx_push / fx_finish)
  unsigned int wait_limit;  // staged kernels: tries per wait for a bulk copy before giving up (kWaitLimit)
};

// Scale exponents of the fixed-point completion for the SVM columns [S_P, S_Q,
// minP, maxQ, Z_P (dp), Z_Q (dp)]: every shifted exponential is <= 1, so
// S_P, S_Q <= n and |Z_.j| <= n D (D the largest point norm); bounds doubled
// for rounding. A pass that breaks them (a D below the true largest norm,
// NaN or Inf inputs) falls back to the row reduction.
struct SvmFxExp {
  int eS, eZ;
  __device__ int operator()(int pc) const { return pc < 2 ? eS : eZ; }
};
__device__ __forceinline__ SvmFxExp svm_fx_exp(int64_t n, double D) {
  const double nn = (double)n;
  return SvmFxExp{fx_exp(2.0 * nn), fx_exp(2.0 * nn * fabs(D) + 1.0)};
}
__device__ __forceinline__ int svm_col_op(int pc) { return pc == 2 ? 2 : (pc == 3 ? 1 : 0); }  // minP min, maxQ max
// S_P and S_Q divide (Tr mu = S_P/S, the Claim 8 vector Z_P/S_P - Z_Q/S_Q): one
// class's sum can be exponentially smaller than the bound, then the rows are reduced
__device__ __forceinline__ bool svm_col_rel(int pc) { return pc < 2; }
__device__ __forceinline__ void svm_emit(const SvmParams& p, float* prow, const SvmFxExp& fe, int pc, float v) {
  prow[pc] = v;
  if (p.fx) fx_push(fx_cols(p.counter, svm_partial_stride(p.d)), pc, svm_col_op(pc), fe(pc), v, svm_col_rel(pc));
}

// Warm-up of the finish's code path in every CTA (see ses_finish_warm).
static __device__ __noinline__ void svm_finish_warm(const SvmParams& p, unsigned char* smem_raw);

template <typename T>
__device__ void svm_finish(const SvmParams& p, unsigned char* smem_raw, const SvmFxExp& fe);

template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) svm_iter_kernel(SvmParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float s_sc[kWarps][4];

  pdl_trigger();
  pdl_wait();  // the state below is the previous launch's output
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
  const WarpSplit ws(p.sink, kWarps, warp);
  if (ws.warm) svm_finish_warm(p, smem_raw);
  const int64_t nwarps = ws.nwarps;
  const int64_t gw = ws.warm ? (p.n + nwarps * (PPW * U)) : ws.gw;  // the warm-up warp streams nothing
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
  const SvmFxExp fe = svm_fx_exp(p.n, p.D);
  float* prow = p.partials + (size_t)blockIdx.x * svm_partial_stride(d);
  for (int j = threadIdx.x; j < d; j += kBlock) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < kWarps; ++w) {
      a += sZ[w * 2 * dp + j];
      b += sZ[w * 2 * dp + dp + j];
    }
    svm_emit(p, prow, fe, 4 + j, a);
    svm_emit(p, prow, fe, 4 + dp + j, b);
  }
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, mn = INFINITY, mx = -INFINITY;
    for (int w = 0; w < kWarps; ++w) {
      a += s_sc[w][0];
      b += s_sc[w][1];
      mn = fminf(mn, s_sc[w][2]);
      mx = fmaxf(mx, s_sc[w][3]);
    }
    svm_emit(p, prow, fe, 0, a);
    svm_emit(p, prow, fe, 1, b);
    svm_emit(p, prow, fe, 2, mn);
    svm_emit(p, prow, fe, 3, mx);
  }
  svm_finish<T>(p, smem_raw, fe);
}

// The O(d) finish of one SVM iteration from the column totals: run by one
// warp (lane = threadIdx.x & 31). raw: [S_P, S_Q, minP, maxQ, Z_P (dp),
// Z_Q (dp)] as compensated pairs; s_mean: the mean read by the pass (FP64,
// shared memory); h: a copy of the state header. Writes the state and the
// step record (out, may be null). FP32 math, FP64 running means (as in
// ses_finish_warp).
// s_dual (may be null: no averaged bound): the state's zbar, read beforehand
// into shared memory; with it the averaged Claim 8 upper bound is advanced.
static __device__ __noinline__ void svm_finish_warp(const float2* raw, const double* s_mean, const StateHdr& h,
                                             void* state, int d, double alpha_d, double D_d, double eta_over_rho,
                                             int eval_only, pdscp_step_out* out, float* tape = nullptr,
                                             const double* s_dual = nullptr, int forced_status = PDSCP_OK) {
  const int lane = threadIdx.x & 31;
  const int dp = dpad4(d);
  StateHdr* hdr = reinterpret_cast<StateHdr*>(state);
  double* mean = state_mean(state);
  float* mean32 = state_mean32(state, d);
  float* best = state_best(state, d);
  auto tot = [&](int pc) { return raw[pc].x + raw[pc].y; };
  const float SP = tot(0), SQ = tot(1), minP = raw[2].x, maxQ = raw[3].x;
  const float S = SP + SQ;
  const float rS = 1.0f / S;
  const float rSP = SP > 0.f ? 1.0f / SP : 0.f, rSQ = SQ > 0.f ? 1.0f / SQ : 0.f;
  const float trmu = SP * rS, trga = SQ * rS;
  const float alpha = (float)alpha_d, D = (float)D_d;
  const double s1b = h.s1bar, s2b = h.s2bar;
  const int64_t t = h.t;
  // Averaged Claim 8 bound: zbar, the average over the alpha-FTP of the vectors
  // P mu/Tr mu - Q gamma/Tr gamma (iterate t weighted by t^2), is again such a
  // vector for the averaged class-normalised weights, so OPT <= |zbar|.
  const bool qp = s_dual != nullptr;
  const bool qpu = qp && !eval_only && t >= 1 && SP > 0.f && SQ > 0.f;
  const double wt = (double)t * (double)t;
  const double wsum = h.dual_w + (qpu ? wt : 0.0);
  const double rw = qpu ? wt * recip_d(wsum) : 0.0;  // Newton-refined reciprocal: FP64 divide is slow here
  double* zbar = state_dual(state, d);
  // |z|^2, Claim 8 |P mu/Tr mu - Q gamma/Tr gamma|^2, |wbar|^2, z . wbar, |zbar|^2
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int j = lane; j < d; j += 32) {
    const float zp = tot(4 + j), zq = tot(4 + dp + j);
    const float z = (zp - zq) * rS;
    const float df = zp * rSP - zq * rSQ;
    const float m = (float)s_mean[j];
    acc[0] = fmaf(z, z, acc[0]);
    acc[1] = fmaf(df, df, acc[1]);
    acc[2] = fmaf(m, m, acc[2]);
    acc[3] = fmaf(z, m, acc[3]);
    if (qp) {
      double b = s_dual[j];
      if (qpu) {
        b += rw * (double)(df - (float)b);
        zbar[j] = b;
      }
      acc[4] = fmaf((float)b, (float)b, acc[4]);
    }
  }
  warp_sum_kf<5>(acc);
  const float UBq = (qp && wsum > 0.0) ? sqrtf(acc[4]) : INFINITY;
  const float rnz = acc[0] > 0.f ? 1.0f / sqrtf(acc[0]) : 0.f;
  const float nz = acc[0] * rnz;
  const float s1 = (trmu <= trga) ? D : alpha - D;
  const float s2 = alpha - s1;
  const float V = nz - trmu * s1 - trga * s2;                           // Eq. (svm_oracle)
  const float UB = (SP > 0.f && SQ > 0.f) ? sqrtf(acc[1]) : INFINITY;  // Claim 8
  const float rnw = acc[2] > 0.f ? 1.0f / sqrtf(acc[2]) : 0.f;
  const float f = acc[2] > 0.f ? fmaxf((minP - maxQ) * rnw, 0.f) : 0.f;  // Sec. 5
  const float wscale = rS * rnz;                                        // w = (Z_P - Z_Q) wscale
  const double fd = (double)f;

  int status = PDSCP_OK;
  if (!(S > 0.f) || !isfinite(S) || !isfinite(V)) status = PDSCP_ERR_NUMERIC;
  if (forced_status != PDSCP_OK) status = forced_status;  // a staged pass whose copy wait gave up
  bool stop = false, failed = false;
  int outcome = PDSCP_OUT_RUNNING;
  const bool better = fd > h.best_f;
  int streak = h.streak;
  bool set_fprev = false;
  if (!eval_only) {
    failed = V < 0.f;
    if (status != PDSCP_OK) {
      stop = true;
    } else if (failed) {
      stop = true;
      outcome = PDSCP_OUT_SEPARATED;
    } else if (h.rules == PDSCP_RULES_PRACTICAL && t > 0) {
      if (fd > alpha_d) {
        stop = true;
        outcome = PDSCP_OUT_BEAT_ALPHA;
      } else {
        const double fp = h.f_prev;
        if (fp > 0.0) {
          streak = (fabs(fd - fp) < h.delta * fp) ? streak + 1 : 0;  // |df|/f < delta, f > 0 (no FP64 divide)
          if (streak >= h.patience) {
            stop = true;
            outcome = PDSCP_OUT_STALLED;
          }
        }
        set_fprev = !stop;
      }
    }
  }
  const bool advance = !eval_only && !stop;
  const float rtp1 = 1.0f / (float)(t + 1);
  for (int j = lane; j < d; j += 32) {
    const double m = s_mean[j];
    if (better) best[j] = (float)m;
    if (advance) {
      const float w = (tot(4 + j) - tot(4 + dp + j)) * wscale;
      const double nm = m + (double)((w - (float)m) * rtp1);
      mean[j] = nm;
      mean32[j] = (float)nm;
    }
  }
  if (tape && advance) {
    // what the pass used (same expressions as the pass kernels) and what it produced
    float* ent = tape + (size_t)t * svm_tape_stride(d);
    for (int j = lane; j < d; j += 32) {
      ent[8 + j] = (float)s_mean[j];
      ent[8 + dp + j] = (tot(4 + j) - tot(4 + dp + j)) * rS;
    }
    if (lane == 0) {
      ent[0] = S;
      ent[1] = nz;
      ent[2] = (float)((double)t * eta_over_rho);
      ent[3] = (float)(h.hint - h.move);
      ent[4] = (float)h.s1bar;
      ent[5] = (float)h.s2bar;
      ent[6] = 0.f;
      ent[7] = 0.f;
    }
  }
  if (lane == 0) {
    const double ubn = (double)fminf(UB, UBq);
    if (!eval_only && ubn < h.ub_best) hdr->ub_best = ubn;
    if (qpu) hdr->dual_w = wsum;
    if (streak != h.streak) hdr->streak = streak;
    if (set_fprev) hdr->f_prev = fd;
    if (better) hdr->best_f = fd;
    hdr->hint = fmin((double)minP - s1b, -(double)maxQ - s2b);
    const int64_t tn = t + (advance ? 1 : 0);
    if (advance) {
      // ||w - wbar||^2 = |w|^2 - 2 w.wbar + |wbar|^2, |w| = 1 (or w = 0)
      const float ww = acc[0] > 0.f ? 1.f : 0.f;
      const float mv2 = ww - 2.f * acc[3] * rnz + acc[2];
      const double n1 = s1b + (double)((s1 - (float)s1b) * rtp1);
      const double n2 = s2b + (double)((s2 - (float)s2b) * rtp1);
      hdr->move = ((double)(D * rtp1 * sqrtf(fmaxf(mv2, 0.f))) + fmax(fabs(n1 - s1b), fabs(n2 - s2b))) * (1.0 + 1e-5);
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
    hdr->last_value = (double)V;
    if (out) {
      pdscp_step_out o;
      o.oracle_value = (double)V;
      o.objective = fd;
      o.lower_bound = fd;
      o.upper_bound = (double)UB;
      o.t = tn;
      o.failed = failed ? 1 : 0;
      o.stopped = (stop || h.stopped) ? 1 : 0;
      o.status = status;
      o.outcome = outcome;
      o.k = (double)t * eta_over_rho;
      o.dual_bound = (double)UBq;
      *out = o;
    }
  }
}

static __device__ __noinline__ void svm_finish_warm(const SvmParams& p, unsigned char* smem_raw) {
  const int d = p.d;
  const float2* raw = reinterpret_cast<const float2*>(smem_raw);
  const double* s_mean = reinterpret_cast<const double*>(smem_raw) + svm_partial_stride(d);
  StateHdr h;
  memset(&h, 0, sizeof(h));
  svm_finish_warp(raw, s_mean, h, p.sink, d, p.alpha, p.D, p.eta_over_rho, p.eval_only, warm_sink_out(p.sink, d),
                  p.tape ? warm_sink_tape(p.sink, d) : nullptr, s_mean + dpad4(d));
}

// O(d) finish of one SVM iteration. Every CTA calls it after writing its
// partial row [S_P, S_Q, minP, maxQ, Z_P (dp), Z_Q (dp)]; the completion
// elects one CTA, which reduces the rows and hands the totals to warp 0.
template <typename T>
__device__ void svm_finish(const SvmParams& p, unsigned char* smem_raw, const SvmFxExp& fe) {
  __shared__ float2 s_scr[kMaxBlock];
  __shared__ __align__(16) double s_hdr[sizeof(StateHdr) / 8];
  __shared__ bool s_flag;
  const int d = p.d;
  const int dp = dpad4(d);
  const int st = svm_partial_stride(d);
  auto opof = [](int pc) { return svm_col_op(pc); };
  if (p.fx ? !fx_arrive(p.counter, &s_flag)
           : !arrive_pass(p.partials, st, p.grows, p.counter, s_scr, &s_flag, opof, p.single))
    return;

  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  double* mean = state_mean(p.state);
  const int tid = threadIdx.x;
  // dynamic shared memory: column totals as (s, c) pairs | mean | zbar | staged partial rows
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  double* s_mean = reinterpret_cast<double*>(smem_raw) + st;
  double* s_dual = s_mean + dp;
  float* stage = reinterpret_cast<float*>(s_dual + dp);
  const double* dual = state_dual(p.state, d);
  // the FP64 header, mean and zbar go straight into shared memory before the
  // reduction (cp.async: their latency overlaps it, no register is held)
  constexpr int HW = (int)(sizeof(StateHdr) / 8);
  if (tid < HW) cp_async8(s_hdr + tid, reinterpret_cast<const double*>(hdr) + tid);
  for (int j = tid; j < d; j += blockDim.x) {
    cp_async8(s_mean + j, mean + j);
    cp_async8(s_dual + j, dual + j);
  }
  if (p.fx)
    fx_finish(p.counter, p.partials, st, raw, s_scr, fe, opof);
  else
    final_reduce(p.partials, st, p.grows, p.counter, s_scr, opof, raw, stage, p.single, 3, 2, st);
  cp_async_wait_all();
  unsigned int* tmo = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(p.counter) + kTimeoutFlagOff);
  const bool timed_out = __ldcg(tmo) != 0u;
  __syncthreads();
  if (timed_out && tid == 0) *tmo = 0u;
  if (p.row_out) {  // a shard of a row-sharded iteration: hand the totals to the merge
    for (int pc = tid; pc < st; pc += blockDim.x)  // a timed-out pass hands on S_P = NaN: the merge reports it
      p.row_out[pc] = (timed_out && pc == 0) ? make_float2(NAN, 0.f) : raw[pc];
    return;
  }
  // The O(d) math runs in the last warp alone (see ses_finish).
  if ((int)(tid >> 5) != (int)(blockDim.x >> 5) - 1) return;
  svm_finish_warp(raw, s_mean, *reinterpret_cast<const StateHdr*>(s_hdr), p.state, d, p.alpha, p.D,
                  p.eta_over_rho, p.eval_only, p.out, p.tape, s_dual, timed_out ? PDSCP_ERR_TIMEOUT : PDSCP_OK);
}

}  // namespace pdscp

namespace pdscp {

// Vector-path form of svm_iter_kernel for rows of at most 32 chunks (see
// ses_iter_t_kernel): the partial dot products x_i^T wbar are
// reduce-scattered so that one lane per point forms the margin, the label
// test and the exponential; the signed weight y_i e^{...} is broadcast back
// for the per-class weighted sums Z_P, Z_Q.
//
// NS = 0: rounds loaded into registers; NS >= 2: rounds staged through a
// per-warp ring of NS shared-memory slots filled by bulk copies, bounded waits
// (as ses_iter_t_kernel).
template <typename T, int VW, int LPP, int NI, int BLOCK, int NS>
__global__ void __launch_bounds__(BLOCK, 1) svm_iter_t_kernel(SvmParams p) {
  using GS = GroupScatter<LPP, NI>;
  constexpr int NW = BLOCK / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float s_sc[NW][4];
  __shared__ uint64_t s_bar[NS > 0 ? NW * NS : 1];

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = d / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  const bool owner = (gl % GS::SHARE) == 0;
  const bool has_chunk = gl < nch;
  const T* pts = reinterpret_cast<const T*>(p.pts);
  pdl_trigger();
  const WarpSplit wsp(p.sink, NW, warp);
  if (wsp.warm) svm_finish_warm(p, smem_raw);
  const int64_t nwarps = wsp.nwarps;
  const int64_t gw = wsp.gw;
  constexpr int ROUND = PPW * NI;
  // each warp streams one contiguous range of points, equal up to 8 points
  // (balanced bytes per warp; starts on 8-point boundaries)
  auto split = [&](int64_t w) { return w >= nwarps ? p.n : ((w * p.n / nwarps) & ~(int64_t)7); };
  const int64_t lo = wsp.warm ? p.n : split(gw), hi = wsp.warm ? p.n : split(gw + 1);
  // the first round's point loads do not depend on the state: issue them first
  float x[NI][VW];
  // BF16 staged rounds are widened into float pairs for paired FP32
  // arithmetic in the dot products and the class sums (n = 1e6, d = 128,
  // back to back: 55.9 -> 53.7 us)
  constexpr bool kPair = sizeof(T) == 2 && NS > 0;
  unsigned long long x2[kPair ? NI : 1][kPair ? VW / 2 : 1];
  auto load_round = [&](int64_t base) {
#pragma unroll
    for (int r = 0; r < NI; ++r) {
        const int64_t i = base + r * PPW + grp;
        if (i < hi && has_chunk) {
          Chunk<T, VW>::load(pts + i * d, gl, x[r]);
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e) x[r][e] = 0.f;
        }
      }
  };
  constexpr int SLOT = 32 * NI * VW * (int)sizeof(T);  // >= ROUND * d * sizeof(T)
  unsigned char* ring = smem_raw + (size_t)warp * (NS > 0 ? NS : 1) * SLOT;
  uint64_t* bar = s_bar + (NS > 0 ? warp * NS : 0);
  auto issue = [&](int kk, int64_t b) {  // lane 0: round starting at row b into slot kk
    const int64_t m = hi - b < ROUND ? hi - b : ROUND;
    bulk_load(ring + kk * SLOT, pts + b * d, (unsigned int)(m * d * (int64_t)sizeof(T)), bar + kk);
  };
  if constexpr (NS > 0) {
    // NS - 1 rounds before the wait for the previous launch, as in ses_iter_t_kernel
    if (lane == 0 && lo < hi) {
#pragma unroll
      for (int kk = 0; kk < NS; ++kk) mbar_init(bar + kk, 1);
      mbar_init_fence();
#pragma unroll
      for (int kk = 0; kk < NS - 1; ++kk)
        if (lo + kk * ROUND < hi) issue(kk, lo + kk * ROUND);
    }
    __syncwarp();
  } else {
    load_round(lo);
  }
  auto read_round = [&](int64_t base, int kk) {
    const unsigned char* sl = ring + kk * SLOT;
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int64_t i = base + r * PPW + grp;
      const uint4 v = (i < hi && has_chunk)
                          ? *reinterpret_cast<const uint4*>(sl + ((size_t)(r * PPW + grp) * d) * sizeof(T) + gl * 16)
                          : make_uint4(0u, 0u, 0u, 0u);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
      if constexpr (sizeof(T) == 2 && NS > 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x2[r][j] = f2_from_bf16x2(w[j]);
      } else if constexpr (sizeof(T) == 2) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // bf16 -> fp32 is a 16-bit left shift of the bit pattern
          x[r][2 * j] = __uint_as_float(w[j] << 16);
          x[r][2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[r][j] = __uint_as_float(w[j]);
      }
    }
  };
  auto drain = [&](int r0) {
    if constexpr (NS > 0) {
      const unsigned int lim = p.wait_limit > kWaitLimit ? p.wait_limit : kWaitLimit;
#pragma unroll
      for (int j = 0; j < NS; ++j)
        if (lo + (int64_t)(r0 + j) * ROUND < hi) mbar_wait(bar + (r0 + j) % NS, (unsigned int)((r0 + j) / NS) & 1u, lim);
    }
  };
  bool timed_out = false;
  // BF16 rows (register rounds): lane 0 of each warp asks L2 for the next
  // round ahead of its loads, as in ses_iter_t_kernel (measured at n = 1e6,
  // d = 128: 86.6 -> 71.7 us; FP32 is 2.5 us slower with it, so not done there)
  auto prefetch_round = [&](int64_t b) {
    if constexpr (sizeof(T) == 2 && NS == 0) {
      if (lane == 0 && b < hi) {
        const int64_t m = hi - b < ROUND ? hi - b : ROUND;
        const unsigned int bytes = (unsigned int)(m * d * (int64_t)sizeof(T));  // whole 16-byte chunks
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(pts + b * d), "r"(bytes) : "memory");
      }
    }
  };

  // the first round's loads are in flight; everything below depends on the
  // previous launch (state, partial rows, counters)
  pdl_wait();
  if constexpr (NS > 0) {
    if (lane == 0 && lo + (NS - 1) * ROUND < hi) issue(NS - 1, lo + (NS - 1) * ROUND);
  }
  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  if (hdr->stopped && !p.eval_only) {
    drain(0);
    return;
  }

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
  unsigned long long wb2[kPair ? VW / 2 : 1], ZP2[kPair ? VW / 2 : 1], ZQ2[kPair ? VW / 2 : 1];
#pragma unroll
  for (int q2 = 0; q2 < (kPair ? VW / 2 : 1); ++q2) {
    wb2[q2] = f2_pack(wb[(2 * q2) % VW], wb[(2 * q2 + 1) % VW]);
    ZP2[q2] = 0ull;
    ZQ2[q2] = 0ull;
  }

  int rnd = 0;
  for (int64_t base = lo; base < hi; base += ROUND, ++rnd) {
    const int ks = NS > 0 ? rnd % (NS > 0 ? NS : 1) : 0;
    if constexpr (NS > 0) {
      if (!mbar_wait(bar + ks, (unsigned int)(rnd / (NS > 0 ? NS : 1)) & 1u, p.wait_limit)) {
        timed_out = true;
        break;
      }
      read_round(base, ks);
    } else {
      prefetch_round(base + ROUND);
      if (base != lo) load_round(base);
    }
    float part[NI];
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      float a = 0.f;
      if constexpr (kPair) {
        unsigned long long acc = 0ull;
#pragma unroll
        for (int q2 = 0; q2 < VW / 2; ++q2) acc = f2_fma(x2[r][q2], wb2[q2], acc);
        float lo2, hi2;
        f2_unpack(acc, lo2, hi2);
        a = lo2 + hi2;
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) a = fmaf(x[r][e], wb[e], a);
      }
      part[r] = a;
    }
    GS::run(part, gl);
    float q[GS::OWN];  // y_i e^{-k (m_i - Hm)}, signed by the label
#pragma unroll
    for (int kk = 0; kk < GS::OWN; ++kk) {
      const int64_t i = base + GS::owned(gl, kk) * PPW + grp;
      q[kk] = 0.f;
      if (i < hi) {
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
      if constexpr (kPair) {
        const unsigned long long qp2 = f2_pack(qp, qp), qq2 = f2_pack(qq, qq);
#pragma unroll
        for (int q2 = 0; q2 < VW / 2; ++q2) {
          ZP2[q2] = f2_fma(qp2, x2[r][q2], ZP2[q2]);
          ZQ2[q2] = f2_fma(qq2, x2[r][q2], ZQ2[q2]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          ZP[e] = fmaf(qp, x[r][e], ZP[e]);
          ZQ[e] = fmaf(qq, x[r][e], ZQ[e]);
        }
      }
    }
    if constexpr (NS > 0) {
      __syncwarp();  // every lane has read slot ks: refill it with the round NS ahead
      if (lane == 0 && base + NS * ROUND < hi) {
        fence_proxy_async_smem();
        issue(ks, base + NS * ROUND);
      }
    }
  }
  if constexpr (NS > 0) {
    if (timed_out) {
      drain(rnd);
      if (lane == 0) atomicOr(reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(p.counter) + kTimeoutFlagOff), 1u);
    }
    __syncthreads();  // every warp is done with its ring before the shared memory is reused
  }

  if constexpr (kPair) {
#pragma unroll
    for (int q2 = 0; q2 < VW / 2; ++q2) {
      f2_unpack(ZP2[q2], ZP[2 * q2], ZP[(2 * q2 + 1) % VW]);
      f2_unpack(ZQ2[q2], ZQ[2 * q2], ZQ[(2 * q2 + 1) % VW]);
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
  const SvmFxExp fe = svm_fx_exp(p.n, p.D);
  float* prow = p.partials + (size_t)blockIdx.x * svm_partial_stride(d);
  for (int j = threadIdx.x; j < d; j += BLOCK) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < NW; ++w) {
      a += sZ[w * 2 * dp + j];
      b += sZ[w * 2 * dp + dp + j];
    }
    svm_emit(p, prow, fe, 4 + j, a);
    svm_emit(p, prow, fe, 4 + dp + j, b);
  }
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, mn = INFINITY, mx = -INFINITY;
    for (int w = 0; w < NW; ++w) {
      a += s_sc[w][0];
      b += s_sc[w][1];
      mn = fminf(mn, s_sc[w][2]);
      mx = fmaxf(mx, s_sc[w][3]);
    }
    svm_emit(p, prow, fe, 0, a);
    svm_emit(p, prow, fe, 1, b);
    svm_emit(p, prow, fe, 2, mn);
    svm_emit(p, prow, fe, 3, mx);
  }
  svm_finish<T>(p, smem_raw, fe);
}

}  // namespace pdscp

namespace pdscp {

// Row-sharded iteration, second half, for SVM (see ses_merge_kernel): the
// shards' column totals, `ranks` rows of svm_partial_stride(d) pairs in rank
// order, reduced in that order, then the O(d) finish. One CTA.
struct SvmMergeParams {
  const float2* rows;
  int ranks;
  int d;
  int eval_only;
  double alpha;
  double eta_over_rho;
  double D;
  void* state;
  pdscp_step_out* out;
};

constexpr int kSvmMergeBlock = 256;

template <int kUnused = 0>  // a template so that only the launching unit instantiates it
__global__ void __launch_bounds__(kSvmMergeBlock) svm_merge_kernel(SvmMergeParams m) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float2 s_scr[kSvmMergeBlock];
  __shared__ __align__(16) double s_hdr[sizeof(StateHdr) / 8];
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(m.state);
  if (hdr->stopped && !m.eval_only) return;
  const int d = m.d, st = svm_partial_stride(d);
  const int tid = threadIdx.x;
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  double* s_mean = reinterpret_cast<double*>(smem_raw) + st;
  double* s_dual = s_mean + dpad4(d);
  constexpr int HW = (int)(sizeof(StateHdr) / 8);
  if (tid < HW) s_hdr[tid] = reinterpret_cast<const double*>(hdr)[tid];
  const double* mean = state_mean(m.state);
  const double* dual = state_dual(m.state, d);
  for (int j = tid; j < d; j += blockDim.x) {
    s_mean[j] = mean[j];
    s_dual[j] = dual[j];
  }
  auto opof = [](int pc) { return pc == 2 ? 2 : (pc == 3 ? 1 : 0); };
  reduce_rows(m.rows, 0, m.ranks, st, raw, s_scr, opof);  // ends with a barrier
  if (tid >= 32) return;
  svm_finish_warp(raw, s_mean, *reinterpret_cast<const StateHdr*>(s_hdr), m.state, d, m.alpha, m.D,
                  m.eta_over_rho, m.eval_only, m.out, nullptr, s_dual);
}

}  // namespace pdscp
