// SES iteration kernel: one streaming pass over the points per MWU iteration
// (Sec. 4.1 with the update of Eq. implement and the ORACLE of Eq. ses_oracle),
// finished by the last CTA to complete (compensated FP32 column totals, an
// FP32 O(d) finish in one warp, the running mean kept in FP64).
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
  float* partials;       // one row of ses_partial_stride(d) floats per CTA
  float2* grows;         // one compensated-FP32 row per completion group
  unsigned int* counter; // completion counters: [0] top, [1 + g] group g
  int single;            // completion stages all partial rows in shared memory (single_level)
  pdscp_step_out* out;   // may be null
  int64_t first;         // first row of the pass: 1 when row 0 is v_1 (the easy cone), else 0
  float2* row_out;       // non-null: a shard's pass; write the column totals here, no finish
  float* tape;           // non-null: the finish records entry t (ses_tape_stride floats) for a reverse sweep
  unsigned char* sink;   // non-null: one warp warms the finish's code path early, writing here (warm_sink_bytes)
  int fx;                // completion through the fixed-point column accumulators (fx_push / fx_finish)
  unsigned int wait_limit;  // staged kernels: tries per wait for a bulk copy before giving up (kWaitLimit)
};

// Scale exponents of the fixed-point completion for the SES columns [S, Wt,
// maxd, Cc, G'_1..G'_d], from bounds on their absolute sums over the n points
// that hold for every pass (H = hint + move bounds dist_i + gamma_i; shifted
// exponentials E1 <= 1): S = sum E1 (2 - em) <= 2n; |G'_j| <= sum c_i dist_i
// <= sum (E1 - E2) <= n; c_i <= 2 (k/sqrt2) E1 gives Cc <= 2 (k/sqrt2) n;
// |a_i (E1 + E2) - dist_i (E1 - E2)| <= 2 (|alpha| + H) + H. Each bound is
// doubled for the FP32 rounding of the terms. A pass whose terms break a
// bound (an evaluation pass over spheres with radii far above alpha, NaN or
// Inf inputs) falls back to the row reduction (fx_finish).
struct SesFxExp {
  int eS, eW, eC, eG;
  __device__ int operator()(int pc) const { return pc == 0 ? eS : (pc == 1 ? eW : (pc == 3 ? eC : eG)); }
};
__device__ __forceinline__ SesFxExp ses_fx_exp(int64_t n, float kr, float H, float alpha) {
  const double nn = (double)n;
  return SesFxExp{fx_exp(4.0 * nn), fx_exp(nn * (4.0 * fabs((double)alpha) + 6.0 * fabs((double)H) + 4.0)),
                  fx_exp(4.0 * nn * (double)kr + 1.0), fx_exp(2.0 * nn + 1.0)};
}
__device__ __forceinline__ int ses_col_op(int pc) { return pc == 2 ? 1 : 0; }  // maxd is a max, the rest sums
// S and Cc divide (g = G'/(sqrt2 S), mu_i = c_i/Cc): they need relative precision
__device__ __forceinline__ bool ses_col_rel(int pc) { return pc == 0 || pc == 3; }

// The finish runs once per launch, in one warp, after every other warp is
// done; its instructions are then cold (a flushed or streamed-over L2 holds
// none of them) and fetching them from HBM costs more than its arithmetic.
// The last warp of every CTA streams no points and instead runs the same
// code at the start of the launch, on whatever shared memory holds, writing
// only to the sink: whichever CTA finishes then finds the code in its SM's
// instruction cache.
template <typename T>
__device__ __noinline__ void ses_finish_warm(const SesParams& p, unsigned char* scratch, size_t scratch_bytes);



template <typename T>
__device__ void ses_finish(const SesParams& p, unsigned char* smem_raw, const SesFxExp& fe);

// This CTA's partial row: the FP32 row (always written: the fallback of the
// fixed-point completion and the row-reduction paths read it) and, with
// p.fx, its fixed-point pushes. Column pc's value v is written by one thread.
__device__ __forceinline__ void ses_emit(const SesParams& p, float* prow, const SesFxExp& fe, int pc, float v) {
  prow[pc] = v;
  if (p.fx && !(pc == 3 && p.radii))
    fx_push(fx_cols(p.counter, ses_partial_stride(p.d)), pc, ses_col_op(pc), fe(pc), v, ses_col_rel(pc));
}

// T: element type of the points; VW: elements per chunk; LPP: lanes per point
// (power of two); NCH: chunks per lane; U: points in flight per lane group.
template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) ses_iter_kernel(SesParams p) {
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

  // k/sqrt2; an evaluation pass needs only distances, so it uses k = 0
  const float kr = p.eval_only ? 0.f : ses_kr(hdr->t, p.eta_over_rho);
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
  float S = 0.f, W = 0.f, Cs = 0.f, maxd = -INFINITY;

  const T* pts = reinterpret_cast<const T*>(p.pts);
  const WarpSplit ws(p.sink, kWarps, warp);
  if (ws.warm) ses_finish_warm<T>(p, smem_raw, (size_t)(ses_partial_stride(p.d) + 3 * dpad4(p.d)) * sizeof(double));
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
        for (int e = 0; e < VW; ++e) {
          x[u][j][e] -= ub[j][e];
          part = fmaf(x[u][j][e], x[u][j][e], part);
        }
      const float dist2 = group_sum<LPP>(part);
      float c = 0.f;
      if (i >= p.first && i < p.n) {
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
          Cs += c;
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
  Cs = warp_sum(Cs);
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
    s_sc[warp][3] = Cs;
  }
  __syncthreads();
  const SesFxExp fe = ses_fx_exp(p.n, kr, H, alpha);
  float* prow = p.partials + (size_t)blockIdx.x * ses_partial_stride(d);
  for (int j = threadIdx.x; j < d; j += kBlock) {
    float s = 0.f;
    for (int w = 0; w < kWarps; ++w) s += sG[w * dp + j];
    ses_emit(p, prow, fe, 4 + j, s);
  }
  if (threadIdx.x == 0) {
    float s0 = 0.f, s1 = 0.f, s3 = 0.f, m = -INFINITY;
    for (int w = 0; w < kWarps; ++w) {
      s0 += s_sc[w][0];
      s1 += s_sc[w][1];
      s3 += s_sc[w][3];
      m = fmaxf(m, s_sc[w][2]);
    }
    ses_emit(p, prow, fe, 0, s0);
    ses_emit(p, prow, fe, 1, s1);
    ses_emit(p, prow, fe, 2, m);
    ses_emit(p, prow, fe, 3, p.radii ? NAN : s3);  // the QP bound holds for points only
  }
  ses_finish<T>(p, smem_raw, fe);
}

// The O(d) finish of one SES iteration from the column totals: run by one
// warp (lane = threadIdx.x & 31). raw: [S, Wt, maxd, Cc, G'_1..G'_d] as
// compensated pairs (Cc = sum of the ORACLE coefficients c_i); s_mean, s_v1:
// the mean read by the pass and v_1 (FP64, shared memory); h: a copy of the
// state header. Writes the state and the step record (out, may be null).
// s_dual (may be null: no averaged bound): the state's Bbar, read beforehand
// into shared memory; with it the averaged QP lower bound is advanced (points:
// a pass over spheres leaves Cc = NaN, which switches the update off).
static __device__ __noinline__ void ses_finish_warp(const float2* raw, const double* s_mean, const double* s_v1,
                                             const StateHdr& h, void* state, int d, double alpha_d, double gam1,
                                             double eta_over_rho, int eval_only, pdscp_step_out* out,
                                             float* tape = nullptr, const double* s_dual = nullptr,
                                             int forced_status = PDSCP_OK, int role = 0) {
  const int lane = threadIdx.x & 31;
  StateHdr* hdr = reinterpret_cast<StateHdr*>(state);
  double* mean = state_mean(state);
  float* mean32 = state_mean32(state, d);
  float* best = state_best(state, d);
  const double alpha_in = alpha_d;
  // role 0: the whole finish in this warp; role 1: all but the averaged QP
  // bound; role 2: only the averaged QP bound (Bbar, Abar, its lower bound,
  // lb_best, dual_A, dual_w and the record's dual_bound), run by a second warp
  // at the same time as role 1 (its FP64 chains are the longest of the finish).
  const bool main_part = role != 2;
  // The finish works in FP32 (FP64 is slow here and its dependent chains
  // dominated this step): its inputs are compensated sums accurate to ~1e-7,
  // and its results feed tolerances of 1e-5. FP64 is kept for the running
  // mean, which accumulates over the whole alpha-FTP, for the averaged QP
  // bound's running averages, and for the Sec. 5 ratio test, which decides an
  // integer as the oracle does.
  auto tot = [&](int pc) { return raw[pc].x + raw[pc].y; };
  const float S = tot(0), Wt = tot(1), maxd = raw[2].x;
  const float alpha = (float)alpha_in;
  const float gam1f = (float)gam1;
  const float inv = 1.0f / ((float)kSqrt2 * S);  // g = G' / (sqrt2 S)
  const int64_t t = h.t;
  // Averaged QP bound (Eq. ses_qp; points): the weights mu_i = c_i / Cc of this
  // pass give, about v_1, A_t = sum mu_i |v_i - v_1|^2 and B_t = sum mu_i (v_i -
  // v_1) = G'/Cc - (v_1 - ubar); both are averaged over the alpha-FTP with
  // iterate t weighted by t^2, and OPT^2 >= Abar - |Bbar|^2.
  const float Cc = tot(3);
  const bool qp = s_dual != nullptr && role != 1;
  const bool qpu = qp && !eval_only && t >= 1 && Cc > 0.f && isfinite(Cc);
  const double wt = qpu ? (double)t * (double)t : 0.0;
  const double wsum = h.dual_w + wt;
  const double rw = qpu ? wt * recip_d(wsum) : 0.0;  // Newton-refined reciprocal: FP64 divide is slow here
  const float rCc = qpu ? 1.0f / Cc : 0.f;
  double* bbar = state_dual(state, d);
  // A = |g|^2, B = g . (v_1 - ubar), C = |ubar - v_1|^2, |Bbar|^2
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j = lane; j < d; j += 32) {
    const float gp = tot(4 + j);
    const float g = gp * inv;
    const float dv = (float)(s_v1[j] - s_mean[j]);
    acc[0] = fmaf(g, g, acc[0]);
    acc[1] = fmaf(g, dv, acc[1]);
    acc[2] = fmaf(dv, dv, acc[2]);
    if (qp) {
      double b = s_dual[j];
      if (qpu) {
        b += rw * (double)(fmaf(gp, rCc, -dv) - (float)b);
        bbar[j] = b;
      }
      acc[3] = fmaf((float)b, (float)b, acc[3]);
    }
  }
  if (qp) {
    warp_sum_kf<4>(acc);
  } else {  // no averaged bound in this warp: three sums
    float a3[3] = {acc[0], acc[1], acc[2]};
    warp_sum_kf<3>(a3);
    acc[0] = a3[0];
    acc[1] = a3[1];
    acc[2] = a3[2];
  }
  const float A = acc[0], B = acc[1], C = acc[2];
  const float rad = alpha - gam1f;
  const float rng = A > 0.f ? 1.0f / sqrtf(A) : 0.f;
  const float ng = A * rng;                 // ||g||
  const float step = rad * rng;             // u = v_1 + step g  (u = v_1 when g = 0)
  const float V = B + step * A + Wt * inv;  // g.(u - ubar) + Wt/(sqrt2 S): Eq. (ses_oracle) value
  const float LB = fmaxf(gam1f, alpha - V / (ng + (float)(1.0 / kSqrt2)));  // Eq. (primal_construction)
  if (role != 1) {
    // A_t = (sum c_i dist_i^2 - 2 G'.(v_1 - ubar)) / Cc + |v_1 - ubar|^2, with
    // sum c_i dist_i^2 = alpha S - Wt for points
    const double Abar = qpu ? h.dual_A + rw * ((double)((alpha_d * S - Wt - 2.f * (float)kSqrt2 * S * B) * rCc + C) - h.dual_A)
                            : h.dual_A;
    const float LBq = (qp && wsum > 0.0) ? sqrtf(fmaxf((float)Abar - acc[3], 0.f)) : 0.f;
    if (lane == 0) {
      const double lbn = (double)fmaxf(LB, LBq);
      if (!eval_only && lbn > h.lb_best) hdr->lb_best = lbn;
      if (qpu) {
        hdr->dual_A = Abar;
        hdr->dual_w = wsum;
      }
      if (out) out->dual_bound = (double)LBq;
    }
  }
  if (!main_part) return;
  const float f = fmaxf(maxd, sqrtf(C) + gam1f);                             // f at the mean read (Sec. 5)
  const double fd = (double)f;

  int status = PDSCP_OK;
  if (!(S > 0.f) || !isfinite(S) || !isfinite(V) || !isfinite(f)) status = PDSCP_ERR_NUMERIC;
  if (forced_status != PDSCP_OK) status = forced_status;  // a staged pass whose copy wait gave up
  bool stop = false, failed = false;
  int outcome = PDSCP_OUT_RUNNING;
  const bool better = (t > 0 && fd < h.best_f);
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
      if (fd < alpha_in) {
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
  const float rtp1 = 1.0f / (float)(t + 1);  // 1 / (t + 1)
  for (int j = lane; j < d; j += 32) {
    const double m = s_mean[j];
    if (better) best[j] = (float)m;
    if (advance) {
      const float mf = (float)m;
      const float u = (float)s_v1[j] + step * (tot(4 + j) * inv);
      const double nm = m + (double)((u - mf) * rtp1);
      mean[j] = nm;
      mean32[j] = (float)nm;
    }
  }
  if (tape && advance) {
    // what the pass used (same expressions as the pass kernels) and what it produced
    float* ent = tape + (size_t)t * ses_tape_stride(d);
    const int dp = dpad4(d);
    for (int j = lane; j < d; j += 32) {
      ent[4 + j] = (float)s_mean[j];
      ent[4 + dp + j] = tot(4 + j) * inv;
    }
    if (lane == 0) {
      ent[0] = S;
      ent[1] = ng;
      ent[2] = ses_kr(t, eta_over_rho);
      ent[3] = (float)(h.hint + h.move);
    }
  }
  if (lane == 0) {
    if (streak != h.streak) hdr->streak = streak;
    if (set_fprev) hdr->f_prev = fd;
    if (better) hdr->best_f = fd;
    hdr->hint = (double)maxd;
    // ||ubar^{t+1} - ubar^t|| = ||u - ubar|| / (t+1), ||u - ubar||^2 = C + 2 step B + step^2 A
    const float mv2 = C + 2.f * step * B + step * step * A;
    hdr->move = advance ? (double)(rtp1 * sqrtf(fmaxf(mv2, 0.f))) * (1.0 + 1e-5) : 0.0;
    const int64_t tn = t + (advance ? 1 : 0);
    hdr->t = tn;
    if (stop) {
      hdr->stopped = 1;
      hdr->outcome = outcome;
    }
    if (status != PDSCP_OK) hdr->status = status;
    hdr->last_value = (double)V;
    if (out) {  // field by field: in role 1 the dual_bound is written by the other warp
      out->oracle_value = (double)V;
      out->objective = fd;
      out->lower_bound = (double)LB;
      out->upper_bound = fd;
      out->t = tn;
      out->failed = failed ? 1 : 0;
      out->stopped = (stop || h.stopped) ? 1 : 0;
      out->status = status;
      out->outcome = outcome;
      out->k = (double)t * eta_over_rho;
    }
  }
}

// scratch (scratch_bytes long): shared memory the finish's code reads
// (garbage; other warps may be writing there), never writes.
template <typename T>
__device__ __noinline__ void ses_finish_warm(const SesParams& p, unsigned char* scratch, size_t scratch_bytes) {
  const int d = p.d;
  const int st = ses_partial_stride(d);
  // totals, mean, v_1 and Bbar
  if ((size_t)(st + 3 * dpad4(d)) * sizeof(double) > scratch_bytes) return;
  unsigned char* smem_raw = scratch;
  const float2* raw = reinterpret_cast<const float2*>(smem_raw);
  const double* s_mean = reinterpret_cast<const double*>(smem_raw) + ses_partial_stride(d);
  const double* s_v1 = s_mean + dpad4(d);
  StateHdr h;
  memset(&h, 0, sizeof(h));
  ses_finish_warp(raw, s_mean, s_v1, h, p.sink, d, p.alpha, 0.0, p.eta_over_rho, p.eval_only,
                  warm_sink_out(p.sink, d), p.tape ? warm_sink_tape(p.sink, d) : nullptr, s_v1 + dpad4(d));
}

// Completion of one SES iteration. Every CTA calls it after writing its
// partial row [S, Wt, maxd, Cc, G'_1..G'_d]; the last CTA to arrive reduces
// the rows and hands the totals to warp 0 (ses_finish_warp), or, for a shard
// of a row-sharded iteration, writes them to row_out.
template <typename T>
__device__ void ses_finish(const SesParams& p, unsigned char* smem_raw, const SesFxExp& fe) {
  __shared__ float2 s_scr[kMaxBlock];
  __shared__ __align__(16) double s_hdr[sizeof(StateHdr) / 8];
  __shared__ bool s_flag;
  const int d = p.d;
  const int st = ses_partial_stride(d);
  auto opof = [](int pc) { return ses_col_op(pc); };
  if (p.fx ? !fx_arrive(p.counter, &s_flag)
           : !arrive_pass(p.partials, st, p.grows, p.counter, s_scr, &s_flag, opof, p.single))
    return;

  StateHdr* hdr = reinterpret_cast<StateHdr*>(p.state);
  double* mean = state_mean(p.state);
  float* mean32 = state_mean32(p.state, d);
  float* best = state_best(p.state, d);
  const T* pts = reinterpret_cast<const T*>(p.pts);
  const int tid = threadIdx.x;
  const int dp = dpad4(d);
  // dynamic shared memory: column totals as (s, c) pairs | mean | v_1 | Bbar | staged partial rows
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  double* s_mean = reinterpret_cast<double*>(smem_raw) + st;
  double* s_v1 = s_mean + dp;
  double* s_dual = s_v1 + dp;
  float* stage = reinterpret_cast<float*>(s_dual + dp);
  const double* dual = state_dual(p.state, d);
  // what the finish reads, fetched before the reduction so that its latency
  // overlaps it: the FP64 header, mean and Bbar straight into shared memory
  // (cp.async: no register is held across the reduction), v_1 into a register
  constexpr int HW = (int)(sizeof(StateHdr) / 8);
  if (tid < HW) cp_async8(s_hdr + tid, reinterpret_cast<const double*>(hdr) + tid);
  for (int j = tid; j < d; j += blockDim.x) {
    cp_async8(s_mean + j, mean + j);
    cp_async8(s_dual + j, dual + j);
  }
  const float v0 = tid < d ? elem_to_float<T>(pts + tid) : 0.f;
  const float gam1 = p.radii ? __ldg(p.radii) : 0.f;
  // a staged pass whose copy wait gave up (read before the reduction, so that
  // the load's latency overlaps it; cleared once every thread has read it)
  unsigned int* tmo = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(p.counter) + kTimeoutFlagOff);
  const bool timed_out = __ldcg(tmo) != 0u;
  if (p.fx) {
    fx_finish(p.counter, p.partials, st, raw, s_scr, fe, opof);
    if (p.radii && tid == 0) raw[3] = make_float2(NAN, 0.f);  // no QP bound for spheres (not pushed)
  } else {
    final_reduce(p.partials, st, p.grows, p.counter, s_scr, opof, raw, stage, p.single, 2, -1, st);
  }
  cp_async_wait_all();
  pdl_trigger();  // (the fixed-point path: the totals are read)
  if (p.row_out) {  // a shard of a row-sharded iteration: hand the totals to the merge
    __syncthreads();
    for (int pc = tid; pc < st; pc += blockDim.x)  // a timed-out pass hands on S = NaN: the merge reports it
      p.row_out[pc] = (timed_out && pc == 0) ? make_float2(NAN, 0.f) : raw[pc];
    if (timed_out && tid == 0) *tmo = 0u;
    return;
  }
  if (tid < d) s_v1[tid] = (double)v0;
  for (int j = tid + blockDim.x; j < d; j += blockDim.x) s_v1[j] = (double)elem_to_float<T>(pts + j);
  __syncthreads();
  if (timed_out && tid == 0) *tmo = 0u;
  // The O(d) math runs in one warp (FP64 work is slow on this GPU and would
  // only contend across warps; no block barrier follows): the last warp,
  // which as the warm-up warp ran the finish's code at the start of the
  // launch, so its scheduler's instruction cache holds that code. The
  // averaged QP bound, whose FP64 chains are the finish's longest, runs at
  // the same time in the warp before it.
  const int nw = (int)(blockDim.x >> 5), w = (int)(tid >> 5);
  const bool split = nw >= 2;
  if (w != nw - 1 && !(split && w == nw - 2)) return;
  ses_finish_warp(raw, s_mean, s_v1, *reinterpret_cast<const StateHdr*>(s_hdr), p.state, d, p.alpha, (double)gam1,
                  p.eta_over_rho, p.eval_only, p.out, p.tape, s_dual, timed_out ? PDSCP_ERR_TIMEOUT : PDSCP_OK,
                  split ? (w == nw - 1 ? 1 : 2) : 0);
}

}  // namespace pdscp

namespace pdscp {

// Vector-path form of ses_iter_kernel for rows of at most 32 chunks: every
// lane holds one 16-byte chunk of each of NI points per round, and the
// scalar work of each point (sqrt, exp, expm1, divide) is done once, by the
// lane that owns the point after a reduce-scatter of the partial squared
// distances (GroupScatter), instead of on all LPP lanes of the point's group.
// The weighted sums G' are then accumulated from the broadcast
// coefficients. Same arithmetic per point as ses_iter_kernel; only the order
// of the FP32 partial sums differs.
//
// S = 0: every lane loads its chunks of a round straight into registers, the
// next round's loads issued after the current round's arithmetic. S >= 2:
// staged rounds. Each streaming warp owns a ring of S slots of shared memory
// (4 KB each, one round) and S mbarriers; lane 0 fills a slot with one bulk
// copy (cp.async.bulk) of the round's contiguous rows, and the copies of the
// next S - 1 rounds are in flight while the warp computes the current one
// from shared memory (bytes in flight no longer bounded by registers). A
// wait that gives up after p.wait_limit tries records a timeout, drains the
// copies still in flight and leaves the loop; the finishing CTA reports
// PDSCP_ERR_TIMEOUT.
template <typename T, int VW, int LPP, int NI, int BLOCK, int NS>
__global__ void __launch_bounds__(BLOCK, 1) ses_iter_t_kernel(SesParams p) {
  using GS = GroupScatter<LPP, NI>;
  constexpr int NW = BLOCK / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float s_sc[NW][4];
  __shared__ uint64_t s_bar[NS > 0 ? NW * NS : 1];
  // per-lane sum of the ORACLE coefficients (kept in shared memory: one more
  // register across the streaming loop costs more than the shared access)
  __shared__ float s_cs[BLOCK];

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = d / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;  // points per load instruction per warp
  const bool owner = (gl % GS::SHARE) == 0;
  const bool has_chunk = gl < nch;
  const T* pts = reinterpret_cast<const T*>(p.pts);
  // Float32 staged passes let the next launch start only once the finishing
  // CTA holds the partial rows in shared memory (final_reduce): started
  // earlier, the next launch's copies compete with that CTA's reads of the
  // rows (measured at n = 1e6, d = 32, back to back: 27.1 -> 26.2 us per
  // iteration). The other CTAs exit after their arrival, which counts as
  // their trigger. Bfloat16 passes, whose streaming is bound by instruction
  // issue rather than bytes, gain from the earlier start (22.7 -> 22.0 us).
  if constexpr (NS == 0 || sizeof(T) == 2) pdl_trigger();
  const WarpSplit wsp(p.sink, NW, warp);
  constexpr int SLOT = 32 * NI * VW * (int)sizeof(T);  // >= ROUND * d * sizeof(T)
  if (wsp.warm) ses_finish_warm<T>(p, smem_raw, (size_t)(ses_partial_stride(p.d) + 3 * dpad4(p.d)) * sizeof(double));
  const int64_t nwarps = wsp.nwarps;
  const int64_t gw = wsp.gw;
  constexpr int ROUND = PPW * NI;
  // each warp streams one contiguous range of points, equal up to 8 points
  // (balanced bytes per warp; starts on 8-point boundaries)
  auto split = [&](int64_t w) { return w >= nwarps ? p.n : ((w * p.n / nwarps) & ~(int64_t)7); };
  const int64_t lo = wsp.warm ? p.n : split(gw), hi = wsp.warm ? p.n : split(gw + 1);
  // the first round's point loads do not depend on the state: issue them first.
  // BF16 rows stay packed (16 bytes = 4 registers per chunk) and are widened
  // where they are used, which halves the registers a round needs.
  constexpr bool kPacked = sizeof(T) == 2;
  float x[kPacked ? 1 : NI][kPacked ? 1 : VW];
  uint4 xr[kPacked ? NI : 1];
  auto load_round = [&](int64_t base) {
#pragma unroll
    for (int r = 0; r < NI; ++r) {
        const int64_t i = base + r * PPW + grp;
        if constexpr (kPacked) {
          xr[r] = (i < hi && has_chunk) ? __ldg(reinterpret_cast<const uint4*>(pts + i * d) + gl) : make_uint4(0u, 0u, 0u, 0u);
        } else if (i < hi && has_chunk) {
          Chunk<T, VW>::load(pts + i * d, gl, x[r]);
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e) x[r][e] = 0.f;
        }
      }
  };
  // element e of round slot r as FP32 (bf16 -> fp32 is a 16-bit left shift of the bit pattern)
  auto xval = [&](int r, int e) -> float {
    const uint4& v = xr[r];
    const int j = e >> 1;
    const uint32_t w = j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
    return __uint_as_float((e & 1) ? (w & 0xffff0000u) : (w << 16));
  };
  // staged rounds: slot k of this warp's ring, one round of contiguous rows
  unsigned char* ring = smem_raw + (size_t)warp * (NS > 0 ? NS : 1) * SLOT;
  uint64_t* bar = s_bar + (NS > 0 ? warp * NS : 0);
  auto issue = [&](int k, int64_t b) {  // lane 0: round starting at row b into slot k
    const int64_t m = hi - b < ROUND ? hi - b : ROUND;
    bulk_load(ring + k * SLOT, pts + b * d, (unsigned int)(m * d * (int64_t)sizeof(T)), bar + k);
  };
  if constexpr (NS > 0) {
    // NS - 1 rounds are issued before the wait for the previous launch: the
    // copies of every CTA of this launch that starts early flood the memory
    // system while the previous launch's finishing CTA reads its partial
    // rows (measured at n = 1e6, d = 32: its staged reduction took 5.1 us with
    // 2 rounds ahead, 3.4 us with 1; the iteration 1.3 us less with 1)
    if (lane == 0 && lo < hi) {
#pragma unroll
      for (int k = 0; k < NS; ++k) mbar_init(bar + k, 1);
      mbar_init_fence();
#pragma unroll
      for (int k = 0; k < NS - 1; ++k)
        if (lo + k * ROUND < hi) issue(k, lo + k * ROUND);
    }
    __syncwarp();
  } else {
    load_round(lo);
  }
  // the round at base, slot k, from shared memory into the round's registers
  auto read_round = [&](int64_t base, int k) {
    const unsigned char* sl = ring + k * SLOT;
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int64_t i = base + r * PPW + grp;
      const uint4 v = (i < hi && has_chunk)
                          ? *reinterpret_cast<const uint4*>(sl + ((size_t)(r * PPW + grp) * d) * sizeof(T) + gl * 16)
                          : make_uint4(0u, 0u, 0u, 0u);
      if constexpr (kPacked) {
        xr[r] = v;
      } else {
        x[r][0] = __uint_as_float(v.x);
        x[r][1] = __uint_as_float(v.y);
        x[r][2] = __uint_as_float(v.z);
        x[r][3] = __uint_as_float(v.w);
      }
    }
  };
  // waits (at least kWaitLimit tries each) for the copies of rounds r0 ..
  // r0 + NS - 1 that were issued, before the ring's memory is reused or the
  // CTA exits
  auto drain = [&](int r0) {
    if constexpr (NS > 0) {
      const unsigned int lim = p.wait_limit > kWaitLimit ? p.wait_limit : kWaitLimit;
#pragma unroll
      for (int j = 0; j < NS; ++j)
        if (lo + (int64_t)(r0 + j) * ROUND < hi) mbar_wait(bar + (r0 + j) % NS, (unsigned int)((r0 + j) / NS) & 1u, lim);
    }
  };
  bool timed_out = false;
  // BF16 rows (register rounds): a round holds twice the points of an FP32
  // round, and its loads wait for the previous round's arithmetic; lane 0 of
  // each warp asks L2 for the next round ahead of its loads (measured at n =
  // 1e6, d = 32: 32.8 -> 30.7 us; no gain for FP32, so not done there)
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
    drain(0);  // staged: the first rounds' copies are in flight
    return;
  }

  const float kr = p.eval_only ? 0.f : ses_kr(hdr->t, p.eta_over_rho);
  const float H = (float)(hdr->hint + hdr->move);
  const float alpha = (float)p.alpha;
  const float* mean32 = state_mean32(p.state, d);
  // the completion's scale exponents, kept in shared memory across the
  // streaming loop rather than in registers
  __shared__ SesFxExp s_fe;
  if (threadIdx.x == 0) s_fe = ses_fx_exp(p.n, kr, H, alpha);

  float ub[VW], G[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    ub[e] = has_chunk ? mean32[gl * VW + e] : 0.f;
    G[e] = 0.f;
  }
  // BF16 rows: the mean and the weighted sums as float pairs, so that the
  // distances and the weighted sums run in paired FP32 arithmetic (one
  // instruction per two elements; the pass is issue-bound for BF16 rows:
  // n = 4e6, d = 32, back to back 60.6 -> 56.0 us). Each element's result is
  // that of the scalar operation; only the order of a point's partial
  // squared distance (even and odd elements summed apart) differs.
  constexpr int VP = kPacked ? VW / 2 : 1;
  unsigned long long ub2[VP], G2[VP];
#pragma unroll
  for (int q = 0; q < VP; ++q) {
    ub2[q] = f2_pack(ub[2 * q], ub[(2 * q + 1) % VW]);
    G2[q] = 0ull;
  }
  auto xword = [&](int r, int q) -> uint32_t {
    const uint4& v = xr[r];
    return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
  };
  float S = 0.f, W = 0.f, maxd = -INFINITY;
  s_cs[threadIdx.x] = 0.f;

  int rnd = 0;
  for (int64_t base = lo; base < hi; base += ROUND, ++rnd) {
    const int k = NS > 0 ? rnd % (NS > 0 ? NS : 1) : 0;
    if constexpr (NS > 0) {
      if (!mbar_wait(bar + k, (unsigned int)(rnd / (NS > 0 ? NS : 1)) & 1u, p.wait_limit)) {
        timed_out = true;
        break;
      }
      read_round(base, k);
    } else {
      prefetch_round(base + ROUND);
      if (base != lo) load_round(base);
    }
    float part[NI];
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      float a = 0.f;
      if constexpr (kPacked) {
        unsigned long long acc = 0ull;
#pragma unroll
        for (int q = 0; q < VP; ++q) {
          const unsigned long long t = f2_sub(f2_from_bf16x2(xword(r, q)), ub2[q]);
          acc = f2_fma(t, t, acc);
        }
        float lo, hi2;
        f2_unpack(acc, lo, hi2);
        a = lo + hi2;
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          x[r][e] -= ub[e];
          a = fmaf(x[r][e], x[r][e], a);
        }
      }
      part[r] = has_chunk ? a : 0.f;
    }
    GS::run(part, gl);
    float c[GS::OWN];
#pragma unroll
    for (int k = 0; k < GS::OWN; ++k) {
      const int64_t i = base + GS::owned(gl, k) * PPW + grp;
      c[k] = 0.f;
      if (i >= p.first && i < hi) {
        const float dist = sqrtf(part[k]);
        const float gam = p.radii ? __ldg(p.radii + i) : 0.f;
        const float a = alpha - gam;
        const float E1 = expf(kr * ((dist + gam) - H));
        const float em = -expm1f(-2.f * kr * dist);
        const float dif = E1 * em;
        const float sum = E1 * (2.f - em);
        c[k] = dist > 0.f ? dif / dist : 2.f * kr * E1;
        if (owner) {
          S += sum;
          W += a * sum - dist * dif;
          s_cs[threadIdx.x] += c[k];
          maxd = fmaxf(maxd, dist + gam);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const float cr = __shfl_sync(0xffffffffu, c[r % GS::OWN], grp * LPP + GS::src_lane(r));
      if constexpr (kPacked) {
        const unsigned long long c2 = f2_pack(cr, cr);
#pragma unroll
        for (int q = 0; q < VP; ++q) G2[q] = f2_fma(c2, f2_sub(f2_from_bf16x2(xword(r, q)), ub2[q]), G2[q]);
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) G[e] = fmaf(cr, x[r][e], G[e]);
      }
    }
    if constexpr (NS > 0) {
      // every lane has read slot k (its values were used above): refill it
      // with the round S ahead
      __syncwarp();
      if (lane == 0 && base + NS * ROUND < hi) {
        fence_proxy_async_smem();
        issue(k, base + NS * ROUND);
      }
    }
  }
  if constexpr (NS > 0) {
    if (timed_out) {
      // drain: wait (again at most wait_limit tries, at least the default)
      // for every copy still in flight before the ring is reused or the
      // CTA exits, then report the timeout
      drain(rnd);
      if (lane == 0) atomicOr(reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(p.counter) + kTimeoutFlagOff), 1u);
    }
  }

  if constexpr (kPacked) {
#pragma unroll
    for (int q = 0; q < VP; ++q) f2_unpack(G2[q], G[2 * q], G[(2 * q + 1) % VW]);
  }
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int e = 0; e < VW; ++e) G[e] += __shfl_xor_sync(0xffffffffu, G[e], o);
  S = warp_sum(S);
  const float Cs = warp_sum(s_cs[threadIdx.x]);
  W = warp_sum(W);
  maxd = warp_max(maxd);
  if constexpr (NS > 0) __syncthreads();  // every warp is done with its ring before the shared memory is reused
  float* sG = reinterpret_cast<float*>(smem_raw);
  if (grp == 0 && has_chunk)
#pragma unroll
    for (int e = 0; e < VW; ++e) sG[warp * dp + gl * VW + e] = G[e];
  if (lane == 0) {
    s_sc[warp][0] = S;
    s_sc[warp][1] = W;
    s_sc[warp][2] = maxd;
    s_sc[warp][3] = Cs;
  }
  __syncthreads();
  const SesFxExp fe = s_fe;
  float* prow = p.partials + (size_t)blockIdx.x * ses_partial_stride(d);
  for (int j = threadIdx.x; j < d; j += BLOCK) {
    float s = 0.f;
    for (int w = 0; w < NW; ++w) s += sG[w * dp + j];
    ses_emit(p, prow, fe, 4 + j, s);
  }
  if (threadIdx.x == 0) {
    float s0 = 0.f, s1 = 0.f, s3 = 0.f, m = -INFINITY;
    for (int w = 0; w < NW; ++w) {
      s0 += s_sc[w][0];
      s1 += s_sc[w][1];
      s3 += s_sc[w][3];
      m = fmaxf(m, s_sc[w][2]);
    }
    ses_emit(p, prow, fe, 0, s0);
    ses_emit(p, prow, fe, 1, s1);
    ses_emit(p, prow, fe, 2, m);
    ses_emit(p, prow, fe, 3, p.radii ? NAN : s3);  // the QP bound holds for points only
  }
  ses_finish<T>(p, smem_raw, fe);
}

}  // namespace pdscp

namespace pdscp {

// Row-sharded iteration, second half: the column totals of the shards
// (`ranks` rows of ses_partial_stride(d) compensated pairs, in rank order)
// are reduced in that fixed order, and the O(d) finish runs as in the
// unsharded kernel. v1 / radius1: the easy cone's centre and radius, which
// only the first shard holds. One CTA of kMergeBlock threads.
struct SesMergeParams {
  const float2* rows;
  int ranks;
  const void* v1;
  const float* radius1;  // may be null
  int d;
  int eval_only;
  double alpha;
  double eta_over_rho;
  void* state;
  pdscp_step_out* out;
};

constexpr int kMergeBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kMergeBlock) ses_merge_kernel(SesMergeParams m) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float2 s_scr[kMergeBlock];
  __shared__ __align__(16) double s_hdr[sizeof(StateHdr) / 8];
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(m.state);
  if (hdr->stopped && !m.eval_only) return;  // as the pass kernels: a stopped FTP is left as is
  const int d = m.d, dp = dpad4(d), st = ses_partial_stride(d);
  const int tid = threadIdx.x;
  // dynamic shared memory: column totals (s, c) | mean | v_1 | Bbar
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  double* s_mean = reinterpret_cast<double*>(smem_raw) + st;
  double* s_v1 = s_mean + dp;
  double* s_dual = s_v1 + dp;
  const double* dual = state_dual(m.state, d);
  constexpr int HW = (int)(sizeof(StateHdr) / 8);
  if (tid < HW) s_hdr[tid] = reinterpret_cast<const double*>(hdr)[tid];
  const double* mean = state_mean(m.state);
  const T* v1 = reinterpret_cast<const T*>(m.v1);
  for (int j = tid; j < d; j += blockDim.x) {
    s_mean[j] = mean[j];
    s_v1[j] = (double)elem_to_float<T>(v1 + j);
    s_dual[j] = dual[j];
  }
  auto opof = [](int pc) { return pc == 2 ? 1 : 0; };
  reduce_rows(m.rows, 0, m.ranks, st, raw, s_scr, opof);  // ends with a barrier
  if (tid >= 32) return;
  const double gam1 = m.radius1 ? (double)__ldg(m.radius1) : 0.0;
  ses_finish_warp(raw, s_mean, s_v1, *reinterpret_cast<const StateHdr*>(s_hdr), m.state, d, m.alpha, gam1,
                  m.eta_over_rho, m.eval_only, m.out, nullptr, s_dual);
}

}  // namespace pdscp
