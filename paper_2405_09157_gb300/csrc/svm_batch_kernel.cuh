// Batched SVM iteration: one launch runs one MWU iteration of the
// minimisation alpha-FTP (Sec. 3, Eq. min_implement; the data of Sec. 4.2,
// as in svm_kernel.cuh) for every instance of a batch of independent
// hard-margin SVM problems of uneven size n_i and dimension d_i <= 64. The
// instances' points are packed in one float32 or bfloat16 buffer, their
// labels (+1: class P, -1: class Q) in one int8 buffer; each instance is cut
// into tiles of consecutive rows. A persistent grid takes tiles from a
// global counter; the CTA that completes an instance's last tile reduces
// that instance's partial rows and runs its O(d) finish (svm_finish_warp)
// while the other CTAs keep streaming. No CTA waits on another.
//
// Per point i of an instance at the means (wbar, s1bar, s2bar):
//   m_i = y_i x_i^T wbar - sbar_{class i},  weight e^{-k (m_i - (hint - move))}
// and per CTA the class sums S_P, S_Q, Z_P, Z_Q and min_P / max_Q of the
// dots (the columns of svm_iter_kernel's partial row).
#pragma once

#include "batch_kernel.cuh"
#include "bf16_chunk4.cuh"
#include "svm_kernel.cuh"

namespace pdscp {

// partial row of one tile: [S_P, S_Q, minP, maxQ, Z_P (dp), Z_Q (dp)], dp <= 64
constexpr int kSvmBatchStride = 4 + 2 * kBatchMaxD;

// Workspace of an SVM batch: the SES batch's regions (counters, header,
// options at kBatchOptsOff, instance and tile tables, partial rows, states,
// search records) plus the label offsets and the largest point norm D of
// every instance (Sec. 4.2: s_1, s_2 <= D), computed by svm_batch_init.
struct SvmBatchHeader {
  BatchHeader b;     // as for the SES batch (b.dtype: the point type)
  int64_t lab_off;   // byte offset of the per-instance label offsets (int64, elements of the label buffer)
  int64_t dval_off;  // byte offset of the per-instance D (double)
};
static_assert(sizeof(SvmBatchHeader) <= 256, "header fits before the options");

struct SvmBatchParams {
  const void* pts;             // packed rows of the kernels' point type T
  const int8_t* labels;        // packed labels
  const double* alpha;         // per instance (plain iterations)
  const double* eta_over_rho;  // per instance (plain iterations)
  unsigned char* ws;
  pdscp_step_out* out;         // per instance, may be null
  BatchSearch* search;         // non-null: device-side search; alpha, eta/rho come from here
};

// Streams rows [r0, r1) of one instance (labels lab) at the mean wbar (shared
// memory, FP32) and leaves the CTA's per-warp totals in sZ / s_sc. Same
// per-point arithmetic as svm_iter_kernel.
template <typename T, int VW, int LPP, int NCH, int U>
__device__ void svm_batch_tile(const T* pts, const int8_t* lab, int d, int64_t r0, int64_t r1, const float* s_wb,
                               float k, float Hm, float s1, float s2, float* sZ, float (*s_sc)[4]) {
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  float wb[NCH][VW], ZP[NCH][VW], ZQ[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      wb[j][e] = (c < nch) ? s_wb[c * VW + e] : 0.f;
      ZP[j][e] = 0.f;
      ZQ[j][e] = 0.f;
    }
  }
  float SP = 0.f, SQ = 0.f, minP = INFINITY, maxQ = -INFINITY;
  for (int64_t base = r0 + (int64_t)warp * (PPW * U); base < r1; base += (int64_t)kBatchWarps * (PPW * U)) {
    float x[U][NCH][VW];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      const T* row = pts + i * d;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        if (i < r1 && c < nch) {
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
      if (i < r1) {
        const bool pos = __ldg(lab + i) > 0;
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
  if (grp == 0) {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int c = gl + j * LPP;
      if (c < nch)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          sZ[warp * 2 * kBatchMaxD + c * VW + e] = ZP[j][e];
          sZ[warp * 2 * kBatchMaxD + kBatchMaxD + c * VW + e] = ZQ[j][e];
        }
    }
  }
  if (lane == 0) {
    s_sc[warp][0] = SP;
    s_sc[warp][1] = SQ;
    s_sc[warp][2] = minP;
    s_sc[warp][3] = maxQ;
  }
}

// svm_batch_tile for rows of 4-element chunks (d = 4 .. 64, d % 4 == 0, rows
// aligned): each warp streams one contiguous part of the tile, NI points per
// lane per round, and each point's margin, label test and exponential run
// once, on the lane that owns the point after a reduce-scatter of the partial
// dot products (GroupScatter, as in svm_iter_t_kernel); the signed weight
// y_i e^{...} is broadcast back for the class sums Z_P, Z_Q.
template <typename T, int VW, int LPP, int NI>
__device__ void svm_batch_tile_t(const T* pts, const int8_t* lab, int d, int64_t r0, int64_t r1, const float* s_wb,
                                 float k, float Hm, float s1, float s2, float* sZ, float (*s_sc)[4]) {
  using GS = GroupScatter<LPP, NI>;
  const int nch = d / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  constexpr int ROUND = PPW * NI;
  const bool owner = (gl % GS::SHARE) == 0;
  const bool has_chunk = gl < nch;
  const int64_t len = r1 - r0;
  const int64_t lo = r0 + (int64_t)warp * len / kBatchWarps, hi = r0 + (int64_t)(warp + 1) * len / kBatchWarps;
  float wb[VW], ZP[VW], ZQ[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    wb[e] = has_chunk ? s_wb[gl * VW + e] : 0.f;
    ZP[e] = 0.f;
    ZQ[e] = 0.f;
  }
  float SP = 0.f, SQ = 0.f, minP = INFINITY, maxQ = -INFINITY;
  for (int64_t base = lo; base < hi; base += ROUND) {
    float x[NI][VW];
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
      if (i < hi) {
        const float dot = part[kk];
        const bool pos = __ldg(lab + i) > 0;
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
  if (grp == 0 && has_chunk)
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      sZ[warp * 2 * kBatchMaxD + gl * VW + e] = ZP[e];
      sZ[warp * 2 * kBatchMaxD + kBatchMaxD + gl * VW + e] = ZQ[e];
    }
  if (lane == 0) {
    s_sc[warp][0] = SP;
    s_sc[warp][1] = SQ;
    s_sc[warp][2] = minP;
    s_sc[warp][3] = maxQ;
  }
}

// A fresh alpha-FTP of an SVM instance: t = 0, means 0 (uniform weights on
// each class at t = 0), as mwu_state_init does for SVM. One warp.
__device__ __forceinline__ void svm_batch_fresh_state(void* state, int d, const BatchSolveOpts* o) {
  const int lane = threadIdx.x & 31;
  const int dp = dpad4(d);
  double* mean = state_mean(state);
  float* mean32 = state_mean32(state, d);
  float* best = state_best(state, d);
  double* dual = state_dual(state, d);
  for (int j = lane; j < dp; j += 32) {
    mean[j] = 0.0;
    mean32[j] = 0.f;
    best[j] = 0.f;
    dual[j] = 0.0;
  }
  if (lane == 0) {
    StateHdr z;
    memset(&z, 0, sizeof(z));
    z.rules = o ? o->rules : PDSCP_RULES_NONE;
    z.patience = o ? o->patience : 1;
    z.delta = o ? o->delta : 0.0;
    z.f_prev = -1.0;
    z.best_f = 0.0;  // SVM: the best margin so far (a lower bound)
    z.ub_best = INFINITY;
    *reinterpret_cast<StateHdr*>(state) = z;
  }
}

// One warp, after the launch that ran the instance's iteration: the decisions
// of svm_solve for one instance (the search of Sec. 3 over alpha in
// (0, 2D]: a separation proves OPT < alpha and sets U = alpha; in the
// practical and theory modes T_i iterations without one, a stall (Sec. 5) or
// a margin above alpha set L = max(L, (1 - eps_i) alpha); certificates: the
// best margin f of an actual direction (lower bound) and the best Claim 8
// value (upper bound); in CERTIFIED mode only proven conclusions, polls
// every o.poll iterations with the certificate and progress tests of the
// single-instance search) and the start of its next alpha-FTP.
static __device__ __forceinline__ void svm_batch_search_update(BatchSearch* sr, void* state, int d, int64_t n,
                                                            double Dinst, const BatchSolveOpts& o,
                                                            unsigned int* done_counter) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  StateHdr* hdr = reinterpret_cast<StateHdr*>(state);
  const StateHdr h = *hdr;
  BatchSearch r = *sr;
  const bool cert = o.mode == PDSCP_MODE_CERTIFIED;
  bool end_ftp = false, start_ftp = false, done = false;
  bool take_w = false;
  if (h.status != PDSCP_OK) {
    r.status = h.status;
    done = true;
  } else if (r.phase == kPhaseBounds) {
    r.D = Dinst;
    if (!(r.D > 0.0)) {
      r.lb = r.ub = r.L = r.U = 0.0;
      done = true;
    } else {
      r.rho = 2.0 * r.D;
      r.logr = log((double)n);
      r.L = 0.0;
      r.U = 2.0 * r.D;
      r.lb = 0.0;
      r.ub = INFINITY;
      r.eta_c = o.eta > 0.0 ? o.eta : 1.0;
      start_ftp = true;
    }
  } else if (r.phase == kPhaseFinal || h.stopped) {
    end_ftp = true;
  } else if (h.t >= r.cap) {
    r.phase = kPhaseFinal;  // the next launch evaluates f at the final mean
  } else if (cert && h.t % o.poll == 0) {
    if (fmin(fmin(r.ub, r.U), h.ub_best) <= (1.0 + o.eps) * fmax(r.lb, h.best_f)) {
      r.why = kWhyClosed;
      r.phase = kPhaseFinal;
    } else if ((double)h.t >= r.next_check) {
      const double gap = h.best_f > 0.0 ? h.ub_best / h.best_f - 1.0 : INFINITY;
      if (gap > kCertShrink * r.last_gap) {
        r.why = kWhyStuck;
        r.phase = kPhaseFinal;
      } else {
        r.last_gap = gap;
        r.next_check *= 2.0;
      }
    }
  }
  if (end_ftp) {
    const int64_t iters = h.t;
    const int oc = h.stopped ? h.outcome : PDSCP_OUT_RUNNING;
    r.total += iters;
    if (h.best_f > r.lb) {
      r.lb = h.best_f;
      take_w = true;
    }
    if (h.ub_best < r.ub) r.ub = h.ub_best;
    if (cert) {
      if (oc == PDSCP_OUT_SEPARATED) r.U = fmin(r.U, r.alpha);
      if (r.why == kWhyStuck) r.eta_c *= 0.5;
      r.U = fmin(r.U, r.ub);
      r.L = fmax(r.L, r.lb);
      r.steps += 1;
      if (oc == PDSCP_OUT_RUNNING && r.why == kWhyBudget) {
        done = true;  // the iteration budget ended this FTP
      } else if (!(fmin(r.ub, r.U) > (1.0 + o.eps) * r.lb && r.total < o.max_iters && r.steps < o.max_steps)) {
        done = true;
      } else {
        start_ftp = true;
      }
      if (done) r.ub = fmin(r.ub, r.U);  // a separation is a proof too
    } else {
      if (oc == PDSCP_OUT_SEPARATED) {
        r.U = fmin(r.U, r.alpha);
      } else if (iters >= r.T || oc == PDSCP_OUT_STALLED || oc == PDSCP_OUT_BEAT_ALPHA) {
        r.L = fmax(fmax(r.L, (1.0 - r.eps_i) * r.alpha), r.lb);
      }
      r.U = fmin(r.U, r.ub);
      r.L = fmax(r.L, r.lb);
      r.steps += 1;
      if (oc == PDSCP_OUT_RUNNING && iters < r.T) {
        done = true;  // the iteration budget ended this FTP
      } else if (!(r.U > (1.0 + o.eps) * r.L && r.ub > (1.0 + o.eps) * r.lb && r.total < o.max_iters &&
                   r.steps < o.max_steps)) {
        done = true;
      } else {
        start_ftp = true;
      }
    }
  }
  // the direction of the best margin (read before a fresh FTP resets the state)
  for (int j = lane; j < d; j += 32)
    if (take_w) r.center[j] = state_best(state, d)[j];
  __syncwarp();
  if (start_ftp) {
    r.alpha = r.U - (r.U - r.L) / 3.0;
    r.eps_i = (r.U - r.L) / (3.0 * r.alpha);
    const double Tf = ceil(64.0 * r.D * r.D * r.logr / (r.eps_i * r.eps_i * r.alpha * r.alpha));
    r.T = Tf > 4.0e18 ? (int64_t)4e18 : (int64_t)Tf;
    const double eta = cert ? r.eta_c : (o.eta > 0.0 ? o.eta : sqrt(r.logr / (double)r.T));
    r.eta_over_rho = eta / r.rho;
    const int64_t left = o.max_iters - r.total;
    if (cert) r.T = left;  // no theorem count: the FTP runs until a proof, the certificates or the budget
    r.cap = r.T < left ? r.T : left;
    r.why = kWhyBudget;
    r.last_gap = INFINITY;
    r.next_check = (cert && eta > kCertMinEta) ? ceil(kCertFirstCheck / eta) : INFINITY;
    r.phase = kPhaseFtp;
    svm_batch_fresh_state(state, d, &o);
  }
  if (done) {
    r.phase = kPhaseDone;
    if (lane == 0) {
      hdr->stopped = 1;  // the instance's tiles are skipped from now on
      atomicAdd(done_counter, 1u);
    }
  }
  __syncwarp();
  if (lane == 0) {
    BatchSearch* dst = sr;
    dst->D = r.D;
    dst->rho = r.rho;
    dst->logr = r.logr;
    dst->L = r.L;
    dst->U = r.U;
    dst->lb = r.lb;
    dst->ub = r.ub;
    dst->alpha = r.alpha;
    dst->eps_i = r.eps_i;
    dst->eta_over_rho = r.eta_over_rho;
    dst->T = r.T;
    dst->cap = r.cap;
    dst->total = r.total;
    dst->steps = r.steps;
    dst->phase = r.phase;
    dst->status = r.status;
    dst->why = r.why;
    dst->eta_c = r.eta_c;
    dst->last_gap = r.last_gap;
    dst->next_check = r.next_check;
  }
  for (int j = lane; j < d; j += 32) sr->center[j] = r.center[j];
}

// One launch: one iteration (or evaluation pass) of every running instance.
// Three CTAs of 256 threads per SM (as ses_batch_kernel).
template <typename T>
static __global__ void __launch_bounds__(kBatchBlock, 3) svm_batch_kernel(SvmBatchParams p) {
  __shared__ float sZ[kBatchWarps * 2 * kBatchMaxD];
  __shared__ float s_sc[kBatchWarps][4];
  __shared__ float s_wb[kBatchMaxD];
  __shared__ float2 raw[kSvmBatchStride];
  __shared__ double s_mean[kBatchMaxD];
  __shared__ double s_dual[kBatchMaxD];
  __shared__ float2 s_scr[kBatchBlock];
  __shared__ __align__(16) double s_hdr[sizeof(StateHdr) / 8];
  __shared__ long long s_tile;
  __shared__ bool s_flag;
  const int tid = threadIdx.x;
  auto opof = [](int pc) { return svm_col_op(pc); };
  const SvmBatchHeader sh = *reinterpret_cast<const SvmBatchHeader*>(p.ws + 256);
  const BatchHeader& bh = sh.b;
  unsigned int* counters = reinterpret_cast<unsigned int*>(p.ws);  // [0] next tile, [1] CTAs done
  unsigned int* inst_counters = reinterpret_cast<unsigned int*>(p.ws + bh.instcnt_off);
  const BatchInst* insts = reinterpret_cast<const BatchInst*>(p.ws + bh.inst_off);
  const BatchTile* tiles = reinterpret_cast<const BatchTile*>(p.ws + bh.tile_off);
  const int64_t* lab_off = reinterpret_cast<const int64_t*>(p.ws + sh.lab_off);
  const double* Dval = reinterpret_cast<const double*>(p.ws + sh.dval_off);
  float* partials = reinterpret_cast<float*>(p.ws + bh.partial_off);

  for (;;) {
    if (tid == 0) s_tile = (long long)atomicAdd(&counters[0], 1u);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= bh.ntiles) break;
    const BatchTile tl = tiles[tile];
    const BatchInst in = insts[tl.inst];
    void* state = p.ws + in.state_off;
    const StateHdr* hdr = reinterpret_cast<const StateHdr*>(state);
    const int d = in.d;
    const int dp = dpad4(d);
    const T* pts = static_cast<const T*>(p.pts) + in.pt_off;
    const int8_t* lab = p.labels + lab_off[tl.inst];
    const BatchSearch* sr = p.search ? p.search + tl.inst : nullptr;
    const int phase = sr ? sr->phase : kPhaseFtp;
    // a stopped FTP (or a finished search) is left as is; the search's first
    // launch only lets the search step start the instance's first FTP
    if (hdr->stopped != 0 || phase == kPhaseBounds) {
      __syncthreads();
      continue;
    }
    const bool eval = phase == kPhaseFinal;
    const double alpha_d = sr ? sr->alpha : p.alpha[tl.inst];
    const double eor_d = sr ? sr->eta_over_rho : p.eta_over_rho[tl.inst];
    const double D_d = Dval[tl.inst];
    {
      const float k = eval ? 0.f : (float)((double)hdr->t * eor_d);
      const float Hm = (float)(hdr->hint - hdr->move);
      const float s1 = (float)hdr->s1bar, s2 = (float)hdr->s2bar;
      const float* mean32 = state_mean32(state, d);
      if (tid < d) s_wb[tid] = mean32[tid];
      __syncthreads();
      switch (in.shape) {
        case 0: svm_batch_tile_t<T, 4, 1, 8>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 1: svm_batch_tile_t<T, 4, 2, 8>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 2: svm_batch_tile_t<T, 4, 4, 8>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 3: svm_batch_tile_t<T, 4, 8, 8>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 4: svm_batch_tile_t<T, 4, 16, 8>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 5: svm_batch_tile<T, 1, 2, 1, 4>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 6: svm_batch_tile<T, 1, 8, 1, 4>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 7: svm_batch_tile<T, 1, 32, 1, 4>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        case 9: svm_batch_tile<T, 1, 1, 4, 4>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
        default: svm_batch_tile<T, 1, 32, 2, 2>(pts, lab, d, tl.r0, tl.r1, s_wb, k, Hm, s1, s2, sZ, s_sc); break;
      }
      __syncthreads();
      float* prow = partials + (size_t)tile * kSvmBatchStride;
      for (int j = tid; j < dp; j += kBatchBlock) {
        float a = 0.f, b = 0.f;
        if (j < d)
          for (int w = 0; w < kBatchWarps; ++w) {
            a += sZ[w * 2 * kBatchMaxD + j];
            b += sZ[w * 2 * kBatchMaxD + kBatchMaxD + j];
          }
        prow[4 + j] = a;
        prow[4 + dp + j] = b;
      }
      if (tid == 0) {
        float a = 0.f, b = 0.f, mn = INFINITY, mx = -INFINITY;
        for (int w = 0; w < kBatchWarps; ++w) {
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
    }
    // arrival of this tile at its instance
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned int prev = atomicAdd(&inst_counters[tl.inst], 1u);
      __threadfence();
      s_flag = (prev == (unsigned int)(in.ntiles - 1));
    }
    __syncthreads();
    if (s_flag) {
      // this CTA completed the instance: reduce its rows and finish it
      if (tid == 0) inst_counters[tl.inst] = 0u;
      constexpr int HW = (int)(sizeof(StateHdr) / 8);
      if (tid < HW) s_hdr[tid] = reinterpret_cast<const double*>(hdr)[tid];
      const double* mean = state_mean(state);
      if (tid < d) {
        s_mean[tid] = mean[tid];
        s_dual[tid] = state_dual(state, d)[tid];
      }
      const int st = svm_partial_stride(d);
      reduce_rows(partials + (size_t)in.tile0 * kSvmBatchStride, 0, in.ntiles, st, raw, s_scr, opof, kSvmBatchStride);
      if (tid < 32)
        svm_finish_warp(raw, s_mean, *reinterpret_cast<const StateHdr*>(s_hdr), state, d, alpha_d, D_d, eor_d,
                        eval ? 1 : 0, p.out ? p.out + tl.inst : nullptr, nullptr, s_dual);
    }
    __syncthreads();
  }
  // last CTA out resets the tile counter for the next launch
  if (tid == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(&counters[1], 1u);
    if (prev == gridDim.x - 1) {
      counters[0] = 0u;
      counters[1] = 0u;
      __threadfence();
    }
  }
}

// The search step of every instance still searching, one warp per instance.
static __global__ void __launch_bounds__(256) svm_batch_search_kernel(unsigned char* ws, int num) {
  const int inst = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (inst >= num) return;
  const SvmBatchHeader* sh = reinterpret_cast<const SvmBatchHeader*>(ws + 256);
  BatchSearch* sr = reinterpret_cast<BatchSearch*>(ws + sh->b.search_off) + inst;
  if (sr->phase == kPhaseDone) return;
  const BatchInst in = reinterpret_cast<const BatchInst*>(ws + sh->b.inst_off)[inst];
  const double D = reinterpret_cast<const double*>(ws + sh->dval_off)[inst];
  svm_batch_search_update(sr, ws + in.state_off, in.d, in.n, D,
                          *reinterpret_cast<const BatchSolveOpts*>(ws + kBatchOptsOff),
                          reinterpret_cast<unsigned int*>(ws) + 2);
}

// Fresh alpha-FTP states for every instance (t = 0, means 0); one warp per instance.
static __global__ void svm_batch_init_kernel(const BatchInst* inst, unsigned char* ws, unsigned int* inst_counters) {
  const BatchInst in = inst[blockIdx.x];
  if (threadIdx.x < 32) svm_batch_fresh_state(ws + in.state_off, in.d, nullptr);
  if (threadIdx.x == 0) inst_counters[blockIdx.x] = 0u;
}

// D = max_i ||x_i|| of every instance (Sec. 4.2): one thread per row of a
// tile, the squared norm summed in FP64, the maximum taken through the
// order of the non-negative doubles' bit patterns (Dbits zeroed beforehand).
template <typename T>
static __global__ void __launch_bounds__(256) svm_batch_norm_kernel(const T* pts, const BatchInst* inst,
                                                             const BatchTile* tiles, int64_t ntiles,
                                                             unsigned long long* Dbits) {
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const BatchTile tl = tiles[tile];
    const BatchInst in = inst[tl.inst];
    const T* rows = pts + in.pt_off;
    double m = 0.0;
    for (int64_t i = tl.r0 + threadIdx.x; i < tl.r1; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < in.d; ++j) {
        const double v = (double)elem_to_float(rows + i * in.d + j);
        s = fma(v, v, s);
      }
      m = fmax(m, s);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(Dbits + tl.inst, (unsigned long long)__double_as_longlong(sqrt(m)));
  }
}

// Means, best directions and D of every instance, packed at inst.mean_off.
static __global__ void svm_batch_read_kernel(const BatchInst* inst, unsigned char* ws, const double* Dval, float* mean_out,
                                      float* best_out, double* D_out) {
  const BatchInst in = inst[blockIdx.x];
  void* state = ws + in.state_off;
  for (int j = threadIdx.x; j < in.d; j += blockDim.x) {
    if (mean_out) mean_out[in.mean_off + j] = state_mean32(state, in.d)[j];
    if (best_out) best_out[in.mean_off + j] = state_best(state, in.d)[j];
  }
  if (threadIdx.x == 0 && D_out) D_out[blockIdx.x] = Dval[blockIdx.x];
}

// Per-instance search results: reports (value = lower_bound = the margin of
// the returned direction, upper_bound = the best certified upper bound) and
// the directions (packed at inst.mean_off).
static __global__ void svm_batch_solve_read_kernel(const BatchInst* inst, const BatchSearch* search, double eps,
                                            pdscp_report* rep, float* w_out) {
  const BatchInst in = inst[blockIdx.x];
  const BatchSearch& r = search[blockIdx.x];
  for (int j = threadIdx.x; j < in.d; j += blockDim.x)
    if (w_out) w_out[in.mean_off + j] = r.center[j];
  if (threadIdx.x == 0 && rep) {
    pdscp_report o;
    o.value = r.lb;
    o.lower_bound = r.lb;
    o.upper_bound = r.ub;
    o.D = r.D;
    o.search_L = r.L;
    o.search_U = r.U;
    o.iters = r.total;
    o.search_steps = r.steps;
    const bool conv = r.phase == kPhaseDone && (r.U <= (1.0 + eps) * r.L || r.ub <= (1.0 + eps) * r.lb);
    o.status = r.status != PDSCP_OK ? r.status : (conv ? PDSCP_OK : PDSCP_ERR_NOT_CONVERGED);
    rep[blockIdx.x] = o;
  }
}

}  // namespace pdscp
