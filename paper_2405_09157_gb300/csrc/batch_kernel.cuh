// Batched SES iteration: one launch runs one MWU iteration (Sec. 4.1 with
// Eq. implement and Eq. ses_oracle, as in ses_kernel.cuh) for every instance
// of a batch of independent SES problems of uneven size n_i and dimension
// d_i <= 64. The instances' points are packed in one float32 or bfloat16
// buffer (the kernels' point type T; bfloat16 rows are widened on load); each
// instance is cut into tiles of consecutive rows. A persistent grid takes
// tiles from a global counter; the CTA that completes an instance's last
// tile reduces that instance's partial rows and runs its O(d) finish while
// the other CTAs keep streaming. No CTA waits on another.
#pragma once

#include "bf16_chunk4.cuh"
#include "ses_kernel.cuh"

namespace pdscp {

constexpr int kBatchMaxD = 64;
constexpr int kBatchStride = 4 + kBatchMaxD;  // partial row: S, Wt, maxd, 0, G'_1..G'_d
constexpr int kBatchBlock = 256;
constexpr int kBatchWarps = kBatchBlock / 32;

struct BatchInst {
  int64_t pt_off;     // element offset of the instance's row 0 in the packed buffer
  int64_t n;          // rows (points) of the instance
  int64_t state_off;  // byte offset of the instance's state in the workspace
  int64_t tile0;      // first tile of the instance
  int64_t mean_off;   // offset of the instance's d values in packed per-instance outputs
  int32_t ntiles;
  int32_t d;
  int32_t shape;      // load/lane layout (batch_shape)
  int32_t pad;
};
static_assert(sizeof(BatchInst) == 56, "instance record layout");

struct BatchTile {
  int32_t inst;
  int32_t pad;
  int64_t r0, r1;  // rows [r0, r1) of the instance
};

// Workspace of a batch: [counters 256 B][BatchHeader at 256][...] with the
// tables at the offsets the header records (written once by ses_batch_init).
struct BatchHeader {
  int64_t num, ntiles;
  int64_t inst_off, instcnt_off, tile_off, partial_off;
  int64_t search_off;
  int32_t dtype;        // PDSCP_F32 or PDSCP_BF16: the point type of ses_batch_*init
  int32_t ctas_per_sm;  // persistent grid of the search launches: 0 = the occupancy limit (ses_batch_set_launch)
};

// Device-side search of Sec. 3 for every instance of a batch (the rules of
// ses_solve, run by the CTA that finishes an instance's iteration), in phases:
constexpr int kPhaseBounds = 0;  // evaluation pass at v_1: f(v_1) = D of Sec. 4.1
constexpr int kPhaseFtp = 1;     // an alpha-FTP is running
constexpr int kPhaseFinal = 2;   // evaluation pass at the mean the FTP ended with
constexpr int kPhaseDone = 3;

struct BatchSearch {
  double D, rho, logr;        // Sec. 4.1 constants of the instance
  double L, U, lb, ub;        // search range and certificates
  double alpha, eps_i, eta_over_rho;
  int64_t T, cap, total;      // theorem count of this FTP, its iteration cap, iterations so far
  int32_t steps, phase, status, why;  // why: how a CERTIFIED FTP ended (kWhy*)
  double eta_c;               // CERTIFIED: the current step size
  double last_gap, next_check;  // CERTIFIED: progress test of the running FTP
  float center[kBatchMaxD];   // the centre achieving ub
};
static_assert(sizeof(BatchSearch) == 400, "search record layout");

struct BatchSolveOpts {
  double eps, delta, eta;     // eta <= 0: eta_i = sqrt(ln r / T_i) (Theorem 2); CERTIFIED: 1
  int64_t max_iters;          // per instance
  int32_t patience, rules, max_steps, mode;  // mode: PDSCP_MODE_*
  int32_t poll, pad;          // CERTIFIED: iterations between certificate tests
};

// How a CERTIFIED alpha-FTP ended besides the device's own stop (ses_solve's rules).
constexpr int kWhyBudget = 0;  // its iteration cap
constexpr int kWhyClosed = 1;  // the certificates closed at a poll
constexpr int kWhyStuck = 2;   // its own gap stopped shrinking: eta is halved
constexpr double kCertFirstCheck = 1024.0;  // first progress test at eta = 1 (1024/eta in general)
constexpr double kCertShrink = 0.8;         // the FTP's own gap must shrink by this while t doubles
constexpr double kCertMinEta = 1.0 / 64.0;  // eta is not halved below this

// The search options live in the workspace at this offset (after the header).
constexpr size_t kBatchOptsOff = 512;

struct BatchParams {
  const void* pts;             // packed rows of the kernels' point type T
  const double* alpha;         // per instance (plain iterations)
  const double* eta_over_rho;  // per instance (plain iterations)
  unsigned char* ws;           // workspace base
  pdscp_step_out* out;         // per instance, may be null
  BatchSearch* search;         // non-null: device-side search; alpha, eta/rho come from here
};

// Load/lane layouts, chosen on the host per instance:
//   0..4: 4-element chunks, LPP = 1, 2, 4, 8, 16 (d = 4 * LPP or less, d % 4 == 0, rows aligned
//        to 4 elements: one 16-byte load per chunk for float32, one 8-byte load for bfloat16)
//   9: scalar, one lane per point (d <= 4: a warp covers 32 consecutive short
//      rows, and each point's exponentials run once, not on several lanes);
//   6: scalar, 8 lanes (d <= 8); 7: scalar, 32 lanes (d <= 32);
//   8: scalar, 32 lanes x 2 (d <= 64); 5 (2 lanes, d <= 2) is kept for callers of old tables
__host__ __device__ inline int batch_shape(int d, bool aligned4) {
  if (d % 4 == 0 && aligned4) {
    const int c = d / 4;
    return c <= 1 ? 0 : c <= 2 ? 1 : c <= 4 ? 2 : c <= 8 ? 3 : 4;
  }
  return d <= 4 ? 9 : d <= 8 ? 6 : d <= 32 ? 7 : 8;
}

// Streams rows [r0, r1) of one instance at mean ubar (in shared memory, FP32)
// and leaves the CTA's totals in sG/s_sc (per warp). Same per-point
// arithmetic as ses_iter_kernel (rows 0 of the instance, v_1, excluded).
template <typename T, int VW, int LPP, int NCH, int U>
__device__ void batch_tile(const T* pts, int d, int64_t r0, int64_t r1, const float* s_ub, float kr, float H,
                           float alpha, float* sG, float (*s_sc)[4], float* s_cs) {
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  float ub[NCH][VW], G[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      ub[j][e] = (c < nch) ? s_ub[c * VW + e] : 0.f;
      G[j][e] = 0.f;
    }
  }
  float S = 0.f, W = 0.f, maxd = -INFINITY;
  s_cs[threadIdx.x] = 0.f;  // per-lane sum of the ORACLE coefficients (shared: no register in the loop)
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
        for (int e = 0; e < VW; ++e) {
          x[u][j][e] -= ub[j][e];
          part = fmaf(x[u][j][e], x[u][j][e], part);
        }
      const float dist2 = group_sum<LPP>(part);
      float c = 0.f;
      if (i >= 1 && i < r1) {
        const float dist = sqrtf(dist2);
        const float E1 = expf(kr * (dist - H));
        const float em = -expm1f(-2.f * kr * dist);
        const float dif = E1 * em;
        const float sum = E1 * (2.f - em);
        c = dist > 0.f ? dif / dist : 2.f * kr * E1;
        if (gl == 0) {
          S += sum;
          W += alpha * sum - dist * dif;
          s_cs[threadIdx.x] += c;
          maxd = fmaxf(maxd, dist);
        }
      }
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) G[j][e] = fmaf(c, x[u][j][e], G[j][e]);
    }
  }
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
      for (int e = 0; e < VW; ++e) G[j][e] += __shfl_xor_sync(0xffffffffu, G[j][e], o);
  S = warp_sum(S);
  const float Cs = warp_sum(s_cs[threadIdx.x]);
  W = warp_sum(W);
  maxd = warp_max(maxd);
  if (grp == 0) {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int c = gl + j * LPP;
      if (c < nch)
#pragma unroll
        for (int e = 0; e < VW; ++e) sG[warp * kBatchMaxD + c * VW + e] = G[j][e];
    }
  }
  if (lane == 0) {
    s_sc[warp][0] = S;
    s_sc[warp][1] = W;
    s_sc[warp][2] = maxd;
    s_sc[warp][3] = Cs;
  }
}

// One warp, after the instance's finish: advances the instance's search
// (the decisions of ses_solve: Sec. 3's update of [L, U] from the FTP's
// outcome, Sec. 5's early exits, the lower bounds of Eq. primal_construction
// and of the averaged QP weights as certificates; in CERTIFIED mode only
// proven conclusions, polls every o.poll iterations) and starts its next
// alpha-FTP.
// Runs in its own kernel after each iteration launch (ses_batch_search_kernel):
// called from the streaming kernel, its FP64 bookkeeping would raise that
// kernel's register count and lower its occupancy.
template <typename T>
static __device__ __forceinline__ void batch_search_update(BatchSearch* sr, void* state, const T* v1, int d,
                                                        int64_t n, const BatchSolveOpts& o,
                                                        unsigned int* done_counter) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  StateHdr* hdr = reinterpret_cast<StateHdr*>(state);
  const StateHdr h = *hdr;  // written by lane 0 of this warp before the __syncwarp
  BatchSearch r = *sr;
  const bool cert = o.mode == PDSCP_MODE_CERTIFIED;
  bool end_ftp = false, start_ftp = false, done = false;
  if (h.status != PDSCP_OK) {
    r.status = h.status;
    done = true;
  } else if (r.phase == kPhaseBounds) {
    r.D = h.hint;  // max_{i>=2} |v_1 - v_i| from the evaluation pass at v_1
    if (!(r.D > 0.0)) {
      r.lb = r.ub = r.L = r.U = 0.0;
      done = true;
    } else {
      r.rho = 3.0 * r.D / kSqrt2;
      r.logr = log(2.0 * (double)(n - 1));
      r.L = r.D / 2.0;
      r.U = r.D;
      r.lb = 0.0;
      r.ub = INFINITY;
      r.eta_c = o.eta > 0.0 ? o.eta : 1.0;
      start_ftp = true;
    }
  } else if (r.phase == kPhaseFinal) {
    end_ftp = true;
  } else if (h.stopped) {
    end_ftp = true;
  } else if (h.t >= r.cap) {
    r.phase = kPhaseFinal;  // the next launch evaluates f at the final mean
  } else if (cert && h.t % o.poll == 0) {
    // a poll: the certificates closed, or the FTP's own gap stopped shrinking
    if (fmin(r.ub, h.best_f) <= (1.0 + o.eps) * fmax(fmax(r.lb, r.L), h.lb_best)) {
      r.why = kWhyClosed;
      r.phase = kPhaseFinal;
    } else if ((double)h.t >= r.next_check) {
      const double gap = h.lb_best > 0.0 ? h.best_f / h.lb_best - 1.0 : INFINITY;
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
    const bool better = h.best_f < r.ub;
    if (better) r.ub = h.best_f;
    for (int j = lane; j < d; j += 32)
      if (better) r.center[j] = state_best(state, d)[j];
    if (h.lb_best > r.lb) r.lb = h.lb_best;
    if (cert) {
      if (oc == PDSCP_OUT_SEPARATED) r.L = fmax(r.L, r.alpha);
      if (oc == PDSCP_OUT_RUNNING && r.why == kWhyStuck) r.eta_c *= 0.5;
      r.U = fmin(r.U, r.ub);
      r.L = fmax(r.L, r.lb);
      r.steps += 1;
      if (oc == PDSCP_OUT_RUNNING && r.why == kWhyBudget) {
        done = true;  // the iteration budget ended this FTP
      } else if (!(r.ub > (1.0 + o.eps) * fmax(r.lb, r.L) && r.total < o.max_iters && r.steps < o.max_steps)) {
        done = true;
      } else {
        start_ftp = true;
      }
      if (done) r.lb = fmax(r.lb, r.L);  // a separation is a proof too
    } else {
      if (oc == PDSCP_OUT_SEPARATED) {
        r.L = fmax(r.L, r.alpha);
      } else if (iters >= r.T || oc == PDSCP_OUT_STALLED || oc == PDSCP_OUT_BEAT_ALPHA) {
        r.U = fmin(fmin(r.U, (1.0 + r.eps_i) * r.alpha), r.ub);
      }
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
  if (start_ftp) {
    r.alpha = r.L + (r.U - r.L) / 3.0;
    r.eps_i = (r.U - r.L) / (3.0 * r.alpha);
    const double Tf = ceil(36.0 * r.D * r.D * r.logr / (r.eps_i * r.eps_i * r.alpha * r.alpha));
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
    // a fresh alpha-FTP: t = 0, mean = v_1 (as mwu_state_init)
    const int dp = dpad4(d);
    double* mean = state_mean(state);
    float* mean32 = state_mean32(state, d);
    float* best = state_best(state, d);
    for (int j = lane; j < dp; j += 32) {
      const double v = j < d ? (double)elem_to_float(v1 + j) : 0.0;
      mean[j] = v;
      mean32[j] = (float)v;
      best[j] = (float)v;
      state_dual(state, d)[j] = 0.0;
    }
    if (lane == 0) {
      StateHdr z;
      memset(&z, 0, sizeof(z));
      z.rules = o.rules;
      z.patience = o.patience;
      z.delta = o.delta;
      z.f_prev = -1.0;
      z.best_f = INFINITY;
      z.ub_best = INFINITY;
      *hdr = z;
    }
  }
  if (done) {
    if (!(r.ub < INFINITY) || !(r.D > 0.0)) {  // no FTP produced a centre: v_1 with radius D encloses every point
      r.ub = r.D;
      for (int j = lane; j < d; j += 32) r.center[j] = elem_to_float(v1 + j);
    }
    r.phase = kPhaseDone;
    if (lane == 0) {
      hdr->stopped = 1;  // the instance's tiles are skipped from now on
      atomicAdd(done_counter, 1u);
    }
  }
  __syncwarp();
  // scalars by lane 0; each lane already wrote its own centre entries
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

// batch_tile for rows of 4-element chunks (d = 4 .. 64, d % 4 == 0): each warp
// streams one contiguous part of the tile, NI points per lane per round (all
// loads of a round in flight together), and each point's scalar work runs
// once, on the lane that owns it after a reduce-scatter of the partial
// squared distances (GroupScatter), as in ses_iter_t_kernel.
template <typename T, int VW, int LPP, int NI>
__device__ void batch_tile_t(const T* pts, int d, int64_t r0, int64_t r1, const float* s_ub, float kr,
                             float H, float alpha, float* sG, float (*s_sc)[4], float* s_cs) {
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
  float ub[VW], G[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    ub[e] = has_chunk ? s_ub[gl * VW + e] : 0.f;
    G[e] = 0.f;
  }
  float S = 0.f, W = 0.f, maxd = -INFINITY;
  s_cs[threadIdx.x] = 0.f;  // per-lane sum of the ORACLE coefficients (shared: no register in the loop)
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
      for (int e = 0; e < VW; ++e) {
        x[r][e] -= ub[e];
        a = fmaf(x[r][e], x[r][e], a);
      }
      part[r] = has_chunk ? a : 0.f;
    }
    GS::run(part, gl);
    float c[GS::OWN];
#pragma unroll
    for (int k = 0; k < GS::OWN; ++k) {
      const int64_t i = base + GS::owned(gl, k) * PPW + grp;
      c[k] = 0.f;
      if (i >= 1 && i < hi) {  // instance row 0 is v_1, the easy cone
        const float dist = sqrtf(part[k]);
        const float E1 = expf(kr * (dist - H));
        const float em = -expm1f(-2.f * kr * dist);
        const float dif = E1 * em;
        const float sum = E1 * (2.f - em);
        c[k] = dist > 0.f ? dif / dist : 2.f * kr * E1;
        if (owner) {
          S += sum;
          W += alpha * sum - dist * dif;
          s_cs[threadIdx.x] += c[k];
          maxd = fmaxf(maxd, dist);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const float cr = __shfl_sync(0xffffffffu, c[r % GS::OWN], grp * LPP + GS::src_lane(r));
#pragma unroll
      for (int e = 0; e < VW; ++e) G[e] = fmaf(cr, x[r][e], G[e]);
    }
  }
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int e = 0; e < VW; ++e) G[e] += __shfl_xor_sync(0xffffffffu, G[e], o);
  S = warp_sum(S);
  const float Cs = warp_sum(s_cs[threadIdx.x]);
  W = warp_sum(W);
  maxd = warp_max(maxd);
  if (grp == 0 && has_chunk)
#pragma unroll
    for (int e = 0; e < VW; ++e) sG[warp * kBatchMaxD + gl * VW + e] = G[e];
  if (lane == 0) {
    s_sc[warp][0] = S;
    s_sc[warp][1] = W;
    s_sc[warp][2] = maxd;
    s_sc[warp][3] = Cs;
  }
}

// Three CTAs per SM: left free, the compiler gave this kernel 111 registers
// (two CTAs per SM); bounded, it needs 78 with no spill, and the extra warps
// raise the batched iteration from 4.9 to 5.9 TB/s.
template <typename T>
static __global__ void __launch_bounds__(kBatchBlock, 3) ses_batch_kernel(BatchParams p) {
  __shared__ float sG[kBatchWarps * kBatchMaxD];
  __shared__ float s_sc[kBatchWarps][4];
  __shared__ float s_cs[kBatchBlock];
  __shared__ float s_ub[kBatchMaxD];
  __shared__ float2 raw[kBatchStride];
  __shared__ double s_mean[kBatchMaxD];
  __shared__ double s_v1[kBatchMaxD];
  __shared__ double s_dual[kBatchMaxD];
  __shared__ float2 s_scr[kBatchBlock];
  __shared__ __align__(16) double s_hdr[sizeof(StateHdr) / 8];
  __shared__ long long s_tile;
  __shared__ bool s_flag;
  const int tid = threadIdx.x;
  auto opof = [](int pc) { return pc == 2 ? 1 : 0; };
  const BatchHeader bh = *reinterpret_cast<const BatchHeader*>(p.ws + 256);
  unsigned int* counters = reinterpret_cast<unsigned int*>(p.ws);  // [0] next tile, [1] CTAs done
  unsigned int* inst_counters = reinterpret_cast<unsigned int*>(p.ws + bh.instcnt_off);
  const BatchInst* insts = reinterpret_cast<const BatchInst*>(p.ws + bh.inst_off);
  const BatchTile* tiles = reinterpret_cast<const BatchTile*>(p.ws + bh.tile_off);
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
    const T* pts = static_cast<const T*>(p.pts) + in.pt_off;
    if (hdr->stopped != 0) {  // a stopped FTP (or a finished search) is left as is
      __syncthreads();
      continue;
    }
    const BatchSearch* sr = p.search ? p.search + tl.inst : nullptr;
    const int phase = sr ? sr->phase : kPhaseFtp;
    const bool eval = phase == kPhaseBounds || phase == kPhaseFinal;
    const double alpha_d = sr ? sr->alpha : p.alpha[tl.inst];
    const double eor_d = sr ? sr->eta_over_rho : p.eta_over_rho[tl.inst];
    {
      const float kr = eval ? 0.f : ses_kr(hdr->t, eor_d);
      const float H = (float)(hdr->hint + hdr->move);
      const float alpha = (float)alpha_d;
      const float* mean32 = state_mean32(state, d);
      if (tid < d) s_ub[tid] = mean32[tid];
      __syncthreads();
      switch (in.shape) {
        case 0: batch_tile_t<T, 4, 1, 8>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 1: batch_tile_t<T, 4, 2, 8>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 2: batch_tile_t<T, 4, 4, 8>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 3: batch_tile_t<T, 4, 8, 8>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 4: batch_tile_t<T, 4, 16, 8>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 5: batch_tile<T, 1, 2, 1, 4>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 6: batch_tile<T, 1, 8, 1, 4>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 7: batch_tile<T, 1, 32, 1, 4>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        case 9: batch_tile<T, 1, 1, 4, 4>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
        default: batch_tile<T, 1, 32, 2, 2>(pts, d, tl.r0, tl.r1, s_ub, kr, H, alpha, sG, s_sc, s_cs); break;
      }
      __syncthreads();
      float* prow = partials + (size_t)tile * kBatchStride;
      for (int j = tid; j < d; j += kBatchBlock) {
        float s = 0.f;
        for (int w = 0; w < kBatchWarps; ++w) s += sG[w * kBatchMaxD + j];
        prow[4 + j] = s;
      }
      if (tid == 0) {
        float s0 = 0.f, s1 = 0.f, s3 = 0.f, m = -INFINITY;
        for (int w = 0; w < kBatchWarps; ++w) {
          s0 += s_sc[w][0];
          s1 += s_sc[w][1];
          s3 += s_sc[w][3];
          m = fmaxf(m, s_sc[w][2]);
        }
        prow[0] = s0;
        prow[1] = s1;
        prow[2] = m;
        prow[3] = s3;
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
      {
        constexpr int HW = (int)(sizeof(StateHdr) / 8);
        if (tid < HW) s_hdr[tid] = reinterpret_cast<const double*>(hdr)[tid];
        const double* mean = state_mean(state);
        if (tid < d) {
          s_mean[tid] = mean[tid];
          s_v1[tid] = (double)elem_to_float(pts + tid);
          s_dual[tid] = state_dual(state, d)[tid];
        }
        const int st = 4 + dpad4(d);
        // rows of this instance: stride kBatchStride, the first st columns used
        reduce_rows(partials + (size_t)in.tile0 * kBatchStride, 0, in.ntiles, st, raw, s_scr, opof, kBatchStride);
        if (tid < 32) {
          ses_finish_warp(raw, s_mean, s_v1, *reinterpret_cast<const StateHdr*>(s_hdr), state, d, alpha_d, 0.0,
                          eor_d, eval ? 1 : 0, p.out ? p.out + tl.inst : nullptr, nullptr, s_dual);

        }
      }
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

// The search step of every instance still searching, one warp per instance,
// after the launch that ran the instance's iteration (or evaluation pass).
template <typename T>
static __global__ void __launch_bounds__(256) ses_batch_search_kernel(const T* pts, unsigned char* ws, int num) {
  const int inst = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (inst >= num) return;
  const BatchHeader* bh = reinterpret_cast<const BatchHeader*>(ws + 256);
  BatchSearch* sr = reinterpret_cast<BatchSearch*>(ws + bh->search_off) + inst;
  if (sr->phase == kPhaseDone) return;
  const BatchInst in = reinterpret_cast<const BatchInst*>(ws + bh->inst_off)[inst];
  batch_search_update(sr, ws + in.state_off, pts + in.pt_off, in.d, in.n,
                      *reinterpret_cast<const BatchSolveOpts*>(ws + kBatchOptsOff),
                      reinterpret_cast<unsigned int*>(ws) + 2);
}

// Fresh alpha-FTP states for every instance (t = 0, mean = v_1); one CTA per instance.
template <typename T>
static __global__ void ses_batch_init_kernel(const T* pts, const BatchInst* inst, unsigned char* ws,
                                      unsigned int* inst_counters) {
  const BatchInst in = inst[blockIdx.x];
  void* state = ws + in.state_off;
  const int d = in.d;
  const int dp = dpad4(d);
  double* mean = state_mean(state);
  float* mean32 = state_mean32(state, d);
  float* best = state_best(state, d);
  for (int j = threadIdx.x; j < dp; j += blockDim.x) {
    const double v = j < d ? (double)elem_to_float(pts + in.pt_off + j) : 0.0;
    mean[j] = v;
    mean32[j] = (float)v;
    best[j] = (float)v;
    state_dual(state, d)[j] = 0.0;
  }
  if (threadIdx.x == 0) {
    StateHdr h;
    memset(&h, 0, sizeof(h));
    h.rules = PDSCP_RULES_NONE;
    h.patience = 1;
    h.f_prev = -1.0;
    h.best_f = INFINITY;
    h.ub_best = INFINITY;
    *reinterpret_cast<StateHdr*>(state) = h;
    inst_counters[blockIdx.x] = 0u;
  }
}

// Lane layouts of every instance for a layout policy (0: 4-element chunks
// where d % 4 == 0 and the rows start on a 4-element boundary, otherwise
// the scalar layouts; 1: the scalar layouts only). elem: bytes per element.
static __global__ void batch_layout_kernel(BatchInst* inst, int num, const void* pts, int elem, int policy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= num) return;
  const bool aligned = ((uintptr_t)pts + (uintptr_t)inst[i].pt_off * (uintptr_t)elem) % (uintptr_t)(4 * elem) == 0;
  inst[i].shape = batch_shape(inst[i].d, aligned && policy == 0);
}

// Means and best centres of every instance, packed at inst.mean_off.
static __global__ void ses_batch_read_kernel(const BatchInst* inst, unsigned char* ws, float* mean_out, float* best_out) {
  const BatchInst in = inst[blockIdx.x];
  void* state = ws + in.state_off;
  for (int j = threadIdx.x; j < in.d; j += blockDim.x) {
    if (mean_out) mean_out[in.mean_off + j] = state_mean32(state, in.d)[j];
    if (best_out) best_out[in.mean_off + j] = state_best(state, in.d)[j];
  }
}

// Per-instance search results: reports and centres (packed at inst.mean_off).
static __global__ void ses_batch_solve_read_kernel(const BatchInst* inst, const BatchSearch* search, double eps,
                                            pdscp_report* rep, float* center_out) {
  const BatchInst in = inst[blockIdx.x];
  const BatchSearch& r = search[blockIdx.x];
  for (int j = threadIdx.x; j < in.d; j += blockDim.x)
    if (center_out) center_out[in.mean_off + j] = r.center[j];
  if (threadIdx.x == 0 && rep) {
    pdscp_report o;
    o.value = r.ub;
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
