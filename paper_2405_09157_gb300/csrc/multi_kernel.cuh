// Multi-candidate SES iteration: one streaming pass over the points advances
// K independent alpha-FTPs (Sec. 3 with the SES data of Sec. 4.1, Eq.
// implement and Eq. ses_oracle) that share the points but have their own
// alpha_j, eta_j/rho, running mean ubar_j and state: the K candidates of a
// K-ary search over alpha, or K restarts. Per point and candidate the
// arithmetic is that of ses_iter_kernel (ses_kernel.cuh): the distance to
// ubar_j, the SOC exponential's two eigenvalue exponentials, the trace and
// weighted sums; candidate j's partial row [S, Wt, maxd, 0, G'_1..G'_d]
// occupies columns [j st, (j+1) st) of the CTA's row (st = 4 + dp). The CTA
// that completes the pass reduces the rows and warp j runs candidate j's
// O(d) finish (ses_finish_warp). A stopped candidate contributes nothing and
// keeps its state. Per point the work is K times that of one candidate while
// the bytes read are the same: the pass stays bound by HBM only while the
// FP32 pipe keeps up (measured in the benchmark for K = 1..8).
#pragma once

#include "ses_kernel.cuh"

namespace pdscp {

constexpr int kMultiMaxK = 8;
constexpr int kMultiMaxD = 64;

struct MultiParams {
  const void* pts;
  const float* radii;  // may be null
  int64_t n;
  int d;
  int k;                        // candidates (== K of the instance)
  const double* alpha;          // k values (device)
  const double* eta_over_rho;   // k values (device)
  unsigned char* states;        // k states, state_stride bytes apart
  size_t state_stride;
  float* partials;              // one row of k * ses_partial_stride(d) floats per CTA
  float2* grows;
  unsigned int* counter;
  int single;
  pdscp_step_out* out;          // k records, may be null
};

// CTAs per SM: at least two from K = 4 on (with one, the register count of K
// means and K weighted sums per lane leaves 2 warps per scheduler and the
// pass stalls on instruction latency; K = 8 also keeps 2 points in flight
// per lane group instead of 4 to fit), three below (no spill either way).
// Measured at n = 1e6, d = 32: K = 8 132 -> 118 us per pass, K = 2 67 -> 64 us.
template <typename T, int VW, int LPP, int NCH, int U, int K>
__global__ void __launch_bounds__(kBlock, (K >= 4 ? 2 : 3)) ses_multi_kernel(MultiParams p) {
  using GS = GroupScatter<LPP, K>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float s_sc[kWarps][K][3];
  __shared__ float2 s_scr[kBlock];
  __shared__ __align__(16) double s_hdr[K][sizeof(StateHdr) / 8];
  __shared__ float s_kr[K], s_H[K], s_alpha[K];
  __shared__ int s_live[K];
  __shared__ bool s_flag;

  const int d = p.d;
  const int dp = dpad4(d);
  const int st = ses_partial_stride(d);
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;

  if (threadIdx.x < K) {
    const int q = threadIdx.x;
    const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.states + (size_t)q * p.state_stride);
    s_live[q] = hdr->stopped == 0;
    s_kr[q] = ses_kr(hdr->t, p.eta_over_rho[q]);
    s_H[q] = (float)(hdr->hint + hdr->move);
    s_alpha[q] = (float)p.alpha[q];
  }
  float ub[K][NCH][VW], G[K][NCH][VW];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float* mean32 = state_mean32(p.states + (size_t)q * p.state_stride, d);
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int c = gl + j * LPP;
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        ub[q][j][e] = (c < nch) ? mean32[c * VW + e] : 0.f;
        G[q][j][e] = 0.f;
      }
    }
  }
  __syncthreads();
  // the scalar work of a (point, candidate) pair is done once, by the lane
  // that owns the candidate after the reduce-scatter of the partial distances
  float S[GS::OWN], W[GS::OWN], maxd[GS::OWN];
  float okr[GS::OWN], oH[GS::OWN], oal[GS::OWN];
  bool olive[GS::OWN];
#pragma unroll
  for (int k = 0; k < GS::OWN; ++k) {
    const int q = GS::owned(gl, k);
    S[k] = 0.f;
    W[k] = 0.f;
    maxd[k] = -INFINITY;
    okr[k] = s_kr[q];
    oH[k] = s_H[q];
    oal[k] = s_alpha[q];
    olive[k] = s_live[q] != 0;
  }
  const bool acc_owner = (gl % GS::SHARE) == 0;

  const T* pts = reinterpret_cast<const T*>(p.pts);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  for (int64_t base = gw * (PPW * U); base < p.n; base += nwarps * (PPW * U)) {
    // from K = 4 on, lane 0 asks L2 for the warp's next chunk while this one
    // is processed (measured at n = 1e6, d = 32: K = 4 79.4 -> 78.3 us, K = 8
    // 118.2 -> 114.8 us; K = 1, 2 lost 1.5-2 us and go without)
    if constexpr (K >= 4 && VW * sizeof(T) == 16 && NCH == 1) {
      const int64_t pb = base + nwarps * (PPW * U);
      if (lane == 0 && pb < p.n) {
        const int64_t m = p.n - pb < (PPW * U) ? p.n - pb : (PPW * U);
        const unsigned int bytes = (unsigned int)(m * d * (int64_t)sizeof(T));  // whole 16-byte chunks
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(pts + pb * d), "r"(bytes) : "memory");
      }
    }
    float x[U][NCH][VW];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        if (i < p.n && c < nch) {
          Chunk<T, VW>::load(pts + i * d, c, x[u][j]);
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e) x[u][j][e] = 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      const bool cone = i >= 1 && i < p.n;
      const float gam = (cone && p.radii) ? __ldg(p.radii + i) : 0.f;
      float v[K];
#pragma unroll
      for (int q = 0; q < K; ++q) {
        float part = 0.f;
#pragma unroll
        for (int j = 0; j < NCH; ++j)
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            const float dl = x[u][j][e] - ub[q][j][e];
            part = fmaf(dl, dl, part);
          }
        v[q] = part;
      }
      GS::run(v, gl);
      float cown[GS::OWN];
#pragma unroll
      for (int k = 0; k < GS::OWN; ++k) {
        cown[k] = 0.f;
        if (cone && olive[k]) {
          const float kr = okr[k];
          const float dist = sqrtf(v[k]);
          const float a = oal[k] - gam;
          const float E1 = expf(kr * ((dist + gam) - oH[k]));
          const float em = -expm1f(-2.f * kr * dist);
          const float dif = E1 * em;
          const float sum = E1 * (2.f - em);
          cown[k] = dist > 0.f ? dif / dist : 2.f * kr * E1;
          if (acc_owner) {
            S[k] += sum;
            W[k] += a * sum - dist * dif;
            maxd[k] = fmaxf(maxd[k], dist + gam);
          }
        }
      }
      const int gbase = lane & ~(LPP - 1);
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const float c = __shfl_sync(0xffffffffu, cown[q % GS::OWN], gbase + GS::src_lane(q));
#pragma unroll
        for (int j = 0; j < NCH; ++j)
#pragma unroll
          for (int e = 0; e < VW; ++e) G[q][j][e] = fmaf(c, x[u][j][e] - ub[q][j][e], G[q][j][e]);
      }
    }
  }

  // owners' scalar totals: across the lane groups of the warp (same gl)
#pragma unroll
  for (int k = 0; k < GS::OWN; ++k) {
#pragma unroll
    for (int o = LPP; o < 32; o <<= 1) {
      S[k] += __shfl_xor_sync(0xffffffffu, S[k], o);
      W[k] += __shfl_xor_sync(0xffffffffu, W[k], o);
      maxd[k] = fmaxf(maxd[k], __shfl_xor_sync(0xffffffffu, maxd[k], o));
    }
    if (grp == 0 && acc_owner) {
      const int q = GS::owned(gl, k);
      s_sc[warp][q][0] = S[k];
      s_sc[warp][q][1] = W[k];
      s_sc[warp][q][2] = maxd[k];
    }
  }

  // CTA reduction of G' per candidate: lane groups of a warp, then warps
  float* sG = reinterpret_cast<float*>(smem_raw);  // [kWarps][K][dp]
#pragma unroll
  for (int q = 0; q < K; ++q) {
#pragma unroll
    for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) G[q][j][e] += __shfl_xor_sync(0xffffffffu, G[q][j][e], o);
    if (grp == 0) {
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        if (c < nch)
#pragma unroll
          for (int e = 0; e < VW; ++e) sG[(warp * K + q) * dp + c * VW + e] = G[q][j][e];
      }
    }
  }
  __syncthreads();
  const int wst = K * st;  // the CTA's row: K candidate rows side by side
  float* prow = p.partials + (size_t)blockIdx.x * wst;
  for (int idx = threadIdx.x; idx < K * dp; idx += kBlock) {
    const int q = idx / dp, j = idx % dp;
    float s = 0.f;
    if (j < d)
      for (int w = 0; w < kWarps; ++w) s += sG[(w * K + q) * dp + j];
    prow[q * st + 4 + j] = s;
  }
  if (threadIdx.x < K) {
    const int q = threadIdx.x;
    float s0 = 0.f, s1 = 0.f, m = -INFINITY;
    for (int w = 0; w < kWarps; ++w) {
      s0 += s_sc[w][q][0];
      s1 += s_sc[w][q][1];
      m = fmaxf(m, s_sc[w][q][2]);
    }
    prow[q * st + 0] = s0;
    prow[q * st + 1] = s1;
    prow[q * st + 2] = m;
    prow[q * st + 3] = 0.f;
  }

  // completion: the last CTA reduces the rows; warp q finishes candidate q
  auto opof = [st](int pc) { return (pc % st) == 2 ? 1 : 0; };
  if (!arrive_pass(p.partials, wst, p.grows, p.counter, s_scr, &s_flag, opof, p.single)) return;
  // dynamic shared memory: totals (K st pairs) | K means | v_1 | staged rows
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  double* s_mean = reinterpret_cast<double*>(smem_raw) + wst;
  double* s_v1 = s_mean + K * dp;
  float* stage = reinterpret_cast<float*>(s_v1 + dp);
  constexpr int HW = (int)(sizeof(StateHdr) / 8);
  // loads the finishes need, issued before the reduction so that their latency overlaps it
  for (int idx = threadIdx.x; idx < K * HW; idx += kBlock) {
    const int q = idx / HW, w = idx % HW;
    s_hdr[q][w] = reinterpret_cast<const double*>(p.states + (size_t)q * p.state_stride)[w];
  }
  double mreg[(K * kMultiMaxD + kBlock - 1) / kBlock];
#pragma unroll
  for (int r = 0; r < (K * kMultiMaxD + kBlock - 1) / kBlock; ++r) {
    const int idx = threadIdx.x + r * kBlock;
    const int q = idx / dp, j = idx % dp;
    mreg[r] = (q < K && j < d) ? state_mean(p.states + (size_t)q * p.state_stride)[j] : 0.0;
  }
  const double v0 = threadIdx.x < d ? (double)elem_to_float<T>(pts + threadIdx.x) : 0.0;
  final_reduce(p.partials, wst, p.grows, p.counter, s_scr, opof, raw, stage, p.single, 2, -1, st);
#pragma unroll
  for (int r = 0; r < (K * kMultiMaxD + kBlock - 1) / kBlock; ++r) {
    const int idx = threadIdx.x + r * kBlock;
    if (idx < K * dp) s_mean[idx] = mreg[r];
  }
  if (threadIdx.x < d) s_v1[threadIdx.x] = v0;
  __syncthreads();
  if (warp >= K) return;
  const int q = warp;
  const double gam1 = p.radii ? (double)__ldg(p.radii) : 0.0;
  const StateHdr& h = *reinterpret_cast<const StateHdr*>(s_hdr[q]);
  if (h.stopped) return;  // a stopped FTP is left as is (as mwu_step)
  ses_finish_warp(raw + q * st, s_mean + q * dp, s_v1, h, p.states + (size_t)q * p.state_stride, d, p.alpha[q],
                  gam1, p.eta_over_rho[q], 0, p.out ? p.out + q : nullptr);
}

}  // namespace pdscp
