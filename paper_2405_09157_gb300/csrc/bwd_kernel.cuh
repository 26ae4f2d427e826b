// Reverse sweep through the unrolled SES alpha-FTP (Sec. 3, Eq. implement with
// the ORACLE of Eq. ses_oracle) at fixed alpha and eta/rho: the gradient of
//   L = f(ubar^T) = max_i ||ubar^T - v_i|| + gamma_i        (f of Sec. 5)
// with respect to the points v_1..v_n.
//
// Forward step t (ubar = ubar^t, kr = eta t/(rho sqrt2), cones i >= 2):
//   delta_i = v_i - ubar, dist_i = |delta_i|, E1, E2 as in the iteration kernel
//   (the SOC exponential of Sec. 2.1, shifted by the tape's common factor),
//   s_i = E1 + E2, c_i = (E1 - E2)/dist_i, S = sum s_i, G' = sum c_i delta_i,
//   g = G'/(sqrt2 S), u = v_1 + r g/|g| (r = alpha - gamma_1; u = v_1 if g = 0),
//   ubar^{t+1} = (t ubar^t + u)/(t + 1).
// Reverse step t, given B = dL/dubar^{t+1}:
//   B' = B/(t+1) reaches v_1 through u; with ghat = g/|g|,
//   gbar = (r/|g|)(B' - ghat (ghat . B')), Gbar = gbar/(sqrt2 S), Sbar = -(gbar . g)/S;
//   ds_i/ddist = kr (E1 - E2), dc_i/ddist = (kr s_i - c_i)/dist_i, so
//   dL/ddelta_i = c_i Gbar + beta_i delta_i,
//   beta_i = [(Gbar . delta_i)(kr s_i - c_i)/dist_i + Sbar kr (E1 - E2)]/dist_i,
//   (beta_i delta_i -> 0 as dist_i -> 0; beta_i = 0 at dist_i = 0);
//   dL/dv_i += dL/ddelta_i,  dL/dubar^t = t/(t+1) B - sum_i dL/ddelta_i.
// At t = 0 every exponent is 0 (g = 0, u = v_1): step 0 only hands B to v_1,
// and ubar^0 = v_1 receives nothing more (its coefficient t/(t+1) is 0).
// The common shift of E1 and E2 cancels in g and in its derivative, so the
// reverse pass reuses the forward's shift from the tape.
//
// Kernels: ses_bwd_argmax_kernel (i* = argmax of f at ubar^T, smallest index on
// ties), ses_bwd_seed_kernel (one CTA: B = dL/dubar^T, row i*, then the
// bookkeeping of step T-1), ses_bwd_step_kernel (one per step s = T-1 .. 1: a
// streaming pass that updates dL/dv_i for every cone and sums dL/ddelta_i,
// then the last CTA updates B and prepares step s-1). Steps the forward did
// not take (it stopped early) are skipped on the device.
#pragma once

#include "bf16_chunk4.cuh"

namespace pdscp {

// Adjoint scratch (in the workspace): B (double, dp) | v_1 adjoint (double,
// dp) | Gbar (float, dp) | Sbar (float) ...
__host__ __device__ inline size_t bwd_scratch_bytes(int d) {
  return (size_t)dpad4(d) * (8 + 8 + 4) + 16;
}

struct BwdParams {
  const void* pts;     // n x d rows of the kernels' point type T (float or bfloat16)
  const float* radii;  // may be null
  int64_t n;
  int d;
  double alpha;
  int64_t s;             // reverse step of this launch
  const void* state;     // the forward's final state: t = steps taken, mean = ubar^T
  const float* tape;     // forward tape, ses_tape_stride(d) floats per step
  unsigned char* bw;     // adjoint scratch
  float* grad;           // n x d, dL/dv
  float* partials;       // one row of ses_partial_stride(d) floats per CTA
  float2* grows;
  unsigned int* counter;
  int single;
  // argmax / seed
  float* cand_val;       // one candidate per CTA of the argmax pass
  long long* cand_idx;
  int ncand;
  const double* seed;    // dL/df (may be null: 1)
  pdscp_step_out* out;   // seed: f at ubar^T and the steps taken (may be null)
  const int8_t* labels;  // SVM: +1 (P) / -1 (Q) per row
};

// Row i of the points, as the kernels' point type T.
template <typename T>
__device__ __forceinline__ const T* bwd_row(const BwdParams& p, int64_t i) {
  return static_cast<const T*>(p.pts) + i * p.d;
}

__device__ __forceinline__ double* bwd_B(unsigned char* bw) { return reinterpret_cast<double*>(bw); }
__device__ __forceinline__ double* bwd_V1(unsigned char* bw, int d) {
  return reinterpret_cast<double*>(bw) + dpad4(d);
}
__device__ __forceinline__ float* bwd_Gbar(unsigned char* bw, int d) {
  return reinterpret_cast<float*>(reinterpret_cast<double*>(bw) + 2 * dpad4(d));
}
__device__ __forceinline__ float* bwd_Sbar(unsigned char* bw, int d) { return bwd_Gbar(bw, d) + dpad4(d); }

// Bookkeeping of reverse step s, run by one warp, given B = dL/dubar^{s+1} in
// the scratch: v_1's share B/(s+1), then Gbar and Sbar of step s from the
// tape; at s = 0 the accumulated v_1 adjoint goes to row 0 of grad.
static __device__ void bwd_prologue(int64_t s, const float* tape, int d, float rad, unsigned char* bw, float* grad) {
  const int lane = threadIdx.x & 31;
  const int dp = dpad4(d);
  double* B = bwd_B(bw);
  double* V1 = bwd_V1(bw, d);
  float* Gb = bwd_Gbar(bw, d);
  const double inv = 1.0 / (double)(s + 1);
  for (int j = lane; j < d; j += 32) V1[j] += B[j] * inv;
  if (s == 0) {
    for (int j = lane; j < d; j += 32) grad[j] += (float)V1[j];
    return;
  }
  const float* ent = tape + (size_t)s * ses_tape_stride(d);
  const float S = ent[0], ng = ent[1];
  const float* g = ent + 4 + dp;
  if (!(ng > 0.f)) {  // u = v_1 at this step: nothing flows to the cones
    for (int j = lane; j < d; j += 32) Gb[j] = 0.f;
    if (lane == 0) *bwd_Sbar(bw, d) = 0.f;
    return;
  }
  const float rng = 1.0f / ng;
  float dot1 = 0.f;
  for (int j = lane; j < d; j += 32) dot1 = fmaf(g[j] * rng, (float)(B[j] * inv), dot1);
  dot1 = warp_sum(dot1);
  const float scale = rad * rng;
  const float rS = 1.0f / S;
  const float gsc = rS * (float)(1.0 / kSqrt2);
  float dot2 = 0.f;
  for (int j = lane; j < d; j += 32) {
    const float gh = g[j] * rng;
    const float gb = scale * ((float)(B[j] * inv) - gh * dot1);
    dot2 = fmaf(gb, g[j], dot2);
    Gb[j] = gb * gsc;
  }
  dot2 = warp_sum(dot2);
  if (lane == 0) *bwd_Sbar(bw, d) = -dot2 * rS;
}

// One reverse step s >= 1: a streaming pass over the cones, then (last CTA)
// B <- s/(s+1) B - sum_i dL/ddelta_i and the bookkeeping of step s - 1.
template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) ses_bwd_step_kernel(BwdParams p) {
  pdl_trigger();
  pdl_wait();  // Gbar, Sbar and the gradient rows are the previous reverse step's output
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float2 s_scr[kMaxBlock];
  __shared__ bool s_flag;
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.state);
  if (p.s >= hdr->t) return;  // the forward stopped before step s

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  const float* ent = p.tape + (size_t)p.s * ses_tape_stride(d);
  const float kr = ent[2], H = ent[3];
  const float* ubar = ent + 4;
  const float* Gbar = bwd_Gbar(p.bw, d);
  const float Sbar = *bwd_Sbar(p.bw, d);

  float ub[NCH][VW], gb[NCH][VW], acc[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      ub[j][e] = (c < nch) ? ubar[c * VW + e] : 0.f;
      gb[j][e] = (c < nch) ? Gbar[c * VW + e] : 0.f;
      acc[j][e] = 0.f;
    }
  }
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  for (int64_t base = gw * (PPW * U); base < p.n; base += nwarps * (PPW * U)) {
    float x[U][NCH][VW];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        if (i < p.n && c < nch) {
          Chunk<T, VW>::load(bwd_row<T>(p, i), c, x[u][j]);
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e) x[u][j][e] = 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      float p2 = 0.f, pd = 0.f;
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          x[u][j][e] -= ub[j][e];  // delta_i = v_i - ubar
          p2 = fmaf(x[u][j][e], x[u][j][e], p2);
          pd = fmaf(gb[j][e], x[u][j][e], pd);
        }
      const float dist2 = group_sum<LPP>(p2);
      const float gdot = group_sum<LPP>(pd);
      float c = 0.f, beta = 0.f;
      const bool cone = i >= 1 && i < p.n;
      if (cone) {
        const float dist = sqrtf(dist2);
        const float gam = p.radii ? __ldg(p.radii + i) : 0.f;
        const float E1 = expf(kr * ((dist + gam) - H));
        const float em = -expm1f(-2.f * kr * dist);
        const float dif = E1 * em;          // E1 - E2
        const float sum = E1 * (2.f - em);  // E1 + E2
        if (dist > 0.f) {
          const float rd = 1.0f / dist;
          c = dif * rd;
          beta = (gdot * (kr * sum - c) * rd + Sbar * kr * dif) * rd;
        } else {
          c = 2.f * kr * E1;
        }
      }
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int ch = gl + j * LPP;
        float dd[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          dd[e] = cone ? fmaf(c, gb[j][e], beta * x[u][j][e]) : 0.f;
          acc[j][e] += dd[e];
        }
        if (cone && ch < nch) {
          float* gp = p.grad + i * d + ch * VW;
          if constexpr (VW == 4) {
            float4 v = *reinterpret_cast<float4*>(gp);
            v.x += dd[0]; v.y += dd[1]; v.z += dd[2]; v.w += dd[3];
            *reinterpret_cast<float4*>(gp) = v;
          } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) gp[e] += dd[e];
          }
        }
      }
    }
  }
  // CTA sum of dL/ddelta: across the lane groups of a warp, then across warps
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
      for (int e = 0; e < VW; ++e) acc[j][e] += __shfl_xor_sync(0xffffffffu, acc[j][e], o);
  float* sA = reinterpret_cast<float*>(smem_raw);  // [kWarps][dp]
  if (grp == 0) {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int c = gl + j * LPP;
      if (c < nch)
#pragma unroll
        for (int e = 0; e < VW; ++e) sA[warp * dp + c * VW + e] = acc[j][e];
    }
  }
  __syncthreads();
  const int st = ses_partial_stride(d);
  float* prow = p.partials + (size_t)blockIdx.x * st;
  for (int j = threadIdx.x; j < dp; j += kBlock) {
    float s = 0.f;
    if (j < d)
      for (int w = 0; w < kWarps; ++w) s += sA[w * dp + j];
    prow[4 + j] = s;
  }
  if (threadIdx.x < 4) prow[threadIdx.x] = 0.f;

  auto opof = [](int) { return 0; };
  if (!arrive_pass(p.partials, st, p.grows, p.counter, s_scr, &s_flag, opof, p.single)) return;
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  float* stage = reinterpret_cast<float*>(raw + st);
  final_reduce(p.partials, st, p.grows, p.counter, s_scr, opof, raw, stage, p.single, -1, -1, st);
  if (threadIdx.x >= 32) return;
  double* B = bwd_B(p.bw);
  const double keep = (double)p.s / (double)(p.s + 1);
  for (int j = lane; j < d; j += 32) B[j] = keep * B[j] - ((double)raw[4 + j].x + (double)raw[4 + j].y);
  __syncwarp();
  const float rad = (float)(p.alpha - (p.radii ? (double)__ldg(p.radii) : 0.0));
  bwd_prologue(p.s - 1, p.tape, d, rad, p.bw, p.grad);
}

// ses_bwd_step_kernel for rows of 16-byte chunks (at most 32 per row): NI
// points per lane per round, their gradient rows loaded with them, and the
// scalar work of each point (its exponentials, c_i, beta_i) done once, on the
// lane that owns it after a reduce-scatter of the two partial dot products.
template <typename T, int VW, int LPP, int NI>
__global__ void __launch_bounds__(kBlock) ses_bwd_step_t_kernel(BwdParams p) {
  using GS = GroupScatter<LPP, NI>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float2 s_scr[kMaxBlock];
  __shared__ bool s_flag;
  pdl_trigger();
  // the forward's state and tape were complete before the sweep began
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.state);
  if (p.s >= hdr->t) return;  // the forward stopped before step s

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = d / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  constexpr int ROUND = PPW * NI;
  const bool owner = (gl % GS::SHARE) == 0;
  const bool has_chunk = gl < nch;
  const float* ent = p.tape + (size_t)p.s * ses_tape_stride(d);
  const float kr = ent[2], H = ent[3];
  const float* ubar = ent + 4;
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  float x[NI][VW], gr[NI][VW];
  auto load_points = [&](int64_t base) {
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int64_t i = base + r * PPW + grp;
      if (i < p.n && has_chunk) {
        Chunk<T, VW>::load(bwd_row<T>(p, i), gl, x[r]);
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) x[r][e] = 0.f;
      }
    }
  };
  // the first round's points do not depend on the previous reverse step
  load_points(gw * ROUND);
  pdl_wait();  // Gbar, Sbar and the gradient rows are the previous step's output
  const float* Gbar = bwd_Gbar(p.bw, d);
  const float Sbar = *bwd_Sbar(p.bw, d);
  float ub[VW], gb[VW], acc[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    ub[e] = has_chunk ? ubar[gl * VW + e] : 0.f;
    gb[e] = has_chunk ? Gbar[gl * VW + e] : 0.f;
    acc[e] = 0.f;
  }
  for (int64_t base = gw * ROUND; base < p.n; base += nwarps * ROUND) {
    if (base != gw * ROUND) load_points(base);
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int64_t i = base + r * PPW + grp;
      if (i < p.n && has_chunk) {
        const float4 g4 = *reinterpret_cast<const float4*>(p.grad + i * d + gl * VW);
        gr[r][0] = g4.x; gr[r][1] = g4.y; gr[r][2] = g4.z; gr[r][3] = g4.w;
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) gr[r][e] = 0.f;
      }
    }
    float p2[NI], pd[NI];
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        x[r][e] -= ub[e];  // delta_i = v_i - ubar
        a = fmaf(x[r][e], x[r][e], a);
        b = fmaf(gb[e], x[r][e], b);
      }
      p2[r] = has_chunk ? a : 0.f;
      pd[r] = has_chunk ? b : 0.f;
    }
    GS::run(p2, gl);
    GS::run(pd, gl);
    float cown[GS::OWN], bown[GS::OWN];
#pragma unroll
    for (int k = 0; k < GS::OWN; ++k) {
      const int64_t i = base + GS::owned(gl, k) * PPW + grp;
      cown[k] = 0.f;
      bown[k] = 0.f;
      if (i >= 1 && i < p.n) {
        const float dist = sqrtf(p2[k]);
        const float gam = p.radii ? __ldg(p.radii + i) : 0.f;
        const float E1 = expf(kr * ((dist + gam) - H));
        const float em = -expm1f(-2.f * kr * dist);
        const float dif = E1 * em;
        const float sum = E1 * (2.f - em);
        if (dist > 0.f) {
          const float rd = 1.0f / dist;
          const float c = dif * rd;
          cown[k] = c;
          bown[k] = (pd[k] * (kr * sum - c) * rd + Sbar * kr * dif) * rd;
        } else {
          cown[k] = 2.f * kr * E1;
        }
      }
    }
    (void)owner;
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int src = grp * LPP + GS::src_lane(r);
      const float cr = __shfl_sync(0xffffffffu, cown[r % GS::OWN], src);
      const float br = __shfl_sync(0xffffffffu, bown[r % GS::OWN], src);
      const int64_t i = base + r * PPW + grp;
      float dd[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        dd[e] = fmaf(cr, gb[e], br * x[r][e]);
        acc[e] += dd[e];
      }
      if (i >= 1 && i < p.n && has_chunk) {
        float4 v;
        v.x = gr[r][0] + dd[0]; v.y = gr[r][1] + dd[1]; v.z = gr[r][2] + dd[2]; v.w = gr[r][3] + dd[3];
        *reinterpret_cast<float4*>(p.grad + i * d + gl * VW) = v;
      }
    }
  }
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int e = 0; e < VW; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
  float* sA = reinterpret_cast<float*>(smem_raw);  // [kWarps][dp]
  if (grp == 0 && has_chunk)
#pragma unroll
    for (int e = 0; e < VW; ++e) sA[warp * dp + gl * VW + e] = acc[e];
  __syncthreads();
  const int st = ses_partial_stride(d);
  float* prow = p.partials + (size_t)blockIdx.x * st;
  for (int j = threadIdx.x; j < dp; j += kBlock) {
    float sum = 0.f;
    if (j < d)
      for (int w = 0; w < kWarps; ++w) sum += sA[w * dp + j];
    prow[4 + j] = sum;
  }
  if (threadIdx.x < 4) prow[threadIdx.x] = 0.f;

  auto opof = [](int) { return 0; };
  if (!arrive_pass(p.partials, st, p.grows, p.counter, s_scr, &s_flag, opof, p.single)) return;
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  float* stage = reinterpret_cast<float*>(raw + st);
  final_reduce(p.partials, st, p.grows, p.counter, s_scr, opof, raw, stage, p.single, -1, -1, st);
  if (threadIdx.x >= 32) return;
  double* B = bwd_B(p.bw);
  const double keep = (double)p.s / (double)(p.s + 1);
  for (int j = lane; j < d; j += 32) B[j] = keep * B[j] - ((double)raw[4 + j].x + (double)raw[4 + j].y);
  __syncwarp();
  const float rad = (float)(p.alpha - (p.radii ? (double)__ldg(p.radii) : 0.0));
  bwd_prologue(p.s - 1, p.tape, d, rad, p.bw, p.grad);
}

// argmax_i dist(ubar^T, v_i) + gamma_i over every row (v_1 included): one
// candidate (value, smallest index) per CTA.
template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) ses_bwd_argmax_kernel(BwdParams p) {
  __shared__ float s_val[kWarps];
  __shared__ long long s_idx[kWarps];
  const int d = p.d;
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  const float* mean32 = state_mean32(const_cast<void*>(p.state), d);
  float ub[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) ub[j][e] = (c < nch) ? mean32[c * VW + e] : 0.f;
  }
  float best = -INFINITY;
  long long bidx = 0x7fffffffffffffffLL;
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  for (int64_t base = gw * (PPW * U); base < p.n; base += nwarps * (PPW * U)) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      float part = 0.f;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        float x[VW];
        if (i < p.n && c < nch) {
          Chunk<T, VW>::load(bwd_row<T>(p, i), c, x);
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            const float dl = x[e] - ub[j][e];
            part = fmaf(dl, dl, part);
          }
        }
      }
      const float dist2 = group_sum<LPP>(part);
      if (i < p.n) {
        const float v = sqrtf(dist2) + (p.radii ? __ldg(p.radii + i) : 0.f);
        if (v > best || (v == best && i < bidx)) {
          best = v;
          bidx = i;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ov > best || (ov == best && oi < bidx)) {
      best = ov;
      bidx = oi;
    }
  }
  if (lane == 0) {
    s_val[warp] = best;
    s_idx[warp] = bidx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float bv = s_val[0];
    long long bi = s_idx[0];
    for (int w = 1; w < kWarps; ++w)
      if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bi)) {
        bv = s_val[w];
        bi = s_idx[w];
      }
    p.cand_val[blockIdx.x] = bv;
    p.cand_idx[blockIdx.x] = bi;
  }
}

// One CTA: picks i* from the candidates, seeds B = dL/dubar^T = seed (ubar^T -
// v_i*)/|ubar^T - v_i*| and row i* of grad, then the bookkeeping of step T-1.
template <typename PT>  // the point type; a template, so only the launching units instantiate it
__global__ void __launch_bounds__(32) ses_bwd_seed_kernel(BwdParams p) {
  const int lane = threadIdx.x;
  const int d = p.d;
  float bv = -INFINITY;
  long long bi = 0x7fffffffffffffffLL;
  for (int k = lane; k < p.ncand; k += 32) {
    const float v = p.cand_val[k];
    const long long i = p.cand_idx[k];
    if (v > bv || (v == bv && i < bi)) {
      bv = v;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.state);
  const int64_t T = hdr->t;
  const float* mean32 = state_mean32(const_cast<void*>(p.state), d);
  const PT* row = bwd_row<PT>(p, bi);
  // the direction in FP32 from the values the argmax pass compared
  float n2 = 0.f;
  for (int j = lane; j < d; j += 32) {
    const float dl = mean32[j] - elem_to_float(row + j);
    n2 = fmaf(dl, dl, n2);
  }
  n2 = warp_sum(n2);
  const float rn = n2 > 0.f ? 1.0f / sqrtf(n2) : 0.f;  // f is not differentiable at a zero distance: 0
  const double sd = p.seed ? *p.seed : 1.0;
  double* B = bwd_B(p.bw);
  double* V1 = bwd_V1(p.bw, d);
  for (int j = lane; j < d; j += 32) {
    const double dir = (double)((mean32[j] - elem_to_float(row + j)) * rn);
    B[j] = sd * dir;
    V1[j] = 0.0;
    p.grad[bi * d + j] -= (float)(sd * dir);
  }
  __syncwarp();
  if (lane == 0 && p.out) {
    pdscp_step_out o;
    o.oracle_value = hdr->last_value;
    o.objective = (double)bv;
    o.lower_bound = hdr->lb_best;
    o.upper_bound = (double)bv;
    o.t = T;
    o.failed = hdr->outcome == PDSCP_OUT_SEPARATED ? 1 : 0;
    o.stopped = hdr->stopped;
    o.status = hdr->status;
    o.outcome = hdr->outcome;
    o.k = (double)bi;  // the row that attains f
    o.dual_bound = 0.0;
    *p.out = o;
  }
  if (T == 0) {  // ubar^0 = v_1
    for (int j = lane; j < d; j += 32) p.grad[j] += (float)B[j];
    return;
  }
  const float rad = (float)(p.alpha - (p.radii ? (double)__ldg(p.radii) : 0.0));
  bwd_prologue(T - 1, p.tape, d, rad, p.bw, p.grad);
}

// ---------------------------------------------------------------------------
// SVM (Sec. 4.2, the minimisation variant of Sec. 3): gradient of
//   L = f(wbar^T) = (min_P x^T wbar - max_Q x^T wbar)/|wbar|   (0 when clipped)
// Forward step t (wbar = wbar^t, k = eta t/rho, Hm the tape's shift):
//   m_i = y_i x_i^T wbar - sbar_c(i), pt_i = e^{-k (m_i - Hm)}, S = sum pt_i,
//   z = sum_i y_i pt_i x_i / S, w = z/|z|, wbar^{t+1} = (t wbar + w)/(t+1).
//   s_1, s_2 are piecewise constant in the points: nothing flows through them.
// Reverse step t, given B = dL/dwbar^{t+1}: B' = B/(t+1),
//   zbar = (B' - what (what . B'))/|z|, zeta = zbar/S, Sbar = -(zbar . z)/S;
//   dL/dx_i += pt_i y_i zeta + beta_i wbar, beta_i = -k pt_i (x_i . zeta + y_i Sbar),
//   dL/dwbar^t = t/(t+1) B + sum_i beta_i x_i.
// Step t = 0 is a full reverse step here (uniform weights; w depends on the
// points); wbar^0 = 0 receives nothing.

// Bookkeeping of SVM reverse step s (one warp), given B = dL/dwbar^{s+1}:
// zeta (in the Gbar slot) and Sbar of step s from the tape.
static __device__ void svm_bwd_prologue(int64_t s, const float* tape, int d, unsigned char* bw) {
  const int lane = threadIdx.x & 31;
  const int dp = dpad4(d);
  const double* B = bwd_B(bw);
  float* zeta = bwd_Gbar(bw, d);
  const float inv = (float)(1.0 / (double)(s + 1));
  const float* ent = tape + (size_t)s * svm_tape_stride(d);
  const float S = ent[0], nz = ent[1];
  const float* z = ent + 8 + dp;
  if (!(nz > 0.f)) {  // w = 0 at this step: nothing flows to the points
    for (int j = lane; j < d; j += 32) zeta[j] = 0.f;
    if (lane == 0) *bwd_Sbar(bw, d) = 0.f;
    return;
  }
  const float rnz = 1.0f / nz;
  float dot1 = 0.f;
  for (int j = lane; j < d; j += 32) dot1 = fmaf(z[j] * rnz, (float)B[j] * inv, dot1);
  dot1 = warp_sum(dot1);
  const float rS = 1.0f / S;
  float dot2 = 0.f;
  for (int j = lane; j < d; j += 32) {
    const float zb = ((float)B[j] * inv - z[j] * rnz * dot1) * rnz;
    dot2 = fmaf(zb, z[j], dot2);
    zeta[j] = zb * rS;
  }
  dot2 = warp_sum(dot2);
  if (lane == 0) *bwd_Sbar(bw, d) = -dot2 * rS;
}

template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) svm_bwd_step_kernel(BwdParams p) {
  pdl_trigger();
  pdl_wait();  // the adjoint scratch and the gradient rows are the previous reverse step's output
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float2 s_scr[kMaxBlock];
  __shared__ bool s_flag;
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.state);
  if (p.s >= hdr->t) return;  // the forward stopped before step s

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  const float* ent = p.tape + (size_t)p.s * svm_tape_stride(d);
  const float k = ent[2], Hm = ent[3], s1 = ent[4], s2 = ent[5];
  const float* wbar = ent + 8;
  const float* zeta = bwd_Gbar(p.bw, d);
  const float Sbar = *bwd_Sbar(p.bw, d);

  float wb[NCH][VW], zt[NCH][VW], acc[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      wb[j][e] = (c < nch) ? wbar[c * VW + e] : 0.f;
      zt[j][e] = (c < nch) ? zeta[c * VW + e] : 0.f;
      acc[j][e] = 0.f;
    }
  }
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  for (int64_t base = gw * (PPW * U); base < p.n; base += nwarps * (PPW * U)) {
    float x[U][NCH][VW];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        if (i < p.n && c < nch) {
          Chunk<T, VW>::load(bwd_row<T>(p, i), c, x[u][j]);
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e) x[u][j][e] = 0.f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      float pw = 0.f, pz = 0.f;
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          pw = fmaf(x[u][j][e], wb[j][e], pw);
          pz = fmaf(x[u][j][e], zt[j][e], pz);
        }
      const float dw = group_sum<LPP>(pw);
      const float dz = group_sum<LPP>(pz);
      const bool row = i < p.n;
      float py = 0.f, beta = 0.f;
      if (row) {
        const bool pos = __ldg(p.labels + i) > 0;
        const float margin = pos ? dw - s1 : -dw - s2;
        const float pt = expf(-k * (margin - Hm));
        const float y = pos ? 1.f : -1.f;
        py = pt * y;
        beta = -k * pt * (dz + y * Sbar);
      }
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int ch = gl + j * LPP;
        float dd[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          dd[e] = fmaf(py, zt[j][e], beta * wb[j][e]);
          acc[j][e] = fmaf(beta, x[u][j][e], acc[j][e]);
        }
        if (row && ch < nch) {
          float* gp = p.grad + i * d + ch * VW;
          if constexpr (VW == 4) {
            float4 v = *reinterpret_cast<float4*>(gp);
            v.x += dd[0]; v.y += dd[1]; v.z += dd[2]; v.w += dd[3];
            *reinterpret_cast<float4*>(gp) = v;
          } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) gp[e] += dd[e];
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
      for (int e = 0; e < VW; ++e) acc[j][e] += __shfl_xor_sync(0xffffffffu, acc[j][e], o);
  float* sA = reinterpret_cast<float*>(smem_raw);  // [kWarps][dp]
  if (grp == 0) {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int c = gl + j * LPP;
      if (c < nch)
#pragma unroll
        for (int e = 0; e < VW; ++e) sA[warp * dp + c * VW + e] = acc[j][e];
    }
  }
  __syncthreads();
  const int st = ses_partial_stride(d);  // [0, 0, 0, 0, sum_i beta_i x_i]
  float* prow = p.partials + (size_t)blockIdx.x * st;
  for (int j = threadIdx.x; j < dp; j += kBlock) {
    float sum = 0.f;
    if (j < d)
      for (int w = 0; w < kWarps; ++w) sum += sA[w * dp + j];
    prow[4 + j] = sum;
  }
  if (threadIdx.x < 4) prow[threadIdx.x] = 0.f;

  auto opof = [](int) { return 0; };
  if (!arrive_pass(p.partials, st, p.grows, p.counter, s_scr, &s_flag, opof, p.single)) return;
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  float* stage = reinterpret_cast<float*>(raw + st);
  final_reduce(p.partials, st, p.grows, p.counter, s_scr, opof, raw, stage, p.single, -1, -1, st);
  if (threadIdx.x >= 32) return;
  double* B = bwd_B(p.bw);
  const double keep = (double)p.s / (double)(p.s + 1);
  for (int j = lane; j < d; j += 32) B[j] = keep * B[j] + ((double)raw[4 + j].x + (double)raw[4 + j].y);
  __syncwarp();
  if (p.s >= 1) svm_bwd_prologue(p.s - 1, p.tape, d, p.bw);
}

// svm_bwd_step_kernel for rows of 16-byte chunks (at most 32 per row), in
// the form of ses_bwd_step_t_kernel: NI points per lane per round with their
// gradient rows, the scalar work once per point after a reduce-scatter of
// the two partial dot products.
template <typename T, int VW, int LPP, int NI>
__global__ void __launch_bounds__(kBlock) svm_bwd_step_t_kernel(BwdParams p) {
  pdl_trigger();
  pdl_wait();  // the adjoint scratch and the gradient rows are the previous reverse step's output
  using GS = GroupScatter<LPP, NI>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ float2 s_scr[kMaxBlock];
  __shared__ bool s_flag;
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.state);
  if (p.s >= hdr->t) return;  // the forward stopped before step s

  const int d = p.d;
  const int dp = dpad4(d);
  const int nch = d / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  constexpr int ROUND = PPW * NI;
  const bool has_chunk = gl < nch;
  const float* ent = p.tape + (size_t)p.s * svm_tape_stride(d);
  const float k = ent[2], Hm = ent[3], s1 = ent[4], s2 = ent[5];
  const float* wbar = ent + 8;
  const float* zeta = bwd_Gbar(p.bw, d);
  const float Sbar = *bwd_Sbar(p.bw, d);
  float wb[VW], zt[VW], acc[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    wb[e] = has_chunk ? wbar[gl * VW + e] : 0.f;
    zt[e] = has_chunk ? zeta[gl * VW + e] : 0.f;
    acc[e] = 0.f;
  }
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  for (int64_t base = gw * ROUND; base < p.n; base += nwarps * ROUND) {
    float x[NI][VW], gr[NI][VW];
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int64_t i = base + r * PPW + grp;
      if (i < p.n && has_chunk) {
        Chunk<T, VW>::load(bwd_row<T>(p, i), gl, x[r]);
        const float4 g4 = *reinterpret_cast<const float4*>(p.grad + i * d + gl * VW);
        gr[r][0] = g4.x; gr[r][1] = g4.y; gr[r][2] = g4.z; gr[r][3] = g4.w;
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          x[r][e] = 0.f;
          gr[r][e] = 0.f;
        }
      }
    }
    float pw[NI], pz[NI];
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        a = fmaf(x[r][e], wb[e], a);
        b = fmaf(x[r][e], zt[e], b);
      }
      pw[r] = a;
      pz[r] = b;
    }
    GS::run(pw, gl);
    GS::run(pz, gl);
    float yown[GS::OWN], bown[GS::OWN];  // pt_i y_i and beta_i of the owned points
#pragma unroll
    for (int kk = 0; kk < GS::OWN; ++kk) {
      const int64_t i = base + GS::owned(gl, kk) * PPW + grp;
      yown[kk] = 0.f;
      bown[kk] = 0.f;
      if (i < p.n) {
        const bool pos = __ldg(p.labels + i) > 0;
        const float margin = pos ? pw[kk] - s1 : -pw[kk] - s2;
        const float pt = expf(-k * (margin - Hm));
        const float y = pos ? 1.f : -1.f;
        yown[kk] = pt * y;
        bown[kk] = -k * pt * (pz[kk] + y * Sbar);
      }
    }
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int src = grp * LPP + GS::src_lane(r);
      const float py = __shfl_sync(0xffffffffu, yown[r % GS::OWN], src);
      const float br = __shfl_sync(0xffffffffu, bown[r % GS::OWN], src);
      const int64_t i = base + r * PPW + grp;
      float dd[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        dd[e] = fmaf(py, zt[e], br * wb[e]);
        acc[e] = fmaf(br, x[r][e], acc[e]);
      }
      if (i < p.n && has_chunk) {
        float4 v;
        v.x = gr[r][0] + dd[0]; v.y = gr[r][1] + dd[1]; v.z = gr[r][2] + dd[2]; v.w = gr[r][3] + dd[3];
        *reinterpret_cast<float4*>(p.grad + i * d + gl * VW) = v;
      }
    }
  }
#pragma unroll
  for (int o = LPP; o < 32; o <<= 1)
#pragma unroll
    for (int e = 0; e < VW; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
  float* sA = reinterpret_cast<float*>(smem_raw);  // [kWarps][dp]
  if (grp == 0 && has_chunk)
#pragma unroll
    for (int e = 0; e < VW; ++e) sA[warp * dp + gl * VW + e] = acc[e];
  __syncthreads();
  const int st = ses_partial_stride(d);  // [0, 0, 0, 0, sum_i beta_i x_i]
  float* prow = p.partials + (size_t)blockIdx.x * st;
  for (int j = threadIdx.x; j < dp; j += kBlock) {
    float sum = 0.f;
    if (j < d)
      for (int w = 0; w < kWarps; ++w) sum += sA[w * dp + j];
    prow[4 + j] = sum;
  }
  if (threadIdx.x < 4) prow[threadIdx.x] = 0.f;

  auto opof = [](int) { return 0; };
  if (!arrive_pass(p.partials, st, p.grows, p.counter, s_scr, &s_flag, opof, p.single)) return;
  float2* raw = reinterpret_cast<float2*>(smem_raw);
  float* stage = reinterpret_cast<float*>(raw + st);
  final_reduce(p.partials, st, p.grows, p.counter, s_scr, opof, raw, stage, p.single, -1, -1, st);
  if (threadIdx.x >= 32) return;
  double* B = bwd_B(p.bw);
  const double keep = (double)p.s / (double)(p.s + 1);
  for (int j = lane; j < d; j += 32) B[j] = keep * B[j] + ((double)raw[4 + j].x + (double)raw[4 + j].y);
  __syncwarp();
  if (p.s >= 1) svm_bwd_prologue(p.s - 1, p.tape, d, p.bw);
}

// min over P and max over Q of x_i^T wbar^T: two candidates (value, smallest
// index) per CTA, at [2 b] (P) and [2 b + 1] (Q).
template <typename T, int VW, int LPP, int NCH, int U>
__global__ void __launch_bounds__(kBlock) svm_bwd_argmax_kernel(BwdParams p) {
  __shared__ float s_val[kWarps][2];
  __shared__ long long s_idx[kWarps][2];
  const int d = p.d;
  const int nch = (d + VW - 1) / VW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  constexpr int PPW = 32 / LPP;
  const float* mean32 = state_mean32(const_cast<void*>(p.state), d);
  float wb[NCH][VW];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int c = gl + j * LPP;
#pragma unroll
    for (int e = 0; e < VW; ++e) wb[j][e] = (c < nch) ? mean32[c * VW + e] : 0.f;
  }
  // track -x.w over P (so both are maxima) and x.w over Q
  float best[2] = {-INFINITY, -INFINITY};
  long long bidx[2] = {0x7fffffffffffffffLL, 0x7fffffffffffffffLL};
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp;
  for (int64_t base = gw * (PPW * U); base < p.n; base += nwarps * (PPW * U)) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * PPW + grp;
      float part = 0.f;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int c = gl + j * LPP;
        float x[VW];
        if (i < p.n && c < nch) {
          Chunk<T, VW>::load(bwd_row<T>(p, i), c, x);
#pragma unroll
          for (int e = 0; e < VW; ++e) part = fmaf(x[e], wb[j][e], part);
        }
      }
      const float dot = group_sum<LPP>(part);
      if (i < p.n) {
        const int cls = __ldg(p.labels + i) > 0 ? 0 : 1;
        const float v = cls == 0 ? -dot : dot;
        if (v > best[cls] || (v == best[cls] && i < bidx[cls])) {
          best[cls] = v;
          bidx[cls] = i;
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best[c], o);
      const long long oi = __shfl_xor_sync(0xffffffffu, bidx[c], o);
      if (ov > best[c] || (ov == best[c] && oi < bidx[c])) {
        best[c] = ov;
        bidx[c] = oi;
      }
    }
    if (lane == 0) {
      s_val[warp][c] = best[c];
      s_idx[warp][c] = bidx[c];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int c = threadIdx.x;
    float bv = s_val[0][c];
    long long bi = s_idx[0][c];
    for (int w = 1; w < kWarps; ++w)
      if (s_val[w][c] > bv || (s_val[w][c] == bv && s_idx[w][c] < bi)) {
        bv = s_val[w][c];
        bi = s_idx[w][c];
      }
    p.cand_val[2 * blockIdx.x + c] = bv;
    p.cand_idx[2 * blockIdx.x + c] = bi;
  }
}

// One warp: picks the rows attaining min_P and max_Q, seeds B = dL/dwbar^T and
// those rows of grad, then the bookkeeping of step T-1.
template <typename PT>  // the point type; a template, so only the launching units instantiate it
__global__ void __launch_bounds__(32) svm_bwd_seed_kernel(BwdParams p) {
  const int lane = threadIdx.x;
  const int d = p.d;
  float bv[2] = {-INFINITY, -INFINITY};
  long long bi[2] = {0x7fffffffffffffffLL, 0x7fffffffffffffffLL};
  for (int k = lane; k < p.ncand; k += 32)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float v = p.cand_val[2 * k + c];
      const long long i = p.cand_idx[2 * k + c];
      if (v > bv[c] || (v == bv[c] && i < bi[c])) {
        bv[c] = v;
        bi[c] = i;
      }
    }
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv[c], o);
      const long long oi = __shfl_xor_sync(0xffffffffu, bi[c], o);
      if (ov > bv[c] || (ov == bv[c] && oi < bi[c])) {
        bv[c] = ov;
        bi[c] = oi;
      }
    }
  const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.state);
  const int64_t T = hdr->t;
  const float* wb = state_mean32(const_cast<void*>(p.state), d);
  float n2 = 0.f;
  for (int j = lane; j < d; j += 32) n2 = fmaf(wb[j], wb[j], n2);
  n2 = warp_sum(n2);
  const bool have = n2 > 0.f && bi[0] != 0x7fffffffffffffffLL && bi[1] != 0x7fffffffffffffffLL;
  const float rn = have ? 1.0f / sqrtf(n2) : 0.f;
  const float L = have ? (-bv[0] - bv[1]) * rn : 0.f;  // (min_P x.w - max_Q x.w)/|w|
  const bool live = have && L > 0.f;                    // a clipped margin has gradient 0
  const double sd = p.seed ? *p.seed : 1.0;
  double* B = bwd_B(p.bw);
  const PT* xP = bwd_row<PT>(p, live ? bi[0] : 0);
  const PT* xQ = bwd_row<PT>(p, live ? bi[1] : 0);
  for (int j = lane; j < d; j += 32) {
    if (live) {
      const float dir = wb[j] * rn;
      B[j] = sd * (double)((elem_to_float(xP + j) - elem_to_float(xQ + j)) * rn - L * dir * rn);
      p.grad[bi[0] * d + j] += (float)(sd * dir);
      p.grad[bi[1] * d + j] -= (float)(sd * dir);
    } else {
      B[j] = 0.0;
    }
  }
  __syncwarp();
  if (lane == 0 && p.out) {
    pdscp_step_out o;
    o.oracle_value = hdr->last_value;
    o.objective = live ? (double)L : 0.0;
    o.lower_bound = o.objective;
    o.upper_bound = hdr->ub_best;
    o.t = T;
    o.failed = hdr->outcome == PDSCP_OUT_SEPARATED ? 1 : 0;
    o.stopped = hdr->stopped;
    o.status = hdr->status;
    o.outcome = hdr->outcome;
    o.k = live ? (double)bi[0] : -1.0;  // the row of P attaining the margin
    o.dual_bound = INFINITY;
    *p.out = o;
  }
  if (T >= 1) svm_bwd_prologue(T - 1, p.tape, d, p.bw);
}

}  // namespace pdscp
