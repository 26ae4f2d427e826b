// Tensor-core form of the multi-candidate SES pass (multi_kernel.cuh) for
// float32 points of d = 32 and up to 16 candidates. Per candidate j and point
// i the pass needs the squared distance |x_i - u_j|^2 and, after the
// exponentials, the weighted sum G'_j = sum_i c_ij (x_i - u_j) (Sec. 4.1,
// Eq. implement and Eq. ses_oracle). Both are dense contractions over a tile
// of 128 points, run as tcgen05 MMAs (kind::tf32) with accumulators in TMEM:
//   P = Y U~^T        (128 x 16, K = 32):  y_i = x_i - m, u~_j = u_j - m,
//                     |x_i - u_j|^2 = |y_i|^2 - 2 P_ij + |u~_j|^2
//   Q = Y^T C         (32 x 16, K = 128 points, accumulated over every tile
//                     of the CTA): sum_i c_ij y_i, and G'_j = Q_j - (sum_i c_ij) u~_j,
// with m the average of the candidates' means (FP32, the same in every CTA).
// Centring on m keeps both identities' cancellation small: u~_j is short, so
// |y_i|^2 dominates the distance, and Q_j differs from G'_j only by
// (sum_i c_ij) u~_j (centred on v_1 instead, Q_j carried the whole offset
// between the means and v_1, and its tf32-split rounding, ~2^-22 of it,
// showed in the means after a few amplifying iterations). FP32 accuracy
// from tf32 operands: each operand a is split as a = a_h + a_l with a_h its
// tf32 truncation, stored as such (exact in tf32), and a_l = a - a_h exact in
// FP32 (its own tf32 conversion costs at most 2^-22 of a), and a.b = a_h.b_h +
// a_h.b_l + a_l.b_h up to ~2^-22 relative. That is four times FP32's
// rounding, and both contractions cancel (the distance identity for points
// near a mean, G'_j against sum_i c_ij |y_i| near the equilibrium), so both
// split their operands in three exact tf32 parts (a = a_1 + a_2 + a_3, a_2
// the truncation of a - a_1, a_3 the rest, at most 2 bits) and keep the six
// products down to 2^-22 of each other: FP32-grade results.
//
// Operands. P's A operand, the three parts of Y (lane = point, one column
// per feature), sits in TMEM: the thread of point r stores its parts into
// TMEM lane r (tcgen05.st). Q's operands sit in shared memory in the
// 128-byte swizzled K-major layout, with the points as the K dimension: the
// threads write Y^T (rows 0-31, 32-63, 64-95: y_1, y_2, y_3; each K-block of
// 32 points is 96 rows) and C^T (48 rows: the three parts of the 16
// candidates), each warp writing one feature (or candidate) row for 32
// consecutive points, which falls on 32 distinct banks. Q's M dimension is
// 128: its rows 96-127 read the next K-block's first rows and are not read
// back. One MMA chain of N = 48 gives the products y_p c_q of all three parts
// of C; the six kept are summed smallest first. The points arrive from HBM
// as tiles of 128 x 32 by TMA loads (three-stage ring, 128-byte swizzle).
//
// The CTA is warp-specialised so that the work on consecutive tiles
// overlaps (one CTA per SM, tiles blockIdx.x, blockIdx.x + gridDim.x, ...;
// tile u uses buffer u & 1 of every double buffer):
//   warps 8-11, one thread per point: centring, the row norm, the three
//     parts into TMEM for P(u), then Y^T for Q into shared memory;
//   warp 12 (one elected lane issues): the TMA loads, and P(u) as soon as
//     tile u's parts are in TMEM and P(u - 2)'s accumulators have been read;
//   warp 13 (likewise): Q(u) once C^T and Y^T of tile u are written;
//   warps 0-7: thread r + 128 h reads row r of P(u) out of TMEM (candidates
//     8 h .. 8 h + 7: warp w reads TMEM lanes 32 (w % 4) ..), the
//     exponentials (straight-line code, so that the 8 candidates of a thread
//     interleave), and writes C^T once Q(u - 2) has released its buffer.
// So while the exponential warps work on tile u, the split warps prepare
// tile u + 1 and the tensor cores run Q(u - 1) and P(u + 1). Every hand-over
// is an mbarrier: the producer's writes to shared memory are fenced for the
// async proxy (its TMEM stores waited for and fenced) before it arrives, the
// MMAs' completion arrives through tcgen05.commit. Each barrier's waits are
// separated from its next completion by a chain of hand-overs through the
// waiting role itself, so a parity never aliases (the arguments are beside
// the waits).
//
// Waits are bounded (the staged passes' limit, and a CTA-wide abort flag
// ends every other role's waits early); a wait that gives up poisons the
// CTA's rows (S = NaN), so that the finishes report PDSCP_ERR_NUMERIC, and
// the MMA warps still wait (bounded) for their MMAs and loads in flight
// before the TMEM and shared memory go.
#pragma once

#include <cuda.h>

#include "multi_kernel.cuh"

namespace pdscp {

constexpr int kTcTile = 128;  // points per tile (the MMAs' M for P)
constexpr int kTcD = 32;      // features (one 128-byte swizzle row of floats)
constexpr int kTcN = 16;      // candidate columns
constexpr int kTcExpWarps = 8, kTcSplitWarps = 4;
constexpr int kTcMmaWarp = kTcExpWarps + kTcSplitWarps;  // TMA loads and P; the next warp: Q
constexpr int kTcThreads = 32 * (kTcMmaWarp + 2);
constexpr int kTcStages = 3;
// dynamic shared memory (bytes from a 1024-aligned base)
constexpr int kTcTileBytes = kTcTile * kTcD * 4;  // TMA stages first
// Q's A operand, two buffers: Y^T, 4 K-blocks of 32 points x 96 rows
constexpr int kTcA2Blk = 3 * kTcD * 128;
constexpr int kTcA2Bytes = 4 * kTcA2Blk;
constexpr int kTcA2 = kTcStages * kTcTileBytes;
// P's B operand: [u~_1; u~_2; u~_3] stacked, 48 rows x 32 features (the three
// 16-row parts are contiguous: each is two 1024-byte atoms); the last Q
// buffer's rows past its end read here
constexpr int kTcU = kTcA2 + 2 * kTcA2Bytes;
// Q's B operand, two buffers: [c_1; c_2; c_3] stacked, 48 rows x 128 points
constexpr int kTcC = kTcU + 3 * kTcN * kTcD * 4;
constexpr int kTcCBlk = 3 * kTcN * 128;
constexpr int kTcCBytes = 4 * kTcCBlk;
constexpr int kTcSmem = kTcC + 2 * kTcCBytes + 1024;  // + alignment slack
static_assert(kTcA2 % 1024 == 0 && kTcU % 1024 == 0 && kTcC % 1024 == 0 && kTcA2Blk % 1024 == 0 &&
                  kTcCBytes % 1024 == 0,
              "swizzle atoms");
static_assert(3 * kTcA2Blk + 128 * 128 <= kTcA2Bytes + 3 * kTcN * kTcD * 4, "Q's rows past the last buffer stay in U");
// TMEM columns (all 512 of the SM): tile u's parts [y_1 y_2 y_3] (P's A
// operand, lane = point) in buffer u & 1 at 96 (u & 1); P(u) in buffer u & 1
// at 192 + 96 (u & 1): six products (y_1 [u_1 u_2 u_3], y_2 [u_1 u_2], y_3 u_1:
// 16 columns each); Q at 384-431 ([c_1 c_2 c_3])
constexpr int kTcTmemCols = 512;
constexpr int kTcYCol = 0;
constexpr int kTcPCol = 192;
constexpr int kTcPCols = 96;
constexpr int kTcQCol = 384;

// byte offset of element (row, col) in a 128-byte swizzled K-major operand of
// `rows` rows (col along K, 32 floats per 128-byte atom row)
__host__ __device__ __forceinline__ int tc_sw128(int row, int col, int rows) {
  return (col >> 5) * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 + ((((col & 31) >> 2) ^ (row & 7)) << 4) +
         ((col & 3) << 2);
}

// shared-memory matrix descriptor: 128-byte swizzle, 8-row atoms 1024 bytes apart
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused by K-major swizzled layouts)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                  // descriptor version of the sm_100 family
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::tf32, FP32 accumulators, A and B K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, bool acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc ? 1u : 0u)
               : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// 8 consecutive FP32 columns of this thread's TMEM lane, without the wait
// (tcgen05.wait::ld before the registers are used)
__device__ __forceinline__ void tc_ld8_nw(uint32_t addr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
// 8 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld8(uint32_t addr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
// a's tf32 truncation (exactly representable: whatever rounding the tensor
// core applies to its FP32 operands leaves it unchanged) and the low part
// a - hi, exact in FP32
__device__ __forceinline__ float tc_hi(float a) { return __uint_as_float(__float_as_uint(a) & 0xFFFFE000u); }
__device__ __forceinline__ float tc_lo(float a) { return a - tc_hi(a); }
// 1 - e^{-x} for x >= 0: the Maclaurin series x - x^2/2! + ... - x^10/10!
// (Horner form; truncation below 2.7e-10 relative) for x < 0.5, 1 - e^{-x}
// from expf above (no cancellation there: the result is at least 0.39).
// Both are computed and one selected: no branch, so that the candidates of a
// thread interleave.
__device__ __forceinline__ float tc_one_minus_exp_neg(float x) {
  const float big = 1.f - expf(-x);
  float t = 1.f / 3628800.f;  // 1/10!
  t = fmaf(-x, t, 1.f / 362880.f);
  t = fmaf(-x, t, 1.f / 40320.f);
  t = fmaf(-x, t, 1.f / 5040.f);
  t = fmaf(-x, t, 1.f / 720.f);
  t = fmaf(-x, t, 1.f / 120.f);
  t = fmaf(-x, t, 1.f / 24.f);
  t = fmaf(-x, t, 1.f / 6.f);
  t = fmaf(-x, t, 0.5f);
  t = fmaf(-x, t, 1.f);
  return x < 0.5f ? x * t : big;
}
// a = p1 + p2 + p3, each exactly representable in tf32
__device__ __forceinline__ void tc_split3(float a, float& p1, float& p2, float& p3) {
  p1 = tc_hi(a);
  const float r = a - p1;
  p2 = tc_hi(r);
  p3 = r - p2;
}

__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap* map, int row0, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(kTcTile * kTcD * 4)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(map), "r"(0), "r"(row0), "r"(smem_u32(bar))
      : "memory");
}

// arrive (release, CTA scope) on an mbarrier
__device__ __forceinline__ void tc_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait for the completion of the phase of parity `parity`; gives up
// after `limit` tries, or earlier once another role has set the abort flag
__device__ __forceinline__ bool tc_wait(uint64_t* bar, unsigned int parity, unsigned int limit,
                                        const volatile int* abort) {
  for (unsigned int i = 0; i < limit; ++i) {
    unsigned int done;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 15u) == 15u && *abort) return false;
  }
  return false;
}

// Candidates per chunk of the staged completion: the rows of nb CTAs (st
// floats per candidate) after the finishing CTA's head (pairs of the totals,
// the K means and v_1 in FP64); 0 if not even one candidate fits.
__host__ __device__ constexpr int tc_stage_candidates(int nb, int K) {
  return (int)(((size_t)kTcSmem - 1024 - (size_t)(K * (4 + kTcD) + K * kTcD + kTcD) * 8) /
               ((size_t)nb * (4 + kTcD) * 4));
}

// Warp-wide forms: every lane of the warp executes them (uniform control
// flow, warp-uniform operands); one lane, chosen by elect.sync, issues.
__device__ __forceinline__ void tc_mma_w(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc ? 1u : 0u)
      : "memory");
}
__device__ __forceinline__ void tc_commit_w(uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_tile_w(uint32_t dst, const CUtensorMap* map, int row0, uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
      " @e cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3, {%4, %5}], [%0];\n}\n"
      ::"r"(smem_u32(bar)), "r"(kTcTile * kTcD * 4), "r"(dst), "l"(map), "r"(0), "r"(row0)
      : "memory");
}
// the same with A in TMEM (lane = row of A, one column per K element)
__device__ __forceinline__ void tc_mma_tw(uint32_t tmem, uint32_t ta, uint64_t db, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
      "r"(ta), "l"(db), "r"(idesc), "r"(acc ? 1u : 0u)
      : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane (tcgen05.wait::st
// before the data is handed on)
__device__ __forceinline__ void tc_st32(uint32_t addr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(addr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])),
      "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])),
      "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])),
      "r"(__float_as_uint(v[23])), "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])),
      "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])),
      "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
// a bounded wait by every lane of a warp, its outcome the same in all lanes
__device__ __forceinline__ bool tc_wait_w(uint64_t* bar, unsigned int parity, unsigned int limit,
                                          const volatile int* abort) {
  return __all_sync(0xffffffffu, tc_wait(bar, parity, limit, abort));
}

// One pass for K <= 16 candidates (states, alphas, step sizes as in
// ses_multi_kernel), points streamed through TMA in tiles of 128 by the
// warp-specialised pipeline above; then the completion of ses_multi_kernel
// (the last CTA reduces the K candidate rows, the warps run the finishes).
template <int K>
__global__ void __launch_bounds__(kTcThreads, 1) ses_multi_tc_kernel(MultiParams p, unsigned int wait_limit,
                                                                     const __grid_constant__ CUtensorMap tmap) {
  static_assert(K >= 1 && K <= kTcN, "up to 16 candidates");
  extern __shared__ __align__(128) unsigned char smem_raw[];  // aligned to 1024 below (the swizzle atoms)
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // mbarriers: TMA stage loaded / read by the split; per buffer (tile u in
  // buffer u & 1): Y parts and norms written, Y^T written, P done, P read,
  // C written, Q done; everything issued done
  __shared__ uint64_t s_full[kTcStages], s_sempty[kTcStages];
  __shared__ uint64_t s_yready[2], s_a2ready[2], s_pdone[2], s_pfree[2], s_cready[2], s_qdone[2], s_fin;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ float s_norm[2][kTcTile];
  __shared__ float s_v1[kTcD], s_ctr[kTcD], s_un[kTcN], s_kr[kTcN], s_H[kTcN], s_al[kTcN];
  __shared__ int s_live[kTcN];
  __shared__ float s_sc[kTcExpWarps][kTcN][4];
  __shared__ float s_q[kTcN][kTcD];
  __shared__ float2 s_scr[kTcThreads];
  __shared__ __align__(16) double s_hdr[K][sizeof(StateHdr) / 8];
  __shared__ bool s_flag;
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = kTcD, dp = kTcD;
  const int st = ses_partial_stride(d);
  const float* pts = reinterpret_cast<const float*>(p.pts);
  const int64_t ntiles = (p.n + kTcTile - 1) / kTcTile;
  // this CTA's tiles: blockIdx.x + u gridDim.x for u < nt
  const int nt = (int64_t)blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;

  // ---- set-up: candidates, v_1, the centre m, U~ in three parts, barriers, TMEM
  if (tid < kTcD) {
    s_v1[tid] = __ldg(pts + tid);
    float m = 0.f;
    for (int q = 0; q < K; ++q) m += state_mean32(p.states + (size_t)q * p.state_stride, d)[tid];
    s_ctr[tid] = m * (1.f / (float)K);
  }
  if (tid < kTcN) {
    const int q = tid;
    if (q < K) {
      const StateHdr* hdr = reinterpret_cast<const StateHdr*>(p.states + (size_t)q * p.state_stride);
      s_live[q] = hdr->stopped == 0;
      s_kr[q] = ses_kr(hdr->t, p.eta_over_rho[q]);
      s_H[q] = (float)(hdr->hint + hdr->move);
      s_al[q] = (float)p.alpha[q];
    } else {
      s_live[q] = 0;
      s_kr[q] = 0.f;
      s_H[q] = 0.f;
      s_al[q] = 0.f;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kTcN * kTcD; idx += kTcThreads) {  // u~_j = u_j - m (0 for padding columns)
    const int q = idx / kTcD, e = idx % kTcD;
    const float u = q < K ? state_mean32(p.states + (size_t)q * p.state_stride, d)[e] - s_ctr[e] : 0.f;
    float u1, u2, u3;
    tc_split3(u, u1, u2, u3);
    *reinterpret_cast<float*>(sm + kTcU + tc_sw128(q, e, 3 * kTcN)) = u1;
    *reinterpret_cast<float*>(sm + kTcU + tc_sw128(kTcN + q, e, 3 * kTcN)) = u2;
    *reinterpret_cast<float*>(sm + kTcU + tc_sw128(2 * kTcN + q, e, 3 * kTcN)) = u3;
  }
  if (tid < kTcN) {
    float s = 0.f;
    for (int e = 0; e < kTcD; ++e) {
      const float u = tid < K ? state_mean32(p.states + (size_t)tid * p.state_stride, d)[e] - s_ctr[e] : 0.f;
      s = fmaf(u, u, s);
    }
    s_un[tid] = s;
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(s_full + s, 1);
      mbar_init(s_sempty + s, 32 * kTcSplitWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(s_yready + b, 32 * kTcSplitWarps);
      mbar_init(s_a2ready + b, 32 * kTcSplitWarps);
      mbar_init(s_pdone + b, 1);
      mbar_init(s_pfree + b, 32 * kTcExpWarps);
      mbar_init(s_cready + b, 32 * kTcExpWarps);
      mbar_init(s_qdone + b, 1);
    }
    mbar_init(&s_fin, 2);
    s_abort = 0;
    mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = smem_u32(sm);

  const unsigned int wl = wait_limit;

  if (warp < kTcExpWarps) {
    // ---- exponential warps: thread (r, h) takes point r of each tile and
    // candidates 8 h .. 8 h + 7 (TMEM lane r: warp w reads lanes 32 (w % 4) ..)
    const int r = tid & (kTcTile - 1), h = tid >> 7;
    float S[8], W[8], M[8], Cs[8];  // sums over this thread's points
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      S[j] = 0.f;
      W[j] = 0.f;
      M[j] = -INFINITY;
      Cs[j] = 0.f;
    }
    const uint32_t lrow = (uint32_t)(32 * (warp & 3)) << 16;
    const int rcc = (r & 31) >> 2;
    const int cb = (r >> 5) * kTcCBlk + (h << 10) + ((r & 3) << 2);
    for (int u = 0; u < nt; ++u) {
      const int b = u & 1;
      // yready[b] completes next for tile u + 2, whose split waits for this
      // role's reads of tile u (pfree[b]); pdone[b] next for P(u + 2), which
      // waits for them too
      bool okw = tc_wait(s_yready + b, (unsigned int)(u >> 1) & 1u, wl, abort_flag);
      okw = okw && tc_wait(s_pdone + b, (unsigned int)(u >> 1) & 1u, wl, abort_flag);
      if (!__all_sync(0xffffffffu, okw)) {  // (a warp reads TMEM only if all its lanes saw the MMAs complete)
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      float P[8];
      {
        const uint32_t la = tmem + lrow + kTcPCol + kTcPCols * b + 8 * h;
        uint32_t p11[8], p12[8], p13[8], p21[8], p22[8], p31[8];
        tc_ld8_nw(la, p11);
        tc_ld8_nw(la + 16, p12);
        tc_ld8_nw(la + 32, p13);
        tc_ld8_nw(la + 48, p21);
        tc_ld8_nw(la + 64, p22);
        tc_ld8_nw(la + 80, p31);
        tc_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j)
          P[j] = (((__uint_as_float(p31[j]) + __uint_as_float(p22[j])) + __uint_as_float(p13[j])) +
                  (__uint_as_float(p21[j]) + __uint_as_float(p12[j]))) +
                 __uint_as_float(p11[j]);
      }
      // these reads of TMEM and of the norm, then the arrival that lets the
      // split of tile u + 2 and P(u + 2) overwrite them
      const float yn = s_norm[b][r];
      tc_fence_before();
      tc_arrive(s_pfree + b);
      const int64_t g = (blockIdx.x + (int64_t)u * gridDim.x) * kTcTile + r;
      const bool cone = g < p.n && g >= 1;
      const float gam = (cone && p.radii) ? __ldg(p.radii + g) : 0.f;
      float c1[8], c2[8], c3[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {  // straight-line (selects, no branches): the 8 chains interleave
        const int q = 8 * h + jj;
        const bool on = cone && s_live[q] != 0;
        const float kr = s_kr[q];
        const float d2 = fmaxf(yn - 2.f * P[jj] + s_un[q], 0.f);
        const float rd = d2 > 0.f ? rsqrtf(d2) : 0.f;
        const float dist = d2 * rd;
        const float a = s_al[q] - gam;
        const float E1 = expf(kr * ((dist + gam) - s_H[q]));
        const float em = tc_one_minus_exp_neg(2.f * kr * dist);
        const float dif = E1 * em;
        const float sum = E1 * (2.f - em);
        const float c = on ? (d2 > 0.f ? dif * rd : 2.f * kr * E1) : 0.f;
        S[jj] += on ? sum : 0.f;
        W[jj] += on ? a * sum - dist * dif : 0.f;
        M[jj] = on ? fmaxf(M[jj], dist + gam) : M[jj];
        Cs[jj] += c;
        tc_split3(c, c1[jj], c2[jj], c3[jj]);
      }
      // C buffer b is free once Q(u - 2) is done; qdone[b] completes next
      // for Q(u), which waits for this role's C of tile u
      if (u >= 2 && !__all_sync(0xffffffffu, tc_wait(s_qdone + b, (unsigned int)((u - 2) >> 1) & 1u, wl,
                                                      abort_flag))) {
        *abort_flag = 1;
        break;
      }
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {  // tc_sw128(16 part + 8 h + jj, r, 48), the row-dependent part hoisted
        const int o = kTcC + b * kTcCBytes + cb + (jj << 7) + ((rcc ^ jj) << 4);
        *reinterpret_cast<float*>(sm + o) = c1[jj];
        *reinterpret_cast<float*>(sm + o + 2048) = c2[jj];
        *reinterpret_cast<float*>(sm + o + 4096) = c3[jj];
      }
      fence_proxy_async_smem();
      tc_arrive(s_cready + b);
    }
    // the warp's sums per candidate [S, Wt, maxd, sum c]
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      float s0 = S[jj], s1 = W[jj], m = M[jj], cs = Cs[jj];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      }
      if (lane == 0) {
        s_sc[warp][8 * h + jj][0] = s0;
        s_sc[warp][8 * h + jj][1] = s1;
        s_sc[warp][8 * h + jj][2] = m;
        s_sc[warp][8 * h + jj][3] = cs;
      }
    }
  } else if (warp < kTcMmaWarp) {
    // ---- split warps: thread r takes point r of each tile (warp 8 + w the
    // points 32 w .., TMEM lanes 32 w .., one K-block of Y^T)
    const int r = tid - 32 * kTcExpWarps;
    const int rc = lane >> 2;
    const int a2b = (r >> 5) * kTcA2Blk + ((lane & 3) << 2);
    const uint32_t ty = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + kTcYCol;
    for (int u = 0, s = 0; u < nt; ++u, s = s + 1 == kTcStages ? 0 : s + 1) {
      const int b = u & 1;
      // full[s] completes next for tile u + 3, loaded after this role's
      // reads of tile u (sempty[s]); pfree[b] next once P(u) has been read,
      // which waits for this role's parts of tile u (the parts and the norm
      // of tile u - 2 in buffer b are free once P(u - 2) has been read)
      bool okw = tc_wait(s_full + s, (unsigned int)(u / kTcStages) & 1u, wl, abort_flag);
      if (u >= 2) okw = okw && tc_wait(s_pfree + b, (unsigned int)((u - 2) >> 1) & 1u, wl, abort_flag);
      if (!__all_sync(0xffffffffu, okw)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int64_t g = (blockIdx.x + (int64_t)u * gridDim.x) * kTcTile + r;
      const bool valid = g < p.n;
      const unsigned char* tptr = sm + s * kTcTileBytes;
      // y = x - m (kept for Y^T) and the row norm; the stage is then free
      float y[kTcD];
      float nrm = 0.f;
#pragma unroll
      for (int c4 = 0; c4 < kTcD / 4; ++c4) {
        const float4 x = *reinterpret_cast<const float4*>(tptr + r * 128 + ((c4 ^ (r & 7)) << 4));
        const int e0 = 4 * c4;
        y[e0] = valid ? x.x - s_ctr[e0] : 0.f;
        y[e0 + 1] = valid ? x.y - s_ctr[e0 + 1] : 0.f;
        y[e0 + 2] = valid ? x.z - s_ctr[e0 + 2] : 0.f;
        y[e0 + 3] = valid ? x.w - s_ctr[e0 + 3] : 0.f;
      }
      tc_arrive(s_sempty + s);
#pragma unroll
      for (int e = 0; e < kTcD; ++e) nrm = fmaf(y[e], y[e], nrm);
      // the three parts into TMEM lane r, buffer b: [y_1 y_2 y_3]
      {
        float v[kTcD];
#pragma unroll
        for (int e = 0; e < kTcD; ++e) v[e] = tc_hi(y[e]);
        tc_st32(ty + kTcPCols * b, v);
#pragma unroll
        for (int e = 0; e < kTcD; ++e) v[e] = tc_hi(y[e] - tc_hi(y[e]));
        tc_st32(ty + kTcPCols * b + kTcD, v);
#pragma unroll
        for (int e = 0; e < kTcD; ++e) {
          const float rr = y[e] - tc_hi(y[e]);
          v[e] = rr - tc_hi(rr);
        }
        tc_st32(ty + kTcPCols * b + 2 * kTcD, v);
      }
      s_norm[b][r] = nrm;
      tc_wait_st();
      tc_fence_before();
      tc_arrive(s_yready + b);
      // Y^T buffer b is free once Q(u - 2) is done; qdone[b] completes next
      // for Q(u), which waits for this role's Y^T of tile u
      if (u >= 2 && !__all_sync(0xffffffffu, tc_wait(s_qdone + b, (unsigned int)((u - 2) >> 1) & 1u, wl, abort_flag))) {
        *abort_flag = 1;
        break;
      }
      unsigned char* a2 = sm + kTcA2 + b * kTcA2Bytes + a2b;
#pragma unroll
      for (int e = 0; e < kTcD; ++e) {  // tc_sw128(32 part + e, r, 96) in K-block r / 32, the lane's part hoisted
        const int o = ((e >> 3) << 10) + ((e & 7) << 7) + ((rc ^ (e & 7)) << 4);
        float y1, y2, y3;  // (split again: cheaper than holding the parts)
        tc_split3(y[e], y1, y2, y3);
        *reinterpret_cast<float*>(a2 + o) = y1;
        *reinterpret_cast<float*>(a2 + o + 4 * 1024) = y2;
        *reinterpret_cast<float*>(a2 + o + 8 * 1024) = y3;
      }
      fence_proxy_async_smem();
      tc_arrive(s_a2ready + b);
    }
  } else if (warp == kTcMmaWarp) {
    // ---- the P warp (one elected lane issues): TMA loads up to three tiles
    // ahead of the split, P(u) as soon as tile u's parts are in TMEM and
    // P(u - 2) has been read
    auto load = [&](int u) {
      const int s = u % kTcStages;
      tma_load_tile_w(sbase + s * kTcTileBytes, &tmap, (int)((blockIdx.x + (int64_t)u * gridDim.x) * kTcTile),
                      s_full + s);
    };
    const uint64_t du = tc_desc(sbase + kTcU);
    int issued = 0;
    for (; issued < nt && issued < kTcStages; ++issued) load(issued);
    bool ok = true;
    for (int u = 0, s = 0; u < nt; ++u, s = s + 1 == kTcStages ? 0 : s + 1) {
      const int b = u & 1;
      if (u >= 1 && u + 2 < nt) {  // tile u + 2 into the stage of tile u - 1 (sempty: next for tile u + 2)
        const int sp = s == 0 ? kTcStages - 1 : s - 1;
        ok = tc_wait_w(s_sempty + sp, (unsigned int)((u - 1) / kTcStages) & 1u, wl, abort_flag);
        if (!ok) break;
        load(u + 2);
        ++issued;
      }
      // yready[b] completes next for tile u + 2, whose split waits for P(u)
      // to be read; pfree[b] next when P(u) has been read
      ok = tc_wait_w(s_yready + b, (unsigned int)(u >> 1) & 1u, wl, abort_flag);
      if (ok && u >= 2) ok = tc_wait_w(s_pfree + b, (unsigned int)((u - 2) >> 1) & 1u, wl, abort_flag);
      if (!ok) break;
      tc_fence_after();
      // P(u) = Y U~^T: six products of the three-part splits in three MMA
      // chains (N = 48, 32, 16 rows of the stacked U~ parts), A from TMEM
      // (8 columns per K step), B's descriptor advancing by (bytes >> 4)
      const uint32_t tp = tmem + kTcPCol + kTcPCols * b;
      const uint32_t ta = tmem + kTcYCol + kTcPCols * b;
#pragma unroll
      for (int k = 0; k < kTcD / 8; ++k) {
        const uint64_t ks = (uint64_t)(k * 32 >> 4);
        tc_mma_tw(tp, ta + 8 * k, du + ks, tc_idesc(48), k > 0);                 // y_1 [u_1 u_2 u_3]
        tc_mma_tw(tp + 48, ta + kTcD + 8 * k, du + ks, tc_idesc(32), k > 0);     // y_2 [u_1 u_2]
        tc_mma_tw(tp + 80, ta + 2 * kTcD + 8 * k, du + ks, tc_idesc(16), k > 0);  // y_3 u_1
      }
      tc_commit_w(s_pdone + b);
    }
    if (!ok) *abort_flag = 1;
    // every MMA of this warp, then every load issued, complete (bounded, at
    // least the default tries) before the TMEM and shared memory go
    const unsigned int lim = wl > kWaitLimit ? wl : kWaitLimit;
    tc_commit_w(&s_fin);
    mbar_wait(&s_fin, 0u, lim);  // (not cut short by the abort flag)
    for (int s = 0; s < kTcStages && s < issued; ++s) {
      const int last = s + kTcStages * ((issued - 1 - s) / kTcStages);
      mbar_wait(s_full + s, (unsigned int)(last / kTcStages) & 1u, lim);
    }
  } else if (warp == kTcMmaWarp + 1) {
    // ---- the Q warp (one elected lane issues): Q(u) += [Y_1^T; Y_2^T; Y_3^T]
    // [c_1 c_2 c_3] over tile u's 128 points, one chain of N = 48, once C and
    // Y^T of tile u are written
    bool ok = true;
    for (int u = 0; u < nt; ++u) {
      // cready[u & 1] and a2ready[u & 1] complete next for tile u + 2, whose
      // C and Y^T wait for Q(u)
      ok = tc_wait_w(s_cready + (u & 1), (unsigned int)(u >> 1) & 1u, wl, abort_flag) &&
           tc_wait_w(s_a2ready + (u & 1), (unsigned int)(u >> 1) & 1u, wl, abort_flag);
      if (!ok) break;
      tc_fence_after();
      const uint64_t da = tc_desc(sbase + kTcA2 + (u & 1) * kTcA2Bytes);
      const uint64_t dc = tc_desc(sbase + kTcC + (u & 1) * kTcCBytes);
#pragma unroll 4
      for (int k = 0; k < kTcTile / 8; ++k) {
        const uint64_t ka = (uint64_t)(((k >> 2) * kTcA2Blk + (k & 3) * 32) >> 4);
        const uint64_t kb = (uint64_t)(((k >> 2) * kTcCBlk + (k & 3) * 32) >> 4);
        tc_mma_w(tmem + kTcQCol, da + ka, dc + kb, tc_idesc(48), u > 0 || k > 0);
      }
      tc_commit_w(s_qdone + (u & 1));
    }
    if (!ok) *abort_flag = 1;
    const unsigned int lim = wl > kWaitLimit ? wl : kWaitLimit;
    tc_commit_w(&s_fin);
    mbar_wait(&s_fin, 0u, lim);  // (not cut short by the abort flag)
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool ok = *abort_flag == 0;
  // ---- Q out of TMEM: lanes 0-31 hold y_1^T C_b (columns kTcQCol + 16 (b - 1) ..),
  // lanes 32-63 y_2^T C_b, lanes 64-95 y_3^T C_b; the six products kept are
  // summed smallest first
  {
    const bool have = nt > 0 && ok;
    if (warp == 2) {  // y_3 c_1
      for (int c8 = 0; c8 < 2; ++c8) {
        float a[8];
        tc_ld8(tmem + (64u << 16) + kTcQCol + 8 * c8, a);
#pragma unroll
        for (int j = 0; j < 8; ++j) s_q[8 * c8 + j][lane] = have ? a[j] : 0.f;
      }
    }
    __syncthreads();
    if (warp == 1) {  // y_2 c_2, y_2 c_1
      for (int c8 = 0; c8 < 2; ++c8) {
        float a[8], b[8];
        tc_ld8(tmem + (32u << 16) + kTcQCol + 16 + 8 * c8, b);
        tc_ld8(tmem + (32u << 16) + kTcQCol + 8 * c8, a);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (have) s_q[8 * c8 + j][lane] += b[j] + a[j];
      }
    }
    __syncthreads();
    if (warp == 0) {  // y_1 c_3, y_1 c_2, y_1 c_1
      for (int c8 = 0; c8 < 2; ++c8) {
        float a[8], b[8], c[8];
        tc_ld8(tmem + kTcQCol + 32 + 8 * c8, c);
        tc_ld8(tmem + kTcQCol + 16 + 8 * c8, b);
        tc_ld8(tmem + kTcQCol + 8 * c8, a);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (have) s_q[8 * c8 + j][lane] = ((s_q[8 * c8 + j][lane] + c[j]) + b[j]) + a[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  // ---- per-CTA candidate rows [S, Wt, maxd, 0, G'_1..G'_32]
  const int wst = K * st;
  float* prow = p.partials + (size_t)blockIdx.x * wst;
  __shared__ float s_tot[kTcN][4];
  if (tid < K) {
    const int q = tid, w0 = q < 8 ? 0 : 4;  // warps 0-3 hold candidates 0-7, warps 4-7 candidates 8-15
    float s0 = 0.f, s1 = 0.f, cs = 0.f, m = -INFINITY;
    for (int w = w0; w < w0 + 4; ++w) {
      s0 += s_sc[w][q][0];
      s1 += s_sc[w][q][1];
      m = fmaxf(m, s_sc[w][q][2]);
      cs += s_sc[w][q][3];
    }
    s_tot[q][0] = ok ? s0 : NAN;  // a wait that gave up poisons the row
    s_tot[q][1] = s1;
    s_tot[q][2] = m;
    s_tot[q][3] = cs;
    prow[q * st + 0] = s_tot[q][0];
    prow[q * st + 1] = s1;
    prow[q * st + 2] = m;
    prow[q * st + 3] = 0.f;
  }
  __syncthreads();
  for (int idx = tid; idx < K * dp; idx += kTcThreads) {
    const int q = idx / dp, e = idx % dp;
    // u~_j from its exact parts in shared memory (u_1 + (u_2 + u_3) = u~_j in FP32)
    const float u = *reinterpret_cast<const float*>(sm + kTcU + tc_sw128(q, e, 3 * kTcN)) +
                    (*reinterpret_cast<const float*>(sm + kTcU + tc_sw128(kTcN + q, e, 3 * kTcN)) +
                     *reinterpret_cast<const float*>(sm + kTcU + tc_sw128(2 * kTcN + q, e, 3 * kTcN)));
    prow[q * st + 4 + e] = s_q[q][e] - s_tot[q][3] * u;  // sum_i c_ij (y_i - u~_j)
  }

  // ---- completion (as ses_multi_kernel): the last CTA reduces, warps finish candidates
  auto opof = [st](int pc) { return (pc % st) == 2 ? 1 : 0; };
  if (!arrive_pass(p.partials, wst, p.grows, p.counter, s_scr, &s_flag, opof, p.single)) return;
  float2* raw = reinterpret_cast<float2*>(sm);
  double* s_mean = reinterpret_cast<double*>(sm) + wst;
  double* s_v1d = s_mean + K * dp;
  float* stage = reinterpret_cast<float*>(s_v1d + dp);
  constexpr int HW = (int)(sizeof(StateHdr) / 8);
  for (int idx = tid; idx < K * HW; idx += kTcThreads) {
    const int q = idx / HW, w = idx % HW;
    s_hdr[q][w] = reinterpret_cast<const double*>(p.states + (size_t)q * p.state_stride)[w];
  }
  for (int idx = tid; idx < K * dp; idx += kTcThreads) {
    const int q = idx / dp, e = idx % dp;
    s_mean[idx] = state_mean(p.states + (size_t)q * p.state_stride)[e];
  }
  if (tid < d) s_v1d[tid] = (double)s_v1[tid];
  if (p.single) {
    // the CTAs' rows staged in shared memory in chunks of whole candidates
    // (every row's columns of candidates q0 ..), then reduced column by column
    const int nb = gridDim.x;
    const int cap = tc_stage_candidates(nb, K);
    for (int q0 = 0; q0 < K; q0 += cap) {
      const int w = (K - q0 < cap ? K - q0 : cap) * st, w4 = w / 4;
      for (int i = tid; i < nb * w4; i += kTcThreads) {
        const int b = i / w4, j = i - b * w4;
        const unsigned int saddr = smem_u32(stage + (size_t)b * w + 4 * j);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr),
                     "l"(p.partials + (size_t)b * wst + q0 * st + 4 * j)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
      // one thread per column: four compensated partial sums over rows
      // b = k mod 4 (independent chains), combined in a fixed order
      for (int pc = tid; pc < w; pc += kTcThreads) {
        const int op = (pc % st) == 2 ? 1 : 0;  // the maxd column of each candidate
        float2 acc[4] = {col_init2(op), col_init2(op), col_init2(op), col_init2(op)};
        int b = 0;
        for (; b + 4 <= nb; b += 4) {
#pragma unroll
          for (int k = 0; k < 4; ++k) col_comb2(op, acc[k], make_float2(stage[(size_t)(b + k) * w + pc], 0.f));
        }
        for (int k = 0; b + k < nb; ++k) col_comb2(op, acc[k], make_float2(stage[(size_t)(b + k) * w + pc], 0.f));
        col_comb2(op, acc[0], acc[1]);
        col_comb2(op, acc[2], acc[3]);
        col_comb2(op, acc[0], acc[2]);
        raw[q0 * st + pc] = acc[0];
      }
      __syncthreads();
    }
    if (tid == 0) p.counter[0] = 0u;
  } else {
    final_reduce(p.partials, wst, p.grows, p.counter, s_scr, opof, raw, stage, false, 2, -1, st);
  }
  __syncthreads();
  const double gam1 = p.radii ? (double)__ldg(p.radii) : 0.0;
  for (int q = warp; q < K; q += kTcThreads / 32) {
    const StateHdr& hq = *reinterpret_cast<const StateHdr*>(s_hdr[q]);
    if (hq.stopped) continue;  // a stopped FTP is left as is
    ses_finish_warp(raw + q * st, s_mean + q * dp, s_v1d, hq, p.states + (size_t)q * p.state_stride, d, p.alpha[q],
                    gam1, p.eta_over_rho[q], 0, p.out ? p.out + q : nullptr);
  }
}

}  // namespace pdscp
