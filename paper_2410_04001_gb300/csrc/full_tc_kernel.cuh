// Full-width LRNR residual + adjoint on the tcgen05 tensor cores (Sec. 2.1
// Eq. 2.1-2.2, Sec. 2.3), BF16, TF32 or split-BF16 operands with FP32 accumulation
// in tensor memory.  The kernel template; its BF16 / split-BF16 instantiations and
// the host-side packing are in full_tc.cu, the TF32 ones in full_tc_tf32.cu.
//
// A CTA owns a tile of 128 collocation points; point p is TMEM lane p.  For every
// hidden layer the M-wide activation is produced and consumed in chunks of NC = 32
// columns, never stored whole (a width-chunked two-GEMM fusion):
//   forward   a_c  = (s * q_c) U_chunk^T            GEMM1  (M=128, N=NC, K=r)
//             z_c  = tanh jet of a (+ bias)          epilogue, CUDA cores, FP32
//             q'_c += z_c Vn_chunk                   GEMM2  (M=128, N=r, K=NC)
//   reverse   a_c  = (s * q_c) U_chunk^T            GEMM1  (recomputed)
//             zb_c = qb'_c Vn_chunk^T                GEMM3  (M=128, N=NC, K=r)
//             ab_c = adjoint of the tanh jet         epilogue; column sums give dL/db
//             pb_c += ab_c U_chunk                   GEMM4  (M=128, N=r, K=NC)
// with one MMA per jet channel c (value, d/dt, d/dx, d2/dx2).  Split-BF16 keeps
// every operand as three BF16 pieces hi + mid + lo (exact to about 2^-27) and
// accumulates the six products whose pieces' orders add up to at most two (hi hi,
// hi mid, mid hi, hi lo, lo hi, mid mid; the three dropped ones are below 2^-24
// relative); its chunk activations, the A operands of GEMM2 and GEMM4, are written
// by the epilogue to tensor memory (tcgen05.st) and read from there by the MMAs, so
// that the three pieces of the rank-r operands fit in shared memory.  The tensor
// core rounds its FP32 accumulation toward zero, so that a long accumulation drifts;
// split-BF16 therefore accumulates GEMM2 / GEMM4 afresh in every 16-column chunk and
// adds the chunks' rank-r results into a running FP32 sum (tensor memory) on the
// CUDA cores, rounding to nearest.  TF32
// (kind::tf32) takes 32-bit operands rounded to a 10-bit mantissa: twice the shared
// memory and half the K of a BF16 MMA, so twice the MMAs per contraction.
//
// Eight warps: warps w and w+4 share TMEM lanes 32(w%4).. and split each chunk's
// epilogue columns; warps 0-3 also do the per-point work.  Lane 0 of warps 0-3
// issues the MMAs of jet channel 0-3 (and commits them), thread 0 the bulk copies.
// Where the chunk activations fit in TMEM beside the accumulators they go to GEMM2 /
// GEMM4 from there (tcgen05.st), else through shared memory.  In the multi-chunk
// kernels GEMM1 (GEMM1 + GEMM3) of chunk j+1 is issued right behind GEMM2 (GEMM4) of
// chunk j under one commit; in the TF32 and split-BF16 forward sweep it is issued
// earlier still, into D3 and D1 in turn, so that it runs during the epilogue of chunk
// j.  The bases are packed chunk by chunk in the operand layout (no-swizzle K-major
// core matrices) so that one cp.async.bulk moves a chunk; later chunks are copied
// while earlier ones are processed (two or four buffers where shared memory allows),
// and in those loops every thread waits for the next chunk's copy on its own, the CTA
// agreeing on a timeout at its next barrier.
// The rank-r layer inputs q (FP32) are kept in a per-CTA global scratch area (it stays
// in L2) for the reverse sweep.  Every mbarrier wait is bounded.
#pragma once

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lrnr_internal.cuh"
#include "point_common.cuh"
#include "simt_common.cuh"
#include "tc_ptx.cuh"

namespace lrnr {
namespace {

constexpr int TNT = 128;   // points per tile = TMEM lanes
constexpr int NTH = 256;   // threads: two per point (column halves of a chunk)
// NC: hidden-width chunk, 32 (full-width networks: one CTA and 512 TMEM columns per
// SM) or 16 (narrow networks such as the FastLRNR reduced layers: two CTAs and 256
// TMEM columns each per SM, so that one CTA's epilogue overlaps the other's MMAs; with
// rank 64 the rank-r accumulators alone take 256 columns and one CTA runs per SM).
// Split-BF16 adds its chunk activations (12 x NC/2 columns) and takes 512 columns.
template <int NC, int RM, int PREC>
constexpr int tmem_cols() { return (NC == 16 && RM <= 32 && PREC != 3) ? 256 : 512; }

// Chunk block of the packed bases (bytes), three equal groups of PIECE bytes: the
// hi pieces of Ub (NC x RM), Vb (NC x RM), Utb (RM x NC), Vtb (RM x NC) followed by
// the chunk's biases (NC floats); then the mid pieces; then the lo pieces.
// A TF32 pack (ES = 4 bytes per element) holds one piece per chunk.
template <int RM, int NC, int ES = 2>
struct Pk {
  static constexpr int T = NC * RM * ES;
  static constexpr int PIECE = 4 * T + 4 * NC;      // offset from a hi tile to its mid tile
  static constexpr int HI = PIECE;                  // bytes needed by BF16 and TF32
  static constexpr int ALL = 3 * PIECE;             // bytes needed by split-BF16
  static constexpr int CHUNK = ES == 4 ? PIECE : ALL;
};

// Operand precision of the kernel: 1 = BF16, 2 = TF32, 3 = split-BF16.
template <int PREC>
constexpr int elem_bytes() { return PREC == 2 ? 4 : 2; }

template <int RM, int PREC, int NC>
struct TcLayout {
  static constexpr int HC = NC / 2;                 // columns per epilogue thread
  static constexpr int ES = elem_bytes<PREC>();     // bytes per operand element
  static constexpr int KPM = 32 / ES;               // K elements per MMA (32 bytes of a row)
  static constexpr int PARTS = PREC == 3 ? 3 : 1;   // pieces of each operand
  static constexpr int A1B = TNT * RM * ES;         // one (channel, piece) rank-r operand
  static constexpr int A24B = TNT * NC * ES;        // one (channel, piece) width operand
  static constexpr bool SPLIT = PREC == 3;
  // tensor-memory columns of one channel's chunk activation: three BF16 pieces of NC/2
  // columns (two BF16 per column), one such piece, or NC TF32 columns
  static constexpr int ACOLS = SPLIT ? 3 * (NC / 2) : (PREC == 2 ? NC : NC / 2);
  static constexpr int TM_A24 = 8 * NC + 4 * RM;
  // chunk activations (the A operand of GEMM2 / GEMM4) in tensor memory wherever they
  // fit beside the accumulators (always for split-BF16, whose pieces would not fit in
  // shared memory): the epilogue's hand-over through tcgen05.st costs less than stores
  // to shared memory and the proxy fence they need
  static constexpr bool A24_TMEM = SPLIT || TM_A24 + 4 * ACOLS <= tmem_cols<NC, RM, PREC>();
  static constexpr int BBYTES = PREC == 3 ? Pk<RM, NC>::ALL : Pk<RM, NC, ES>::HI;
  static constexpr int OFF_A1 = 0;
  static constexpr int OFF_A3 = OFF_A1 + 4 * PARTS * A1B;
  static constexpr int OFF_A24 = OFF_A3 + 4 * PARTS * A1B;
  static constexpr int OFF_B = OFF_A24 + (A24_TMEM ? 0 : 4 * A24B);
  // tensor-memory columns: D1 [4][NC], D3 [4][NC], D24 [4][RM], then the chunk
  // activations [4 channels][ACOLS] and (split-BF16) the running sum R24 [4][RM] of the
  // chunks' rank-r results
  static constexpr int TM_R24 = TM_A24 + 4 * ACOLS;
  static constexpr int TM_END = SPLIT ? TM_R24 + 4 * RM : (A24_TMEM ? TM_R24 : TM_A24);
  static constexpr int BSTRIDE = (BBYTES + 127) & ~127;
  // B buffers: four for the pipelined forward sweep where they fit (TF32 32-column and
  // split-BF16 kernels: chosen by measurement, the BF16 kernel ran 2 % slower with it),
  // else two, else one
  static constexpr bool NB4 = ((NC == 32 && PREC == 2) || SPLIT) &&
                              OFF_B + 4 * BSTRIDE + 16 * 1024 <= 227 * 1024;
  static constexpr int NB = NB4 ? 4 : (OFF_B + 2 * BSTRIDE + 16 * 1024 <= 227 * 1024 ? 2 : 1);
  static constexpr int OFF_F = OFF_B + NB * BSTRIDE;
  // MMA issue order: GEMM1 of the next chunk right behind GEMM2 of this one (needs two B
  // buffers); chosen for the 32-column full-width kernels and split-BF16, whose layers
  // have several chunks, and not for the reduced network's 16-column chunks (one chunk
  // per layer at rhat = 16, where it measured slower)
  static constexpr bool B2B = NB >= 2 && (NC == 32 || SPLIT);
  // forward sweep pipelined: GEMM1 of chunk j + 1 (into D3 and D1 in turn; D3 is free in
  // the forward sweep) runs during the epilogue of chunk j
  static constexpr bool PIPE = NB == 4;
  // float area: s [(L+1)*RM], red [4][PL] (loss, dL/ds, output-bias dL/db), dbw [8][HC];
  // then the mbarriers and the TMEM base address
  static __host__ __device__ int floats(int L) { return (L + 1) * RM + 4 * (2 + (L + 1) * RM) + 8 * HC; }
  static __host__ __device__ int bytes(int L) { return OFF_F + floats(L) * 4 + 128; }
};

// All threads wait for `bar` to complete the phase with parity `ph`; false (and the
// device status set) if the wait timed out.  The expected parity advances only on
// success, so that after a timeout the drain at the end of the kernel waits for the
// very phase (the MMA or copy still in flight) that timed out.
// A thread whose own earlier wait failed (ok_before false) does not wait and votes for
// the failure.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t &ph, bool &pend, const KParams &p,
                                         bool ok_before = true) {
  const bool ok = ok_before && tc::mbar_wait(bar, ph, p.max_wait);
  const bool all = __syncthreads_and(ok);
  if (all) {
    ph ^= 1u;
    pend = false;
  }
  if (!all && threadIdx.x == 0) set_status(p.status, DEV_TIMEOUT);
  tc::fence_after_sync();
  return all;
}

// One thread's own bounded wait, without a CTA barrier, for a completion that only
// this thread's next steps depend on; the CTA agrees on a failure at its next barrier
// (the caller passes the result there).
__device__ __forceinline__ bool wait_own(uint64_t *bar, uint32_t &ph, bool &pend, const KParams &p) {
  const bool ok = tc::mbar_wait(bar, ph, p.max_wait);
  if (ok) {
    ph ^= 1u;
    pend = false;
  } else {
    set_status(p.status, DEV_TIMEOUT);
  }
  tc::fence_after_sync();
  return ok;
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}

// Store 8 consecutive K entries (k0 a multiple of 8) of one row of a K-major operand
// with K columns: BF16, the three BF16 pieces of split-BF16 (piece i at base + i *
// pstride), or TF32 (round to nearest).
template <int PREC>
__device__ __forceinline__ void put8(unsigned char *base, uint32_t pstride, int row, int k0, int K,
                                     const float (&w)[8]) {
  if constexpr (PREC == 2) {
    *reinterpret_cast<uint4 *>(base + tc::kmajor_off_e(row, k0, K, 4)) =
        tc::pack4_tf32(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(base + tc::kmajor_off_e(row, k0 + 4, K, 4)) =
        tc::pack4_tf32(w[4], w[5], w[6], w[7]);
  } else if constexpr (PREC == 3) {
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tc::split3_bf16x2(w[2 * i], w[2 * i + 1], h[i], m[i], l[i]);
    const uint32_t off = tc::kmajor_off(row, k0, K);
    *reinterpret_cast<uint4 *>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(base + pstride + off) = make_uint4(m[0], m[1], m[2], m[3]);
    *reinterpret_cast<uint4 *>(base + 2 * pstride + off) = make_uint4(l[0], l[1], l[2], l[3]);
  } else {
    uint4 hi, lo;
    tc::pack8_bf16(w, hi, lo);
    *reinterpret_cast<uint4 *>(base + tc::kmajor_off(row, k0, K)) = hi;
  }
}

// Write a rank-r row (this thread's point) of channel c into a K-major operand.
template <int RM, int PREC, int NC>
__device__ __forceinline__ void put_rank_row(unsigned char *base, int c, const float *v, int row) {
  using Lay = TcLayout<RM, PREC, NC>;
#pragma unroll
  for (int k0 = 0; k0 < RM; k0 += 8) {
    float w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = v[k0 + i];
    put8<PREC>(base + (Lay::PARTS * c) * Lay::A1B, Lay::A1B, row, k0, RM, w);
  }
}

// Pieces (i of A, j of B) of the split-BF16 products, largest first: every pair
// with i + j <= 2.
constexpr int kSplitProducts = 6;
__device__ __forceinline__ constexpr int split_ai(int t) { return t == 2 ? 1 : (t == 4 ? 2 : (t == 5 ? 1 : 0)); }
__device__ __forceinline__ constexpr int split_bj(int t) { return t == 1 ? 1 : (t == 3 ? 2 : (t == 5 ? 1 : 0)); }

// D (+)= A B^T with A in shared memory (piece i of A at aBase + i * aStride bytes,
// piece j of B at b + j * PIECE bytes).  BF16: one product.  Split-BF16: the six
// products hi hi, hi mid, mid hi, hi lo, lo hi, mid mid.  TF32: one product of TF32
// operands.
template <int RM, int PREC, int NC>
__device__ __forceinline__ void mma_split(uint32_t d, uint32_t aBase, uint32_t aStride, uint32_t b,
                                          uint32_t sboA, uint32_t sboB, uint32_t idesc,
                                          uint32_t acc) {
  if constexpr (PREC == 2) {
    tc::mma_tf32(d, tc::sdesc(aBase, 128, sboA), tc::sdesc(b, 128, sboB), idesc, acc);
  } else if constexpr (PREC == 3) {
    constexpr uint32_t PC = Pk<RM, NC>::PIECE;
#pragma unroll
    for (int t = 0; t < kSplitProducts; ++t)
      tc::mma_bf16(d, tc::sdesc(aBase + split_ai(t) * aStride, 128, sboA),
                   tc::sdesc(b + split_bj(t) * PC, 128, sboB), idesc, t == 0 ? acc : 1u);
  } else {
    tc::mma_bf16(d, tc::sdesc(aBase, 128, sboA), tc::sdesc(b, 128, sboB), idesc, acc);
  }
}

// Split-BF16 with A in tensor memory (piece i at column aT + i * aCols): the six
// products of mma_split.
template <int RM, int NC>
__device__ __forceinline__ void mma_split_t(uint32_t d, uint32_t aT, uint32_t aCols, uint32_t b,
                                            uint32_t sboB, uint32_t idesc, uint32_t acc) {
  constexpr uint32_t PC = Pk<RM, NC>::PIECE;
#pragma unroll
  for (int t = 0; t < kSplitProducts; ++t)
    tc::mma_bf16_ts(d, aT + split_ai(t) * aCols, tc::sdesc(b + split_bj(t) * PC, 128, sboB), idesc,
                    t == 0 ? acc : 1u);
}

// Write n consecutive chunk-activation values of channel c (this thread's row, K
// positions k0..k0+n-1 of the chunk, k0 even) to the tensor-memory A operand of GEMM2 /
// GEMM4.  Split-BF16 (PREC 3): the three BF16 pieces, two per column, piece i at
// NC/2 * i columns further; BF16 (PREC 1): one piece, rounded to nearest even like
// the shared-memory operand; TF32 (PREC 2): one element per column, rounded to nearest
// (ties away) like the shared-memory operand.  n = 16 or 8.
template <int NC, int n, int PREC>
__device__ __forceinline__ void put_act_tmem(uint32_t ta_row, int c, int k0, const float *v) {
  constexpr int HALF = NC / 2;           // columns per (channel, piece)
  if constexpr (PREC == 2) {
    const uint32_t col = ta_row + (uint32_t)(c * NC + k0);
#pragma unroll
    for (int g = 0; g < n; g += 8) {
      uint32_t w[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w[i]) : "f"(v[g + i]));
      tc::tmem_st8(col + g, w);
    }
    return;
  }
  constexpr int PIECES = PREC == 3 ? 3 : 1;
  const uint32_t col = ta_row + (uint32_t)(PIECES * c * HALF + k0 / 2);
  if constexpr (PIECES == 3) {
    uint32_t h[n / 2], m[n / 2], l[n / 2];
#pragma unroll
    for (int i = 0; i < n / 2; ++i) tc::split3_bf16x2(v[2 * i], v[2 * i + 1], h[i], m[i], l[i]);
    if constexpr (n == 16) {
      tc::tmem_st8(col, h);
      tc::tmem_st8(col + HALF, m);
      tc::tmem_st8(col + 2 * HALF, l);
    } else {
      static_assert(n == 8, "activation group");
      tc::tmem_st4(col, h);
      tc::tmem_st4(col + HALF, m);
      tc::tmem_st4(col + 2 * HALF, l);
    }
  } else {
    uint32_t h[n / 2];
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      h[i] = *reinterpret_cast<const uint32_t *>(&b);
    }
    if constexpr (n == 16) tc::tmem_st8(col, h);
    else tc::tmem_st4(col, h);
  }
}

// tanh and its first two derivatives, z, d1 = 1 - z^2, d2 = -2 z d1, at two adjacent
// columns, the arithmetic around the tanh on the packed two-lane FP32 pipe (each lane
// rounds like the scalar instruction)
template <int PREC>
__device__ __forceinline__ void act_jet2(float2 a0, float2 &z, float2 &d1, float2 &d2) {
  if constexpr (PREC == 1) {
    // BF16 operands: the MUFU tanh (about 2^-11 relative) is below their rounding
    z = make_float2(tc::tanh_approx(a0.x), tc::tanh_approx(a0.y));
    d1 = __ffma2_rn(make_float2(-z.x, -z.y), z, make_float2(1.0f, 1.0f));
    d2 = __fmul2_rn(__fmul2_rn(z, make_float2(-2.0f, -2.0f)), d1);
  } else {
    // the FP32 kernels' tanh jet (errors of a few 1e-7)
    tanh_d(a0.x, z.x, d1.x, d2.x);
    tanh_d(a0.y, z.y, d1.y, d2.y);
  }
}

// Forward tanh jets of a thread's HC columns in place, two columns per step on the
// packed FP32 pipe: pre-activations a[c] (c = value, t, x, xx; the value channel
// without its bias) become z, z_t = s' a_t, z_x = s' a_x, z_xx = s'' a_x^2 + s' a_xx
template <int C, int HC, int PREC>
__device__ __forceinline__ void fwd_jets(float (&a)[C][HC], const float *__restrict__ bias) {
#pragma unroll
  for (int i = 0; i < HC; i += 2) {
    const float2 bb = *reinterpret_cast<const float2 *>(bias + i);
    float2 z, d1, d2;
    act_jet2<PREC>(__fadd2_rn(make_float2(a[0][i], a[0][i + 1]), bb), z, d1, d2);
    if constexpr (C == 4) {
      const float2 ax = make_float2(a[2][i], a[2][i + 1]);
      const float2 zxx = __ffma2_rn(__fmul2_rn(d2, ax), ax,
                                    __fmul2_rn(d1, make_float2(a[3][i], a[3][i + 1])));
      const float2 zt = __fmul2_rn(make_float2(a[1][i], a[1][i + 1]), d1);
      const float2 zx = __fmul2_rn(ax, d1);
      a[1][i] = zt.x;
      a[1][i + 1] = zt.y;
      a[2][i] = zx.x;
      a[2][i + 1] = zx.y;
      a[3][i] = zxx.x;
      a[3][i + 1] = zxx.y;
    }
    a[0][i] = z.x;
    a[0][i + 1] = z.y;
  }
}

struct Ctl {
  uint64_t *b1, *b2, *bb;   // GEMM barriers, B-buffer barriers [NB]
  uint32_t ph1, ph2, phb[4];
  int chunk_ctr;            // chunks consumed so far (selects the B buffer)
  // an MMA commit or a copy is outstanding on the barrier (uniform over the CTA): the
  // drain after a timeout waits for exactly these
  bool p1, p2, pb[4];
};

template <int RM, int PREC, int C, int NC>
__device__ void tc_tile(const KParams &p, const Tile &T, int tile, unsigned char *sm,
                        const unsigned char *__restrict__ pack, float *__restrict__ qst,
                        uint32_t tb, Ctl &ctl, bool &dead) {
  using Lay = TcLayout<RM, PREC, NC>;
  using PK = Pk<RM, NC, Lay::ES>;
  constexpr int KPM = Lay::KPM;
  constexpr int HC = NC / 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (TNT - 1);       // point / TMEM lane
  const int half = tid >> 7;             // column half of the epilogue
  const bool lead = tid < TNT;           // threads doing the per-point work
  // MMA issuers: lane 0 of warps 0-3, one per jet channel; each issues its channel's
  // MMAs (so that every accumulator's MMAs come from one thread, in order) and commits
  // them, so that the issue is spread over four warps; the MMA barriers count four
  // commits, and an issuer without a channel (tiles of one channel) commits nothing
  // pending, which arrives at once
  const bool issuer = (tid & 31) == 0 && warp < 4;
  const int ic = warp;                   // the issuer's channel
  const int L = p.L, M = p.M;
  const int NCH = (M + NC - 1) / NC;
  unsigned char *sA1 = sm + Lay::OFF_A1;
  unsigned char *sA3 = sm + Lay::OFF_A3;
  unsigned char *sA24 = sm + Lay::OFF_A24;
  unsigned char *sB0 = sm + Lay::OFF_B;
  float *fa = reinterpret_cast<float *>(sm + Lay::OFF_F);
  const float *s_s = fa;
  const int PL = 2 + (L + 1) * RM;
  float *red_w = fa + (L + 1) * RM + (warp & 3) * PL;
  float *dbw = fa + (L + 1) * RM + 4 * PL;
  const float *tail = reinterpret_cast<const float *>(pack + (size_t)L * NCH * PK::CHUNK);
  const float Uout = tail[2 * R1], bout = tail[2 * R1 + 1];
  const uint32_t sA1u = tc::smem_u32(sA1), sA3u = tc::smem_u32(sA3), sA24u = tc::smem_u32(sA24);
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t D1 = tb, D3 = tb + 4 * NC, D24 = tb + 8 * NC;
  const uint32_t TA = tb + Lay::TM_A24;   // chunk activations in TMEM (A of GEMM2 / GEMM4)
  const uint32_t R24 = tb + Lay::TM_R24;  // split-BF16 running sum of the chunks' GEMM2 / GEMM4
  constexpr uint32_t ID_W = PREC == 2 ? tc::idesc_tf32(128, NC) : tc::idesc_bf16(128, NC);
  constexpr uint32_t ID_R = PREC == 2 ? tc::idesc_tf32(128, RM) : tc::idesc_bf16(128, RM);
  // byte stride between 8-row core-matrix groups: K elements of ES bytes, 8 rows
  constexpr uint32_t SBO_R = RM * Lay::ES * 8, SBO_W = NC * Lay::ES * 8;

  const PointIn pt = load_point(p, T, row);
  // Rank-r jets are handled one channel at a time (RM floats live at a time): the
  // input jet of layer 0, the rank-r accumulator in TMEM, the layer-input store.
  auto input_jet_c = [&](int c, float (&v)[RM]) {
#pragma unroll
    for (int k = 0; k < RM; ++k) v[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      if (c == 0) v[k] = tail[k] * pt.x + tail[R1 + k] * pt.t;
      else if (c == 1) v[k] = tail[R1 + k];
      else if (c == 2) v[k] = tail[k];
    }
  };
  auto rank_c = [&](int c, float (&v)[RM]) {
#pragma unroll
    for (int k0 = 0; k0 < RM; k0 += 16) {
      float w[16];
      tc::tmem_ld16(D24 + lane_base + c * RM + k0, w);
      if (Lay::SPLIT && NCH > 1) {
        float r[16];
        tc::tmem_ld16(R24 + lane_base + c * RM + k0, r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] += r[i];
      }
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[k0 + i] = w[i];
    }
  };
  // split-BF16: add the rank-r result of the chunk just finished (D24, accumulated
  // afresh by each chunk) into R24, rounding to nearest; the first chunk of a layer
  // initialises R24.  Thread (row, half) takes half of each channel's RM columns.
  auto fold_chunk = [&](bool first) {
    constexpr int HR = RM / 2;
    // each group of 8 columns: every channel's loads behind one wait, the additions on
    // the packed FP32 pipe
#pragma unroll
    for (int i0 = 0; i0 < HR; i0 += 8) {
      float d[C][8], r[C][8];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const uint32_t col = lane_base + c * RM + half * HR + i0;
        tc::tmem_ld8(D24 + col, d[c]);
        if (!first) tc::tmem_ld8(R24 + col, r[c]);
      }
      tc::tmem_ld_wait();
#pragma unroll
      for (int c = 0; c < C; ++c) {
        uint32_t w8[8];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          const float2 v = first ? make_float2(d[c][i], d[c][i + 1])
                                 : __fadd2_rn(make_float2(d[c][i], d[c][i + 1]),
                                              make_float2(r[c][i], r[c][i + 1]));
          w8[i] = __float_as_uint(v.x);
          w8[i + 1] = __float_as_uint(v.y);
        }
        tc::tmem_st8(R24 + lane_base + c * RM + half * HR + i0, w8);
      }
    }
    tc::tmem_st_wait();
  };
  auto stored_c = [&](int l, int c, float (&v)[RM]) {   // input jet of layer l >= 1
#pragma unroll
    for (int k = 0; k < RM; ++k) v[k] = qst[(((l - 1) * 4 + c) * RM + k) * TNT + row];
  };
  auto put_scaled = [&](unsigned char *base, int c, const float (&v)[RM], int l) {
    float y[RM];
#pragma unroll
    for (int k = 0; k < RM; ++k) y[k] = v[k] * s_s[l * RM + k];
    put_rank_row<RM, PREC, NC>(base, c, y, row);
  };
  auto bbuf = [&](int n) { return sB0 + (n % Lay::NB) * Lay::BSTRIDE; };
  // Stream the chunks of a layer through the B buffers: before chunk j, chunk j+1
  // (or, with one buffer, chunk j itself) is requested.
  auto fetch = [&](const unsigned char *lp, int j, int n) {
    if (tid == 0)
      bulk_copy(bbuf(n), lp + (size_t)j * PK::CHUNK, Lay::BBYTES, &ctl.bb[n % Lay::NB]);
    ctl.pb[n % Lay::NB] = true;
  };
  auto wait_b = [&](int n) {
    return wait_bar(&ctl.bb[n % Lay::NB], ctl.phb[n % Lay::NB], ctl.pb[n % Lay::NB], p);
  };
  auto wait_b_own = [&](int n) {
    return wait_own(&ctl.bb[n % Lay::NB], ctl.phb[n % Lay::NB], ctl.pb[n % Lay::NB], p);
  };

  // MMA issue (thread 0) for the chunk whose bases are in B buffer n
  // forward GEMM1: a_c = (s q_c) U_chunk^T into the accumulator at column D
  auto issue_g1d = [&](int n, uint32_t D) {
    const uint32_t sB = tc::smem_u32(bbuf(n));
    const int c = ic;
    if (c < C)
#pragma unroll
      for (int kk = 0; kk < RM / KPM; ++kk)
        mma_split<RM, PREC, NC>(D + c * NC, sA1u + (Lay::PARTS * c) * Lay::A1B + kk * 256,
                                Lay::A1B, sB + kk * 256, SBO_R, SBO_R, ID_W, kk > 0);
  };
  auto issue_g1 = [&](int n) { issue_g1d(n, D1); };
  // GEMM2 (forward, rank-r tile at 3T) or GEMM4 (reverse, at 2T) of chunk j of the
  // layer: the chunk activations times the tile, into D24 (split-BF16 afresh per chunk)
  auto issue_g24 = [&](int n, int j, int toff) {
    const uint32_t sB = tc::smem_u32(bbuf(n)) + (uint32_t)toff;
    const int c = ic;
    if (c < C)
#pragma unroll
      for (int kk = 0; kk < NC / KPM; ++kk) {
        if constexpr (Lay::SPLIT)
          mma_split_t<RM, NC>(D24 + c * RM, TA + 3 * c * (NC / 2) + kk * 8, NC / 2,
                              sB + kk * 256, SBO_W, ID_R, kk > 0);
        else if constexpr (Lay::A24_TMEM && PREC == 2)
          tc::mma_tf32_ts(D24 + c * RM, TA + c * Lay::ACOLS + kk * 8,
                          tc::sdesc(sB + kk * 256, 128, SBO_W), ID_R, (j > 0 || kk > 0) ? 1u : 0u);
        else if constexpr (Lay::A24_TMEM)
          tc::mma_bf16_ts(D24 + c * RM, TA + c * Lay::ACOLS + kk * 8,
                          tc::sdesc(sB + kk * 256, 128, SBO_W), ID_R, (j > 0 || kk > 0) ? 1u : 0u);
        else
          mma_split<RM, PREC, NC>(D24 + c * RM, sA24u + c * Lay::A24B + kk * 256, Lay::A24B,
                                  sB + kk * 256, SBO_W, SBO_W, ID_R, (j > 0 || kk > 0));
      }
  };
  auto fwd_epilogue = [&](int n) {
    const float *bias_s = reinterpret_cast<const float *>(bbuf(n) + 4 * PK::T);
    {
      const int c0 = half * HC;
      float a[C][HC];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if constexpr (HC == 16) tc::tmem_ld16(D1 + lane_base + c * NC + c0, a[c]);
        else tc::tmem_ld8(D1 + lane_base + c * NC + c0, a[c]);
      }
      tc::tmem_ld_wait();
      fwd_jets<C, HC, PREC>(a, bias_s + c0);
      if constexpr (Lay::A24_TMEM) {
#pragma unroll
        for (int c = 0; c < C; ++c) put_act_tmem<NC, HC, PREC>(TA + lane_base, c, c0, a[c]);
        tc::tmem_st_wait();
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int h = 0; h < HC / 8; ++h) {
            float w8[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w8[i] = a[c][h * 8 + i];
            put8<PREC>(sA24 + c * Lay::A24B, Lay::A24B, row, c0 + h * 8, NC, w8);
          }
      }
    }
  };

  auto issue_g13 = [&](int n) {   // reverse GEMM1 into D1 and GEMM3 into D3
    const uint32_t sB = tc::smem_u32(bbuf(n));
    const int c = ic;
    if (c < C)
#pragma unroll
      for (int kk = 0; kk < RM / KPM; ++kk) {
        mma_split<RM, PREC, NC>(D1 + c * NC, sA1u + (Lay::PARTS * c) * Lay::A1B + kk * 256,
                                Lay::A1B, sB + kk * 256, SBO_R, SBO_R, ID_W, kk > 0);
        mma_split<RM, PREC, NC>(D3 + c * NC, sA3u + (Lay::PARTS * c) * Lay::A1B + kk * 256,
                                Lay::A1B, sB + PK::T + kk * 256, SBO_R, SBO_R, ID_W, kk > 0);
      }
  };
  auto rev_epilogue = [&](int n) {
    const float *bias_s = reinterpret_cast<const float *>(bbuf(n) + 4 * PK::T);
#pragma unroll
    for (int h8 = 0; h8 < HC / 8; ++h8) {
      const int c0 = half * HC + h8 * 8;
      float a[C][8], wb[C][8];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        tc::tmem_ld8(D1 + lane_base + c * NC + c0, a[c]);
        tc::tmem_ld8(D3 + lane_base + c * NC + c0, wb[c]);
      }
      tc::tmem_ld_wait();
      // two columns per step on the packed FP32 pipe
#pragma unroll
      for (int i = 0; i < 8; i += 2) {
        const float2 bb = *reinterpret_cast<const float2 *>(bias_s + c0 + i);
        float2 z, d1, d2;
        act_jet2<PREC>(__fadd2_rn(make_float2(a[0][i], a[0][i + 1]), bb), z, d1, d2);
        float2 ab0 = __fmul2_rn(make_float2(wb[0][i], wb[0][i + 1]), d1);
        if constexpr (C == 4) {
          const float2 at = make_float2(a[1][i], a[1][i + 1]);
          const float2 ax = make_float2(a[2][i], a[2][i + 1]);
          const float2 axx = make_float2(a[3][i], a[3][i + 1]);
          const float2 w1 = make_float2(wb[1][i], wb[1][i + 1]);
          const float2 w2 = make_float2(wb[2][i], wb[2][i + 1]);
          const float2 w3 = make_float2(wb[3][i], wb[3][i + 1]);
          // third derivative of tanh: d1 (6 z^2 - 2)
          const float2 d3 = __fmul2_rn(d1, __ffma2_rn(__fmul2_rn(z, z), make_float2(6.0f, 6.0f),
                                                      make_float2(-2.0f, -2.0f)));
          ab0 = __ffma2_rn(d2, __ffma2_rn(w2, ax, __fmul2_rn(w1, at)), ab0);
          ab0 = __ffma2_rn(w3, __ffma2_rn(__fmul2_rn(d3, ax), ax, __fmul2_rn(d2, axx)), ab0);
          const float2 n2 = __ffma2_rn(__fmul2_rn(__fmul2_rn(w3, make_float2(2.0f, 2.0f)), d2), ax,
                                       __fmul2_rn(w2, d1));
          const float2 n3 = __fmul2_rn(w3, d1);
          const float2 n1 = __fmul2_rn(w1, d1);
          wb[1][i] = n1.x;
          wb[1][i + 1] = n1.y;
          wb[2][i] = n2.x;
          wb[2][i + 1] = n2.y;
          wb[3][i] = n3.x;
          wb[3][i + 1] = n3.y;
        }
        wb[0][i] = ab0.x;
        wb[0][i + 1] = ab0.y;
      }
      if constexpr (Lay::A24_TMEM) {
#pragma unroll
        for (int c = 0; c < C; ++c) put_act_tmem<NC, 8, PREC>(TA + lane_base, c, c0, wb[c]);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) put8<PREC>(sA24 + c * Lay::A24B, Lay::A24B, row, c0, NC, wb[c]);
      }
      float g8[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) g8[i] = wb[0][i];
      const float r = warp_reduce_scatter<8>(g8);
      if ((lane & 3) == 0) dbw[warp * HC + h8 * 8 + (lane >> 2)] = r;
    }
    if constexpr (Lay::A24_TMEM) tc::tmem_st_wait();
  };

  // ---------------- forward (the operand A1 of layer l >= 1 is written at the end
  // of layer l - 1, from its rank-r result)
  if (lead) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float v[RM];
      input_jet_c(c, v);
      put_scaled(sA1, c, v, 0);
    }
  }
  float qL[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // the last layer's rank-1 result, per channel
  for (int l = 0; l < L && !dead; ++l) {
    const unsigned char *lp = pack + (size_t)l * NCH * PK::CHUNK;
    const int n0 = ctl.chunk_ctr;
    if constexpr (Lay::PIPE) {
      // GEMM1 of chunk j + 1 is issued, into the other of D1 / D3, as soon as GEMM1 of
      // chunk j is done, so that it runs during the epilogue of chunk j; GEMM2 of chunk
      // j - 1 runs then too, and the epilogue waits for it only before it overwrites the
      // chunk activations.  B(j + 2) goes into the buffer of chunk j - 2, whose MMAs the
      // wait for GEMM1(j) covers (each issuer's commit covers its earlier MMAs)
      auto dacc = [&](int j) { return (j & 1) ? D3 : D1; };
      fetch(lp, 0, n0);
      if (NCH > 1) fetch(lp, 1, n0 + 1);
      if (!wait_b(n0)) { dead = true; return; }
      tc::fence_async_smem();
      __syncthreads();
      if (issuer) {
        tc::fence_after_sync();
        issue_g1d(n0, D1);
        tc::mma_commit(ctl.b1);
      }
      ctl.p1 = true;
      for (int j = 0; j < NCH; ++j) {
        const int n = n0 + j;
        if (!wait_bar(ctl.b1, ctl.ph1, ctl.p1, p)) { dead = true; return; }   // GEMM1(j) done
        if (j + 2 < NCH) fetch(lp, j + 2, n + 2);
        bool b_ok = true;
        if (j + 1 < NCH) {
          // every thread waits for B(j + 1) on its own (the issuers before GEMM1(j + 1),
          // the others before the next epilogue reads the biases); the CTA agrees on a
          // timeout at the barrier below
          b_ok = wait_b_own(n + 1);
          if (b_ok) {
            if (issuer) {
              issue_g1d(n + 1, dacc(j + 1));
              tc::mma_commit(ctl.b1);
            }
            ctl.p1 = true;
          }
          __syncwarp();   // the warp reconverges before the tensor-memory loads below
        }
        const float *bias_s = reinterpret_cast<const float *>(bbuf(n) + 4 * PK::T);
        const uint32_t Dj = dacc(j);
        const int c0 = half * HC;
        float a[C][HC];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          if constexpr (HC == 16) tc::tmem_ld16(Dj + lane_base + c * NC + c0, a[c]);
          else tc::tmem_ld8(Dj + lane_base + c * NC + c0, a[c]);
        }
        tc::tmem_ld_wait();
        fwd_jets<C, HC, PREC>(a, bias_s + c0);
        bool own_ok = true;
        if (j > 0) {
          // GEMM2(j - 1) has read the activations (split-BF16: its result is folded);
          // each thread waits for itself, the CTA agrees at the barrier below
          own_ok = wait_own(ctl.b2, ctl.ph2, ctl.p2, p);
          if constexpr (Lay::SPLIT) fold_chunk(j == 1);
        }
        if constexpr (Lay::A24_TMEM) {
#pragma unroll
          for (int c = 0; c < C; ++c) put_act_tmem<NC, HC, PREC>(TA + lane_base, c, c0, a[c]);
          tc::tmem_st_wait();
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c)
#pragma unroll
            for (int h = 0; h < HC / 8; ++h) {
              float w8[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) w8[i] = a[c][h * 8 + i];
              put8<PREC>(sA24 + c * Lay::A24B, Lay::A24B, row, c0 + h * 8, NC, w8);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (__syncthreads_or(!own_ok || !b_ok)) { dead = true; return; }
        if (issuer) {
          tc::fence_after_sync();
          issue_g24(n, j, 3 * PK::T);
          tc::mma_commit(ctl.b2);
        }
        ctl.p2 = true;
      }
    } else if constexpr (Lay::B2B) {
      // GEMM1 of chunk j + 1 is issued right behind GEMM2 of chunk j, under one commit
      // (the tensor core runs them in order), so that a chunk waits for one MMA
      // completion, not two; B(j + 1) is requested once the wait for GEMM1(j) has
      // shown GEMM2(j - 1), the last reader of its buffer, complete
      fetch(lp, 0, n0);
      if (NCH > 1) fetch(lp, 1, n0 + 1);
      if (!wait_b(n0)) { dead = true; return; }
      tc::fence_async_smem();
      __syncthreads();
      if (issuer) {
        tc::fence_after_sync();
        issue_g1(n0);
        tc::mma_commit(ctl.b1);
      }
      ctl.p1 = true;
      bool b_ok = true;   // this thread's own wait for the next chunk's bases
      for (int j = 0; j < NCH; ++j) {
        const int n = n0 + j;
        // GEMM1(j) done, and with it GEMM2(j - 1); a failed wait for B(j) is agreed on here
        if (!wait_bar(ctl.b1, ctl.ph1, ctl.p1, p, b_ok)) { dead = true; return; }
        if constexpr (Lay::SPLIT) if (j > 0) fold_chunk(j == 1);
        if (j >= 1 && j + 1 < NCH) fetch(lp, j + 1, n + 1);
        fwd_epilogue(n);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (issuer) {
          tc::fence_after_sync();
          issue_g24(n, j, 3 * PK::T);
        }
        if (j + 1 < NCH) {
          // every thread waits for B(j + 1) on its own, without a CTA barrier: the MMA
          // issuers before GEMM1(j + 1), the others before the next epilogue reads the
          // chunk's biases
          b_ok = wait_b_own(n + 1);
          if (b_ok) {
            if (issuer) {
              issue_g1(n + 1);
              tc::mma_commit(ctl.b1);
            }
            ctl.p1 = true;
          } else {
            // GEMM2(j) is in flight: commit it for the drain
            if (issuer) tc::mma_commit(ctl.b2);
            ctl.p2 = true;
          }
          __syncwarp();
        } else {
          if (issuer) tc::mma_commit(ctl.b2);
          ctl.p2 = true;
        }
      }
    } else {
      fetch(lp, 0, n0);
      for (int j = 0; j < NCH; ++j) {
        const int n = n0 + j;
        if (j > 0 && !wait_bar(ctl.b2, ctl.ph2, ctl.p2, p)) { dead = true; return; }   // GEMM2(j-1) done
        if constexpr (Lay::SPLIT) if (j > 0) fold_chunk(j == 1);
        if (Lay::NB == 1 && j > 0) fetch(lp, j, n);
        if (!wait_b(n)) { dead = true; return; }
        if (Lay::NB >= 2 && j + 1 < NCH) fetch(lp, j + 1, n + 1);
        tc::fence_async_smem();
        __syncthreads();
        if (issuer) {
          tc::fence_after_sync();
          issue_g1(n);
          tc::mma_commit(ctl.b1);
        }
        ctl.p1 = true;
        if (!wait_bar(ctl.b1, ctl.ph1, ctl.p1, p)) { dead = true; return; }
        fwd_epilogue(n);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (issuer) {
          tc::fence_after_sync();
          issue_g24(n, j, 3 * PK::T);
          tc::mma_commit(ctl.b2);
        }
        ctl.p2 = true;
      }
    }
    ctl.chunk_ctr = n0 + NCH;
    if (!wait_bar(ctl.b2, ctl.ph2, ctl.p2, p)) { dead = true; return; }
    if (lead) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float v[RM];
        rank_c(c, v);
        if (l + 1 < L) {
          if (p.grad) {
#pragma unroll
            for (int k = 0; k < RM; ++k) qst[((l * 4 + c) * RM + k) * TNT + row] = v[k];
          }
          put_scaled(sA1, c, v, l + 1);
        } else {
          qL[c] = v[0];
        }
      }
    }
    tc::fence_before_sync();
  }
  float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float sL = s_s[L * RM];
  if (lead) {
#pragma unroll
    for (int c = 0; c < C; ++c) u[c] = Uout * sL * qL[c];
    u[0] += bout;
  }
  float ub[4] = {0.0f, 0.0f, 0.0f, 0.0f}, lpv = 0.0f;
  bool go = false;
  if (lead) go = residual_and_seeds(p, T, pt, row, u, ub, lpv);
  if (!__syncthreads_or(go)) return;      // evaluation mode: done

  // ---------------- reverse sweep
  const int DB0 = partial_db0(L, RM);
  float *prow = p.partial + (int64_t)tile * p.P;
  if (lead) {
    // loss, dL/ds of the linear output layer, dL/db of the output bias
    const float ls = warp_sum(lpv);
    float dsL = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) dsL += Uout * ub[c] * qL[c];
    const float s0 = warp_sum(dsL);
    const float s1 = warp_sum(ub[0]);
    if (lane == 0) {
      red_w[0] += ls;
      red_w[1 + L * RM] += s0;
      red_w[PL - 1] += s1;
    }
    // A3 of the last hidden layer: the output adjoint seeds
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float qb[RM];
#pragma unroll
      for (int k = 0; k < RM; ++k) qb[k] = 0.0f;
      qb[0] = sL * Uout * ub[c];
      put_rank_row<RM, PREC, NC>(sA3, c, qb, row);
    }
  }
  // (A3 of layer l < L - 1 is written at the end of layer l + 1: pbar * s^(l+1))
  for (int l = L - 1; l >= 0 && !dead; --l) {
    const unsigned char *lp = pack + (size_t)l * NCH * PK::CHUNK;
    if (lead) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float v[RM];
        if (l > 0) stored_c(l, c, v);
        else input_jet_c(c, v);
        put_scaled(sA1, c, v, l);
      }
    }
    const int n0 = ctl.chunk_ctr;
    if constexpr (Lay::B2B) {
      // as in the forward sweep: GEMM1 / GEMM3 of chunk j + 1 right behind GEMM4 of
      // chunk j, one commit for both
      fetch(lp, 0, n0);
      if (NCH > 1) fetch(lp, 1, n0 + 1);
      if (!wait_b(n0)) { dead = true; return; }
      tc::fence_async_smem();
      __syncthreads();
      if (issuer) {
        tc::fence_after_sync();
        issue_g13(n0);
        tc::mma_commit(ctl.b1);
      }
      ctl.p1 = true;
      bool b_ok = true;   // this thread's own wait for the next chunk's bases
      for (int j = 0; j < NCH; ++j) {
        const int n = n0 + j;
        // GEMM1 / GEMM3 (j) done, and with them GEMM4(j - 1); a failed wait for B(j) is
        // agreed on here
        if (!wait_bar(ctl.b1, ctl.ph1, ctl.p1, p, b_ok)) { dead = true; return; }
        if constexpr (Lay::SPLIT) if (j > 0) fold_chunk(j == 1);
        if (j >= 1 && j + 1 < NCH) fetch(lp, j + 1, n + 1);
        rev_epilogue(n);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (issuer) {
          tc::fence_after_sync();
          issue_g24(n, j, 2 * PK::T);
        }
        if (j + 1 < NCH) {
          // each thread's own wait for B(j + 1), as in the forward sweep
          b_ok = wait_b_own(n + 1);
          if (b_ok) {
            if (issuer) {
              issue_g13(n + 1);
              tc::mma_commit(ctl.b1);
            }
            ctl.p1 = true;
          } else {
            // GEMM4(j) is in flight: commit it for the drain
            if (issuer) tc::mma_commit(ctl.b2);
            ctl.p2 = true;
          }
          __syncwarp();
        } else {
          if (issuer) tc::mma_commit(ctl.b2);
          ctl.p2 = true;
        }
        // the chunk's dL/db columns, after the MMA issue (thread 0 issues too); the
        // partial sums in dbw are rewritten only after the next CTA-wide wait
        if (tid < NC) {
          // column tid of the chunk: warps (0..3) hold the first half, (4..7) the second
          const int h = tid / HC, cc = tid % HC;
          const float v = dbw[(4 * h + 0) * HC + cc] + dbw[(4 * h + 1) * HC + cc] +
                          dbw[(4 * h + 2) * HC + cc] + dbw[(4 * h + 3) * HC + cc];
          const int col = j * NC + tid;
          if (col < M) prow[DB0 + l * M + col] = v;
        }
        __syncwarp();
      }
    } else {
      fetch(lp, 0, n0);
      for (int j = 0; j < NCH; ++j) {
        const int n = n0 + j;
        if (j > 0 && !wait_bar(ctl.b2, ctl.ph2, ctl.p2, p)) { dead = true; return; }
        if constexpr (Lay::SPLIT) if (j > 0) fold_chunk(j == 1);
        if (Lay::NB == 1 && j > 0) fetch(lp, j, n);
        if (!wait_b(n)) { dead = true; return; }
        if (Lay::NB >= 2 && j + 1 < NCH) fetch(lp, j + 1, n + 1);
        tc::fence_async_smem();
        __syncthreads();
        if (issuer) {
          tc::fence_after_sync();
          issue_g13(n);
          tc::mma_commit(ctl.b1);
        }
        ctl.p1 = true;
        if (!wait_bar(ctl.b1, ctl.ph1, ctl.p1, p)) { dead = true; return; }
        rev_epilogue(n);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (issuer) {
          tc::fence_after_sync();
          issue_g24(n, j, 2 * PK::T);
          tc::mma_commit(ctl.b2);
        }
        ctl.p2 = true;
        if (tid < NC) {
          // column tid of the chunk: warps (0..3) hold the first half, (4..7) the second
          const int h = tid / HC, cc = tid % HC;
          const float v = dbw[(4 * h + 0) * HC + cc] + dbw[(4 * h + 1) * HC + cc] +
                          dbw[(4 * h + 2) * HC + cc] + dbw[(4 * h + 3) * HC + cc];
          const int col = j * NC + tid;
          if (col < M) prow[DB0 + l * M + col] = v;
        }
      }
    }
    ctl.chunk_ctr = n0 + NCH;
    if (!wait_bar(ctl.b2, ctl.ph2, ctl.p2, p)) { dead = true; return; }
    if (lead) {
      // dL/ds^l = sum_c pbar_c * q_c, and the output adjoint of layer l - 1
      float g[RM];
#pragma unroll
      for (int k = 0; k < RM; ++k) g[k] = 0.0f;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float pb[RM], v[RM];
        rank_c(c, pb);
        if (l > 0) stored_c(l, c, v);
        else input_jet_c(c, v);
#pragma unroll
        for (int k = 0; k < RM; ++k) g[k] = fmaf(pb[k], v[k], g[k]);
        if (l > 0) put_scaled(sA3, c, pb, l);
      }
      warp_accumulate<RM>(g, red_w, [&](int jj) { return 1 + l * RM + jj; });
    }
    tc::fence_before_sync();
  }
}

template <int RM, int PREC, int NC>
__global__ void __launch_bounds__(NTH, (tmem_cols<NC, RM, PREC>() == 256) ? 2 : 1) k_full_tc(const __grid_constant__ KParams p,
                                                  const unsigned char *__restrict__ pack) {
  using Lay = TcLayout<RM, PREC, NC>;
  static_assert(Lay::TM_END <= tmem_cols<NC, RM, PREC>(), "tensor-memory columns");
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x;
  const int L = p.L;
  float *fa = reinterpret_cast<float *>(sm + Lay::OFF_F);
  float *s_s = fa;
  const int PL = 2 + (L + 1) * RM;
  float *red_s = fa + (L + 1) * RM;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + ((Lay::OFF_F + Lay::floats(L) * 4 + 15) & ~15));
  uint32_t *tbase = reinterpret_cast<uint32_t *>(bar + 2 + Lay::NB);
  if (tid < 32) tc::tmem_alloc(tbase, tmem_cols<NC, RM, PREC>());
  if (tid == 0) {
    // b1, b2: one commit per MMA issuer; the B-buffer barriers: one arrival (expect_tx)
    for (int i = 0; i < 2 + Lay::NB; ++i) tc::mbar_init(&bar[i], i < 2 ? 4u : 1u);
    tc::fence_mbar_init();
  }
  if (p.step && blockIdx.x == 0 && tid == 0) atomicAdd((unsigned long long *)p.step, 1ull);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tbase;
  Ctl ctl{&bar[0], &bar[1], &bar[2], 0u, 0u, {0u, 0u, 0u, 0u}, 0, false, false,
          {false, false, false, false}};
  bool dead = false;
  float *qst = p.scratch + (size_t)blockIdx.x * (size_t)(L > 1 ? L - 1 : 1) * 4 * RM * TNT;
  const int ntiles = __ldg(p.tile_off + p.n_inst);
  for (int tile = blockIdx.x; tile < ntiles && !dead; tile += gridDim.x) {
    const Tile T = decode_tile(p, tile);
    __syncthreads();
    for (int j = tid; j < (L + 1) * RM; j += NTH) {
      const int l = j / RM, k = j % RM;
      s_s[j] = (k < p.r[l]) ? __ldg(p.s + (int64_t)T.inst * p.sum_r + p.roff[l] + k) : 0.0f;
    }
    for (int j = tid; j < 4 * PL; j += NTH) red_s[j] = 0.0f;
    __syncthreads();
    if (T.kind == KIND_INT)
      tc_tile<RM, PREC, 4, NC>(p, T, tile, sm, pack, qst, tb, ctl, dead);
    else
      tc_tile<RM, PREC, 1, NC>(p, T, tile, sm, pack, qst, tb, ctl, dead);
    if (dead) break;
    if (p.grad) {
      __syncthreads();
      for (int j = tid; j < PL; j += NTH) {
        const float acc = red_s[j] + red_s[PL + j] + red_s[2 * PL + j] + red_s[3 * PL + j];
        if (j == 0 && !isfinite(acc)) set_status(p.status, DEV_NONFINITE);
        // entries 0 .. PL-2 are the loss and dL/ds; the last is the output-bias dL/db
        const int dst = j < PL - 1 ? j : partial_db0(L, RM) + L * p.M;
        p.partial[(int64_t)tile * p.P + dst] = acc;
      }
    }
  }
  if (dead) {
    // let the MMAs and copies this CTA started finish before TMEM and shared memory
    // are released: a fixed bound of its own, whatever the caller's wait cap
    constexpr uint32_t kDrainPolls = 1u << 20;
    if (ctl.p1) tc::mbar_wait(ctl.b1, ctl.ph1, kDrainPolls);
    if (ctl.p2) tc::mbar_wait(ctl.b2, ctl.ph2, kDrainPolls);
    for (int b = 0; b < Lay::NB; ++b)
      if (ctl.pb[b]) tc::mbar_wait(&ctl.bb[b], ctl.phb[b], kDrainPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tb, tmem_cols<NC, RM, PREC>());
}

template <int RM, int PREC, int NC>
cudaError_t launch_tc_t(const KParams &p, const void *pack, int grid_cap, cudaStream_t st) {
  using Lay = TcLayout<RM, PREC, NC>;
  const size_t bytes = (size_t)Lay::bytes(p.L);
  cudaError_t e = cudaFuncSetAttribute(k_full_tc<RM, PREC, NC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // every CTA holds tmem_cols<NC, RM, PREC>() TMEM columns: at most 512 / that many per SM
  const int grid = std::max(1, std::min(grid_cap, sms * (512 / tmem_cols<NC, RM, PREC>())));
  k_full_tc<RM, PREC, NC><<<grid, NTH, bytes, st>>>(p, static_cast<const unsigned char *>(pack));
  return cudaGetLastError();
}

template <int RM, int NC, int ES = 2>
int pk_chunk() { return Pk<RM, NC, ES>::CHUNK; }

}  // namespace
}  // namespace lrnr
