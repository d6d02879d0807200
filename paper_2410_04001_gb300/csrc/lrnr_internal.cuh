// Internal declarations shared by the CUDA translation units of liblrnr.so.
//
// Work decomposition.  Collocation points are cut into tiles of NT points that
// never straddle an instance or a point class (interior, initial, periodic pair);
// tile_off[i] is the first tile of instance i.  A persistent grid walks the tile
// list; each tile leaves one row of partial sums (loss, dL/ds, dL/db) in the
// workspace, and a second kernel adds an instance's rows in tile order, so the
// result does not depend on scheduling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lrnr.h"

namespace lrnr {

constexpr int LMAX = 16;      // hidden layers supported
constexpr int R1 = 2;         // padded rank of the input layer (input is (x, t))
constexpr int RMAX = 64;      // largest padded hidden rank
constexpr int RHMAX = 32;     // largest EIM row count per layer
constexpr float TWO_PI_F = 6.28318530717958647692f;

enum PointKind { KIND_INT = 0, KIND_IC = 1, KIND_BC = 2 };

// Error codes the kernels write into the device status word (first writer wins).
// DEV_BADBATCH: a batch's CSR offsets decrease, start below zero or end past the
// host totals; no point of the call is processed.
enum DevStatus { DEV_OK = 0, DEV_NONFINITE = 1, DEV_TIMEOUT = 2, DEV_SINGULAR = 3, DEV_BADBATCH = 4 };

struct KParams {
  int L, M, n_inst;
  int RM;                      // padded hidden rank used by the packs
  int RH;                      // padded EIM row count (fast form)
  int rh[LMAX];                // EIM rows kept per hidden layer (fast form)
  int r[LMAX + 1];             // ranks of the L+1 weight layers
  int roff[LMAX + 2];          // offsets of each layer's s in an instance vector
  int sum_r;
  // batch (device)
  const float *beta, *nu, *rho, *s;
  const int64_t *int_off, *ic_off, *bc_off;
  const float *x_int, *t_int, *x_ic, *t_bc;
  int64_t tot[3];              // host totals of interior points, initial points, pairs
  const int64_t *norm;         // [n_inst][3] MSE denominators, or null: the own counts
  // schedule
  const int32_t *tile_off;     // [n_inst+1]
  int nt;                      // points per tile (pairs per periodic tile: nt/2)
  // packed weights (device)
  const float *pack;
  // gradient mode
  int grad;
  float *partial;              // [n_tiles][P]
  int P;
  int loss;                    // lrnr_loss
  float w[3];
  // evaluation mode outputs (any may be null)
  float *u, *ut, *ux, *uxx, *res, *res_ic, *res_bc;
  int64_t *step;               // spinprop: incremented once by block 0
  int *status;
  float *scratch;              // per-CTA store of layer inputs (FP32 and tensor-core kernels)
  int fused_tiles;             // the tile kernel computes the tile offsets itself
  int fast_regs;               // FastLRNR kernel build: 3 = 168 registers, else 255
  int fastk;                   // FastLRNR in reduced coordinates (ranks 32 / 64, fastk.cu)
  uint32_t max_wait;           // iteration cap of every device-side wait
  // Fixed-order reduction inside the FastLRNR kernel (fused_red != 0; chosen for
  // batches whose tiles fit in one round of the grid, where a second launch would
  // cost more than the reduction).  Tiles form groups of kRedGroup consecutive
  // tiles; the CTA that completes a group (ticket) sums the group's rows of each
  // instance in tile order into gpart[g + inst]; the CTA that completes an
  // instance's last group sums its group rows in order and writes the outputs, or
  // applies Adam to s when adam_s is set.
  int fused_red;
  int n_groups;                // groups of the tile list (host bound)
  float *gpart;                // [(n_groups + n_inst)][P] group rows
  int *tickets;                // [n_groups] group, [n_inst] instance, [1] step tickets (zero)
  const int32_t *rows;         // fast dL/db scatter map [L][RH] (-1 = unused)
  int sum_m;
  float *loss_out, *dL_ds, *dL_db;
  float *adam_s, *adam_m, *adam_v;
  float lr, b1, b2, eps, lam;
  const float *anchor;
};

constexpr int kRedGroup = 32;   // tiles per reduction group

// --- layout of the FP32 packs -------------------------------------------------
// Fast pack: per hidden layer l: Uh [RH][RM], bh [RH], Vh [RH][RM]; then V^0 [2][R1],
// then U^L (scalar), b^L (scalar).  Unused (padded) entries are zero.
__host__ __device__ inline int fast_layer_floats(int RM, int RH) { return RH * RM * 2 + RH; }
__host__ __device__ inline int fast_pack_floats(int L, int RM, int RH) {
  return L * fast_layer_floats(RM, RH) + 2 * R1 + 2;
}
// Full pack: per hidden layer l: U^l [M][RM], b^l [pad4(M)], V^{l+1} [M][RM]; then
// V^0 [2][R1], U^L, b^L.  Every row starts on a 16-byte boundary.
__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }
__host__ __device__ inline int64_t full_layer_floats(int M, int RM) {
  return (int64_t)M * RM * 2 + pad4(M);
}
__host__ __device__ inline int64_t full_pack_floats(int L, int M, int RM) {
  return (int64_t)L * full_layer_floats(M, RM) + 2 * R1 + 2;
}

// Partial-sum row layout: [0] loss, [1 + l*RM + k] dL/ds (l = 0..L), then dL/db:
// fast: [DB0 + l*RH + i] (hidden layers) and [DB0 + L*RH] (output bias);
// full: [DB0 + l*M + i] and [DB0 + L*M].
__host__ __device__ inline int partial_db0(int L, int RM) { return 1 + (L + 1) * RM; }
__host__ __device__ inline int partial_len(int L, int RM, int nb) { return partial_db0(L, RM) + nb + 1; }

// --- device helpers ----------------------------------------------------------
__device__ __forceinline__ void set_status(int *status, int code) {
  if (status) atomicCAS(status, DEV_OK, code);
}

struct Tile {
  int inst, kind;
  int64_t first;   // first point (interior / initial) or first pair (periodic)
  int count;       // points (or pairs) in this tile
};

// Tiles of instance i: interior and initial points nt per tile, periodic pairs
// nt/2 per tile.
__device__ __forceinline__ int32_t tiles_of(const int64_t *io, const int64_t *co, const int64_t *bo,
                                            int i, int nt) {
  const int64_t nI = io[i + 1] - io[i], nC = co[i + 1] - co[i], nB = bo[i + 1] - bo[i];
  const int half = nt / 2;
  return (int32_t)((nI + nt - 1) / nt + (nC + nt - 1) / nt + (nB + half - 1) / half);
}

// True when the CSR offsets of instances [b, e) are non-decreasing, and, for the
// first and last instance, start at or above zero and end at or below the host
// totals: then every tile reads points inside the caller's arrays and the tile
// count is within the host bound the workspace was sized for.
__device__ __forceinline__ bool offsets_ok(const int64_t *io, const int64_t *co, const int64_t *bo,
                                           const int64_t (&tot)[3], int n_inst, int b, int e) {
  bool ok = true;
  for (int i = b; i < e; ++i)
    ok = ok && io[i + 1] >= io[i] && co[i + 1] >= co[i] && bo[i + 1] >= bo[i];
  if (b == 0 && e > 0) ok = ok && io[0] >= 0 && co[0] >= 0 && bo[0] >= 0;
  if (e == n_inst && b < e)
    ok = ok && io[n_inst] <= tot[0] && co[n_inst] <= tot[1] && bo[n_inst] <= tot[2];
  return ok;
}

// Tile offsets computed by one CTA into shared memory (toff_s[n_inst + 1]); used by
// kernels that fuse the tile schedule.  Block 0 also publishes them to p.tile_off
// for the reduction kernel that runs next.  A batch whose offsets fail offsets_ok
// gets no tiles (every offset zero) and DEV_BADBATCH.  Call with all threads of the
// block.
__device__ __forceinline__ void block_tile_offsets(const KParams &p, int32_t *toff_s,
                                                   int32_t *scan_s) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int chunk = (p.n_inst + nth - 1) / nth;
  const int b = min(p.n_inst, tid * chunk), e = min(p.n_inst, b + chunk);
  const bool bad =
      __syncthreads_or(!offsets_ok(p.int_off, p.ic_off, p.bc_off, p.tot, p.n_inst, b, e));
  int32_t acc = 0;
  if (!bad)
    for (int i = b; i < e; ++i) acc += tiles_of(p.int_off, p.ic_off, p.bc_off, i, p.nt);
  scan_s[tid] = acc;
  __syncthreads();
  for (int off = 1; off < nth; off *= 2) {
    const int32_t v = tid >= off ? scan_s[tid - off] : 0;
    __syncthreads();
    scan_s[tid] += v;
    __syncthreads();
  }
  int32_t run = scan_s[tid] - acc;
  for (int i = b; i < e; ++i) {
    toff_s[i] = run;
    if (!bad) run += tiles_of(p.int_off, p.ic_off, p.bc_off, i, p.nt);
  }
  if (tid == nth - 1) toff_s[p.n_inst] = scan_s[nth - 1];
  if (bad && blockIdx.x == 0 && tid == 0) set_status(p.status, DEV_BADBATCH);
  __syncthreads();
  if (blockIdx.x == 0)
    for (int i = tid; i <= p.n_inst; i += nth) const_cast<int32_t *>(p.tile_off)[i] = toff_s[i];
}

__device__ __forceinline__ Tile decode_tile(const KParams &p, int tile,
                                            const int32_t *toff = nullptr) {
  if (!toff) toff = p.tile_off;
  // largest i with tile_off[i] <= tile
  int lo = 0, hi = p.n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  Tile t;
  t.inst = lo;
  int j = tile - toff[lo];
  int64_t a = __ldg(p.int_off + lo), nI = __ldg(p.int_off + lo + 1) - a;
  int ntI = (int)((nI + p.nt - 1) / p.nt);
  if (j < ntI) {
    t.kind = KIND_INT; t.first = a + (int64_t)j * p.nt;
    t.count = (int)(nI - (int64_t)j * p.nt < p.nt ? nI - (int64_t)j * p.nt : p.nt);
    return t;
  }
  j -= ntI;
  int64_t c = __ldg(p.ic_off + lo), nC = __ldg(p.ic_off + lo + 1) - c;
  int ntC = (int)((nC + p.nt - 1) / p.nt);
  if (j < ntC) {
    t.kind = KIND_IC; t.first = c + (int64_t)j * p.nt;
    t.count = (int)(nC - (int64_t)j * p.nt < p.nt ? nC - (int64_t)j * p.nt : p.nt);
    return t;
  }
  j -= ntC;
  int half = p.nt / 2;
  int64_t e = __ldg(p.bc_off + lo), nB = __ldg(p.bc_off + lo + 1) - e;
  t.kind = KIND_BC; t.first = e + (int64_t)j * half;
  t.count = (int)(nB - (int64_t)j * half < half ? nB - (int64_t)j * half : half);
  return t;
}

// Sum N values (N a power of two, <= 32) over the 32 lanes of a warp by recursive
// halving.  On return lane l holds the warp total of value index l / (32 / N).
template <int N>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[N]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = N / 2, off = 16; h >= 1; h /= 2, off /= 2) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      float send = up ? v[i] : v[i + h];
      float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float r = v[0];
#pragma unroll
  for (int off = 16 / N; off >= 1; off /= 2) r += __shfl_xor_sync(0xffffffffu, r, off);
  return r;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off >= 1; off /= 2) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Drop the L2 copy of a scratch range of this CTA without writing it back to
// DRAM (discard.global.L2 on whole 128-byte lines; the contents become undefined).
// The range is data the tile no longer needs (the layer stores of the gradient
// sweep, re-written before the next read), so its dirty lines would otherwise be
// written back to DRAM for nothing.  Call with all threads of the CTA, after a
// barrier that follows every read of the range; `base` and `bytes` are multiples
// of 128.
__device__ __forceinline__ void l2_discard(const void *base, size_t bytes) {
  const char *b = static_cast<const char *>(base);
  for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)blockDim.x * 128)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(b + o) : "memory");
}

// tanh jet: value z = tanh(a), first derivative d1 = 1 - z^2 and second d2 = -2 z d1.
// For |a| >= 1/2, from the identity tanh|a| = 1 - q with q = 2 / (exp(2|a|) + 1) in
// (0, 1], so that 1 - z^2 = q (2 - q) keeps its relative accuracy where tanh
// saturates; exp on the MUFU unit (ex2.approx, relative error about 2^-22) and its
// reciprocal give z and d1 to a few 1e-7 relative there.  For |a| < 1/2, where
// 1 - q cancels, z comes from the Maclaurin series of tanh, whose coefficient of
// a^(2n-1) is 2^(2n) (2^(2n) - 1) B_2n / (2n)! (B_2n the Bernoulli numbers), taken
// to a^15: the first omitted term is below 1e-8 of z at |a| = 1/2, and z keeps a
// relative error of about 1e-7 down to the smallest normal |a| (z = a there; ftz
// flushes subnormal a to zero).  d1 is q (2 - q) for every a.  Large |a| overflows
// exp to +inf, whose reciprocal is +0 (z = +-1, d1 = 0); a NaN input stays NaN.
__device__ __forceinline__ void tanh_d(float a, float &z, float &d1, float &d2) {
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fabsf(a) * 2.88539008177792681f));   // 2 / ln 2
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.0f));
  const float q = 2.0f * r;
  const float a2 = a * a;
  float c = -929569.0f / 638512875.0f;
  c = fmaf(a2, c, 21844.0f / 6081075.0f);
  c = fmaf(a2, c, -1382.0f / 155925.0f);
  c = fmaf(a2, c, 62.0f / 2835.0f);
  c = fmaf(a2, c, -17.0f / 315.0f);
  c = fmaf(a2, c, 2.0f / 15.0f);
  c = fmaf(a2, c, -1.0f / 3.0f);
  const float zs = fmaf(a * a2, c, a);
  z = fabsf(a) < 0.5f ? zs : copysignf(1.0f - q, a);
  d1 = q * (2.0f - q);
  d2 = -2.0f * z * d1;
}

// --- host-side launchers (defined in the .cu files) --------------------------
constexpr int kSmemBudget = 220 * 1024;   // dynamic shared memory a tile kernel may use

size_t fast_smem_bytes(int L, int RM, int RH, int NT, int P);
int fast_choose_nt(int L, int RM, int RH, int P);
int fast_ctas_per_sm(const KParams &p);                 // resident CTAs of k_fast per SM
size_t fast_scratch_floats(int L, int RM, int RH, int NT, int grid);  // gradient-sweep store
size_t full_fp32_smem_bytes(int L, int RM, int NT, int P);
int full_fp32_choose_nt(int L, int RM, int P);
int full_fp32_ctas_per_sm(const KParams &p);
size_t full_fp32_scratch_floats(int L, int RM, int NT, int grid);
cudaError_t launch_tile_offsets(const KParams &p, int32_t *tile_off, cudaStream_t st);
// grid_cap bounds the persistent grid (never more CTAs than tiles); the FastLRNR
// kernel is launched with exactly `grid` CTAs (its scratch is sized for them).
cudaError_t launch_fast(const KParams &p, int grid, cudaStream_t st);
// FastLRNR FP32 in reduced coordinates for padded ranks 32 and 64 (RH 8 or 16);
// fused_inst > 0: the layout with the tile offsets of that many instances in shared
// memory (KParams::fused_tiles).
bool fastk_supported(int L, int RM, int RH, int P, int fused_inst);
int fastk_nt();
size_t fastk_scratch_floats(int L, int RH, int grid);
int fastk_ctas_per_sm(const KParams &p);
cudaError_t launch_fastk(const KParams &p, int grid, cudaStream_t st);
cudaError_t launch_full_fp32(const KParams &p, int grid, cudaStream_t st);
// Full-width FP32 at padded ranks 32 and 64: RM / 16 threads per point
// (full_fp32_sliced.cu); points per tile, shared memory, scratch, occupancy, launch.
int full_fp32_sl_nt(int RM);
size_t full_fp32_sl_smem_bytes(int L, int M, int RM);
size_t full_fp32_sl_scratch_floats(int L, int RM, int grid);
int full_fp32_sl_ctas_per_sm(const KParams &p);
cudaError_t launch_full_fp32_sl(const KParams &p, int grid, cudaStream_t st);
// NC: 32-column chunks (full-width networks, one CTA per SM) or 16-column chunks
// (narrow networks, two CTAs per SM while RM <= 32).
cudaError_t launch_full_tc_tf32(const KParams &p, const void *tc_pack, int NC, int grid_cap,
                                cudaStream_t st);
cudaError_t launch_full_tc(const KParams &p, const void *tc_pack, int prec, int NC, int grid_cap,
                           cudaStream_t st);
cudaError_t launch_reduce(const KParams &p, int nb_needed, int form_fast, const int32_t *rows,
                          int rows_stride, float *loss_out, float *dL_ds, float *dL_db,
                          int sum_m, int num_sms, cudaStream_t st);
// Batches of a few instances (at most 2 * num_sms / 8) reduce with one 8-CTA
// cluster per instance; otherwise the two-level reduction runs on gsum (n_inst x
// groups x entries floats) and cnt (n_inst zeroed ints), which must then be given.
cudaError_t launch_reduce_adam(const KParams &p, float *s, float *m, float *v, const int64_t *step,
                               float lr, float b1, float b2, float eps, float lam,
                               const float *anchor, float *loss_out, float *gsum, int *cnt,
                               int num_sms, cudaStream_t st);
size_t adam_group_floats(int n_inst, int L, int RM);
cudaError_t launch_eim_greedy(double *R, int M, int64_t K, int rhat, double tol, int32_t *rows,
                              double *Xi, int *used_dev, double *colmax, int64_t *colarg,
                              int *status, cudaStream_t st);

}  // namespace lrnr
