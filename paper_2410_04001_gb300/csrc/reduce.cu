// Tile schedule, fixed-order reduction of per-tile partial sums, and the fused
// Adam step on s (Sec. 2.3 gradient assembly; Sec. 3.2 Eq. 3.7; Sec. 4 Adam).
#include <cooperative_groups.h>

#include "lrnr_internal.cuh"

namespace lrnr {
namespace {

// The reduction kernels are launched as programmatic dependents of the tile kernel
// before them (launch_dependent): they may start while its last tiles run, and wait
// here, after any prologue that reads nothing the tile kernel writes, until it has
// completed and its writes are visible.  Without the launch attribute this returns at
// once.
__device__ __forceinline__ void wait_prerequisite_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch `kernel` on `st` as a programmatic dependent of the kernel before it.
template <typename Kern, typename... Args>
cudaError_t launch_dependent(Kern kernel, dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// tile_off[i] = first tile of instance i (exclusive prefix sum); one block.  A batch
// whose offsets fail offsets_ok gets no tiles (every offset zero) and DEV_BADBATCH.
__global__ void __launch_bounds__(1024) k_tile_offsets(const __grid_constant__ KParams p,
                                                       int32_t *tile_off) {
  __shared__ int32_t sums[1024];
  const int tid = threadIdx.x;
  const int n_inst = p.n_inst;
  const int64_t *io = p.int_off, *co = p.ic_off, *bo = p.bc_off;
  const int chunk = (n_inst + 1023) / 1024;
  const int b = min(n_inst, tid * chunk), e = min(n_inst, b + chunk);
  const bool bad = __syncthreads_or(!offsets_ok(io, co, bo, p.tot, n_inst, b, e));
  int32_t acc = 0;
  if (!bad)
    for (int i = b; i < e; ++i) acc += tiles_of(io, co, bo, i, p.nt);
  sums[tid] = acc;
  __syncthreads();
  for (int off = 1; off < 1024; off *= 2) {
    const int32_t v = tid >= off ? sums[tid - off] : 0;
    __syncthreads();
    sums[tid] += v;
    __syncthreads();
  }
  int32_t run = sums[tid] - acc;
  for (int i = b; i < e; ++i) {
    tile_off[i] = run;
    if (!bad) run += tiles_of(io, co, bo, i, p.nt);
  }
  if (tid == 1023) tile_off[n_inst] = sums[1023];
  if (bad && tid == 0) set_status(p.status, DEV_BADBATCH);
}

// Sum of column j over the rows t0 + g, t0 + g + 32, ... < t1 of the partial
// matrix, in row order; the loads of up to 16 rows are issued before their
// additions (one L2 round trip per 16 rows).
__device__ __forceinline__ float column_sum(const float *__restrict__ part, int P, int j, int t0,
                                            int t1, int g) {
  float acc = 0.0f;
  for (int t = t0 + g; t < t1; t += 16 * 32) {
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int tq = t + 32 * q;
      v[q] = tq < t1 ? __ldg(part + (int64_t)tq * P + j) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) acc += v[q];
  }
  return acc;
}

struct RedArgs {
  const float *partial;
  const int32_t *tile_off;
  int P, n_needed;        // row length, leading entries to reduce
  int L, M, RM, RH, fast;
  int r[LMAX + 1], roff[LMAX + 2];
  int sum_r, sum_m;
  const int32_t *rows;    // fast: [L][RH], -1 = unused
  float *loss_out, *dL_ds, *dL_db;
};

__device__ __forceinline__ void scatter_out(const RedArgs &a, int i, int j, float v) {
  const int DB0 = 1 + (a.L + 1) * a.RM;
  if (j == 0) {
    if (a.loss_out) a.loss_out[i] = v;
  } else if (j < DB0) {
    const int l = (j - 1) / a.RM, k = (j - 1) % a.RM;
    if (k < a.r[l]) a.dL_ds[(int64_t)i * a.sum_r + a.roff[l] + k] = v;
  } else if (a.dL_db) {
    const int jj = j - DB0;
    float *db = a.dL_db + (int64_t)i * a.sum_m;
    if (a.fast) {
      if (jj == a.L * a.RH) db[a.L * a.M] = v;
      else {
        const int l = jj / a.RH, ii = jj % a.RH;
        const int row = a.rows[l * a.RH + ii];
        if (row >= 0) db[l * a.M + row] = v;
      }
    } else {
      db[jj] = v;   // hidden layers l*M + i, then the output bias at L*M
    }
  }
}

// grid (n_inst, ceil(n_needed / 32)), block (32, 32): x = entry, y = tile group.
__global__ void __launch_bounds__(1024) k_reduce(const __grid_constant__ RedArgs a) {
  __shared__ float sh[32][33];
  wait_prerequisite_grid();
  const int i = blockIdx.x;
  const int j = blockIdx.y * 32 + threadIdx.x;
  const int t0 = a.tile_off[i], t1 = a.tile_off[i + 1];
  float acc = 0.0f;
  if (j < a.n_needed)
    acc = column_sum(a.partial, a.P, j, t0, t1, threadIdx.y);
  sh[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && j < a.n_needed) {
    float tot = 0.0f;
#pragma unroll
    for (int g = 0; g < 32; ++g) tot += sh[g][threadIdx.x];
    scatter_out(a, i, j, tot);
  }
}

struct AdamArgs {
  RedArgs red;
  float *s, *m, *v;
  const int64_t *step;
  float lr, b1, b2, eps, lam;
  const float *anchor;
};

// Two-level version for the SPInProp step: block (i, g) sums the partial rows
// t = t0 + g, t0 + g + TG, ... of instance i for every entry and writes one group
// row; the last block of instance i to finish (atomic ticket) adds the TG group
// rows in order and applies Adam.  Deterministic: the order of every sum is fixed.
constexpr int kAdamGroups = 32;

__global__ void __launch_bounds__(256) k_reduce_adam2(const __grid_constant__ AdamArgs A,
                                                      float *__restrict__ gsum, int *cnt) {
  const RedArgs &a = A.red;
  __shared__ float gsh[(LMAX + 1) * RMAX];
  __shared__ float lsum[8];
  __shared__ float loss_sh;
  __shared__ int last;
  const int i = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
  wait_prerequisite_grid();
  const int t0 = a.tile_off[i], t1 = a.tile_off[i + 1];
  const int DB0 = 1 + (a.L + 1) * a.RM;
  float *grow = gsum + ((int64_t)i * kAdamGroups + g) * DB0;
  for (int j = tid; j < DB0; j += 256) {
    // rows t0 + g, t0 + g + G, ... in order; the loads of up to 16 rows are issued
    // before their additions (one L2 round trip per 16 rows)
    float acc = 0.0f;
    for (int t = t0 + g; t < t1; t += 16 * kAdamGroups) {
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int tq = t + q * kAdamGroups;
        v[q] = tq < t1 ? __ldg(a.partial + (int64_t)tq * a.P + j) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += v[q];
    }
    grow[j] = acc;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&cnt[i], 1) == kAdamGroups - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const float *gi = gsum + (int64_t)i * kAdamGroups * DB0;
  for (int j = tid; j < DB0; j += 256) {
    float v[kAdamGroups];
#pragma unroll
    for (int gg = 0; gg < kAdamGroups; ++gg) v[gg] = __ldcg(gi + gg * DB0 + j);
    float tot = 0.0f;
#pragma unroll
    for (int gg = 0; gg < kAdamGroups; ++gg) tot += v[gg];
    if (j == 0) loss_sh = tot;
    else {
      const int l = (j - 1) / a.RM, k = (j - 1) % a.RM;
      if (k < a.r[l]) gsh[a.roff[l] + k] = tot;
    }
  }
  __syncthreads();
  const int64_t k = *A.step;
  const float bc1 = 1.0f - powf(A.b1, (float)k);
  const float bc2 = 1.0f - powf(A.b2, (float)k);
  float loc = 0.0f;
  for (int q = tid; q < a.sum_r; q += 256) {
    const int64_t o = (int64_t)i * a.sum_r + q;
    const float sv = A.s[o];
    float gr = gsh[q];
    if (A.anchor) {
      const float d = sv - A.anchor[o];
      loc += A.lam * fabsf(d);
      gr += A.lam * (float)((d > 0.0f) - (d < 0.0f));
    }
    const float mv = A.b1 * A.m[o] + (1.0f - A.b1) * gr;
    const float vv = A.b2 * A.v[o] + (1.0f - A.b2) * gr * gr;
    A.m[o] = mv;
    A.v[o] = vv;
    A.s[o] = sv - A.lr * (mv / bc1) / (sqrtf(vv / bc2) + A.eps);
  }
  loc = warp_sum(loc);
  if ((tid & 31) == 0) lsum[tid >> 5] = loc;
  __syncthreads();
  if (tid == 0) {
    float lt = 0.0f;
    for (int w = 0; w < 8; ++w) lt += lsum[w];
    if (a.loss_out) a.loss_out[i] = loss_sh + lt;
    cnt[i] = 0;   // ready for the next step
  }
}

// Cluster form of the reduction + Adam (one cluster of kClRed CTAs per instance):
// CTA c of the cluster sums the instance's tile rows t0 + c + kClRed * m in COLS-wide
// column slices (1024 / COLS row phases per CTA, one round of up to 16 loads per
// thread for the batches it is used for), adds its row phases in order into a
// shared row, and CTA 0 adds the kClRed shared rows through distributed shared
// memory in rank order before the Adam update.  No tickets, no second pass over
// global memory; every sum is taken in a fixed order.
constexpr int kClRed = 8;
constexpr int kClThreads = 1024;

template <int COLS>
__global__ void __cluster_dims__(kClRed, 1, 1) __launch_bounds__(kClThreads)
    k_reduce_adam_cl(const __grid_constant__ AdamArgs A) {
  namespace cg = cooperative_groups;
  constexpr int PH = kClThreads / COLS;          // row phases per CTA
  cg::cluster_group cl = cg::this_cluster();
  const RedArgs &a = A.red;
  __shared__ float part[PH][COLS];
  __shared__ float tot[COLS];
  __shared__ float gsh[(LMAX + 1) * RMAX];
  __shared__ float lsum[kClThreads / 32];
  const int i = blockIdx.x / kClRed;
  const int crank = (int)cl.block_rank();
  const int tid = threadIdx.x, col = tid % COLS, ph = tid / COLS;
  const int DB0 = 1 + (a.L + 1) * a.RM;
  // CTA 0 starts reading s, m, v (and the anchor) of its Adam entries now (the tile
  // kernel before this one reads s and writes none of them)
  float sv = 0.0f, mv0 = 0.0f, vv0 = 0.0f, an = 0.0f;
  const int64_t o = (int64_t)i * a.sum_r + tid;
  const bool adam_lane = crank == 0 && tid < a.sum_r;
  if (adam_lane) {
    sv = A.s[o];
    mv0 = A.m[o];
    vv0 = A.v[o];
    if (A.anchor) an = A.anchor[o];
  }
  wait_prerequisite_grid();
  const int t0 = a.tile_off[i], t1 = a.tile_off[i + 1];
  float acc = 0.0f;
  if (col < DB0) {
    constexpr int STEP = kClRed * PH;             // distance between this thread's rows
    for (int t = t0 + crank + kClRed * ph; t < t1; t += 16 * STEP) {
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int tq = t + q * STEP;
        v[q] = tq < t1 ? __ldg(a.partial + (int64_t)tq * a.P + col) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += v[q];
    }
  }
  part[ph][col] = acc;
  __syncthreads();
  if (tid < COLS) {
    float s2 = 0.0f;
#pragma unroll
    for (int q = 0; q < PH; ++q) s2 += part[q][tid];
    tot[tid] = s2;
  }
  cl.sync();
  if (crank == 0) {
    for (int j = tid; j < DB0; j += kClThreads) {
      float g = 0.0f;
      for (int r = 0; r < kClRed; ++r) g += cl.map_shared_rank(tot, r)[j];
      if (j == 0) part[0][0] = g;
      else {
        const int l = (j - 1) / a.RM, k = (j - 1) % a.RM;
        if (k < a.r[l]) gsh[a.roff[l] + k] = g;
      }
    }
  }
  // every CTA's shared row stays alive until CTA 0 has read it
  cl.sync();
  if (crank != 0) return;
  const int64_t k = *A.step;
  const float bc1 = 1.0f - powf(A.b1, (float)k);
  const float bc2 = 1.0f - powf(A.b2, (float)k);
  float loc = 0.0f;
  if (adam_lane) {
    float gr = gsh[tid];
    if (A.anchor) {
      const float d = sv - an;
      loc = A.lam * fabsf(d);
      gr += A.lam * (float)((d > 0.0f) - (d < 0.0f));
    }
    const float mv = A.b1 * mv0 + (1.0f - A.b1) * gr;
    const float vv = A.b2 * vv0 + (1.0f - A.b2) * gr * gr;
    A.m[o] = mv;
    A.v[o] = vv;
    A.s[o] = sv - A.lr * (mv / bc1) / (sqrtf(vv / bc2) + A.eps);
  }
  loc = warp_sum(loc);
  if ((tid & 31) == 0) lsum[tid >> 5] = loc;
  __syncthreads();
  if (tid == 0) {
    float lt = 0.0f;
    for (int w = 0; w < kClThreads / 32; ++w) lt += lsum[w];
    if (a.loss_out) a.loss_out[i] = part[0][0] + lt;
  }
}

// Cluster form of the plain reduction (loss, dL/ds, dL/db): cluster (instance i,
// column block y of 128 entries) of kClRed CTAs; CTA c sums the rows t0 + c + kClRed m
// in 8 row phases, CTA 0 adds the CTAs' rows through distributed shared memory in rank
// order and writes the results.
__global__ void __cluster_dims__(kClRed, 1, 1) __launch_bounds__(kClThreads)
    k_reduce_cl(const __grid_constant__ RedArgs a) {
  namespace cg = cooperative_groups;
  constexpr int COLS = 128, PH = kClThreads / COLS;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ float part[PH][COLS];
  __shared__ float tot[COLS];
  const int i = blockIdx.x / kClRed;
  const int crank = (int)cl.block_rank();
  const int tid = threadIdx.x, col = tid % COLS, ph = tid / COLS;
  const int j = blockIdx.y * COLS + col;
  wait_prerequisite_grid();
  const int t0 = a.tile_off[i], t1 = a.tile_off[i + 1];
  float acc = 0.0f;
  if (j < a.n_needed) {
    constexpr int STEP = kClRed * PH;
    for (int t = t0 + crank + kClRed * ph; t < t1; t += 16 * STEP) {
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int tq = t + q * STEP;
        v[q] = tq < t1 ? __ldg(a.partial + (int64_t)tq * a.P + j) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += v[q];
    }
  }
  part[ph][col] = acc;
  __syncthreads();
  if (tid < COLS) {
    float s2 = 0.0f;
#pragma unroll
    for (int q = 0; q < PH; ++q) s2 += part[q][tid];
    tot[tid] = s2;
  }
  cl.sync();
  if (crank == 0 && tid < COLS && j < a.n_needed) {
    float g = 0.0f;
    for (int r = 0; r < kClRed; ++r) g += cl.map_shared_rank(tot, r)[tid];
    scatter_out(a, i, j, g);
  }
  cl.sync();
}

// Adam on s from a given gradient (the update of spinprop_step, Sec. 4, with the
// l1 locality subgradient of Eq. 3.7); block i updates instance i.  The step number
// is the counter's value plus one (k_step_advance moves the counter afterwards).
// loss_out[i] = loss_in[i] + lam sum |s - anchor| (the locality term at the s the
// gradient was taken at), summed in a fixed order.
__global__ void __launch_bounds__(256) k_adam_update(int sum_r, const float *__restrict__ g,
                                                     float *s, float *m, float *v,
                                                     const int64_t *step, float lr, float b1,
                                                     float b2, float eps, float lam,
                                                     const float *anchor, const float *loss_in,
                                                     float *loss_out) {
  __shared__ float lsh[8];
  const int i = blockIdx.x, tid = threadIdx.x;
  const float kstep = (float)(*step + 1);
  const float bc1 = 1.0f - powf(b1, kstep);
  const float bc2 = 1.0f - powf(b2, kstep);
  float loc = 0.0f;
  for (int q = tid; q < sum_r; q += 256) {
    const int64_t o = (int64_t)i * sum_r + q;
    const float sv = s[o];
    float gr = g[o];
    if (anchor) {
      const float d = sv - anchor[o];
      loc += lam * fabsf(d);
      gr += lam * (float)((d > 0.0f) - (d < 0.0f));
    }
    const float mv = b1 * m[o] + (1.0f - b1) * gr;
    const float vv = b2 * v[o] + (1.0f - b2) * gr * gr;
    m[o] = mv;
    v[o] = vv;
    s[o] = sv - lr * (mv / bc1) / (sqrtf(vv / bc2) + eps);
  }
  loc = warp_sum(loc);
  if ((tid & 31) == 0) lsh[tid >> 5] = loc;
  __syncthreads();
  if (tid == 0 && loss_out) {
    float lt = 0.0f;
    for (int w = 0; w < 8; ++w) lt += lsh[w];
    loss_out[i] = (loss_in ? loss_in[i] : 0.0f) + lt;
  }
}

__global__ void k_step_advance(int64_t *step) { *step += 1; }

void fill_red(RedArgs &a, const KParams &p, int n_needed, int fast, const int32_t *rows,
              float *loss_out, float *dL_ds, float *dL_db, int sum_m) {
  a.partial = p.partial;
  a.tile_off = p.tile_off;
  a.P = p.P;
  a.n_needed = n_needed;
  a.L = p.L;
  a.M = p.M;
  a.RM = p.RM;
  a.RH = p.RH;
  a.fast = fast;
  for (int l = 0; l <= LMAX; ++l) a.r[l] = p.r[l];
  for (int l = 0; l <= LMAX + 1; ++l) a.roff[l] = p.roff[l];
  a.sum_r = p.sum_r;
  a.sum_m = sum_m;
  a.rows = rows;
  a.loss_out = loss_out;
  a.dL_ds = dL_ds;
  a.dL_db = dL_db;
}

}  // namespace

cudaError_t launch_tile_offsets(const KParams &p, int32_t *tile_off, cudaStream_t st) {
  k_tile_offsets<<<1, 1024, 0, st>>>(p, tile_off);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const KParams &p, int n_needed, int form_fast, const int32_t *rows,
                          int /*rows_stride*/, float *loss_out, float *dL_ds, float *dL_db,
                          int sum_m, int num_sms, cudaStream_t st) {
  RedArgs a;
  fill_red(a, p, n_needed, form_fast, rows, loss_out, dL_ds, dL_db, sum_m);
  const int64_t blocks = ((int64_t)n_needed + 127) / 128;
  if ((int64_t)p.n_inst * kClRed * blocks <= 2 * (int64_t)num_sms) {
    // few instances: one cluster per (instance, 128 entries), one round of loads
    return launch_dependent(k_reduce_cl, dim3(p.n_inst * kClRed, (unsigned)blocks), dim3(kClThreads),
                            st, a);
  } else {
    dim3 grid(p.n_inst, (n_needed + 31) / 32), block(32, 32);
    return launch_dependent(k_reduce, grid, block, st, a);
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce_adam(const KParams &p, float *s, float *m, float *v, const int64_t *step,
                               float lr, float b1, float b2, float eps, float lam,
                               const float *anchor, float *loss_out, float *gsum, int *cnt,
                               int num_sms, cudaStream_t st) {
  AdamArgs A;
  fill_red(A.red, p, 1 + (p.L + 1) * p.RM, 0, nullptr, loss_out, nullptr, nullptr, 0);
  A.s = s;
  A.m = m;
  A.v = v;
  A.step = step;
  A.lr = lr;
  A.b1 = b1;
  A.b2 = b2;
  A.eps = eps;
  A.lam = lam;
  A.anchor = anchor;
  const int DB0 = 1 + (p.L + 1) * p.RM;
  // the cluster form pays off while the clusters fit in about two waves of the grid;
  // many instances already give the two-level form enough parallelism
  if (p.sum_r <= kClThreads && DB0 <= 256 && (int64_t)p.n_inst * kClRed <= 2 * (int64_t)num_sms) {
    if (DB0 <= 128)
      return launch_dependent(k_reduce_adam_cl<128>, dim3(p.n_inst * kClRed), dim3(kClThreads), st, A);
    else
      return launch_dependent(k_reduce_adam_cl<256>, dim3(p.n_inst * kClRed), dim3(kClThreads), st, A);
  } else if (gsum && cnt) {
    return launch_dependent(k_reduce_adam2, dim3(p.n_inst, kAdamGroups), dim3(256), st, A, gsum, cnt);
  } else {
    return cudaErrorInvalidValue;   // the two-level form needs its group rows and tickets
  }
  return cudaGetLastError();
}

size_t adam_group_floats(int n_inst, int L, int RM) {
  return (size_t)n_inst * kAdamGroups * partial_db0(L, RM);
}

cudaError_t launch_adam_update(int n_inst, int sum_r, const float *g, float *s, float *m, float *v,
                               int64_t *step, float lr, float b1, float b2, float eps, float lam,
                               const float *anchor, const float *loss_in, float *loss_out,
                               cudaStream_t st) {
  k_adam_update<<<n_inst, 256, 0, st>>>(sum_r, g, s, m, v, step, lr, b1, b2, eps, lam, anchor,
                                        loss_in, loss_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_step_advance<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

}  // namespace lrnr
