// Full-width LRNR residual + adjoint in FP32 for padded ranks 32 and 64 (Sec. 2.1
// Eq. 2.1-2.2, Sec. 2.3): the paper's convection-diffusion-reaction network
// r = (1, 49, 30, 25, 1) pads to 64, the adjoint-stress network to 32.
//
// A point's rank-r jets do not fit in one thread's registers at these ranks (two jets
// of 4 channels x RM floats are live through a layer), so TPP = RM / 16 consecutive
// threads share a point: thread q of the point holds entries [16 q, 16 q + 16) of
// every rank-r jet of the point.  Per row i of a layer:
//   a_i  = sum over the slices of U_i . (s * q)   (partial dot products, completed by
//                                                  log2(TPP) shuffles; every thread of
//                                                  the point then holds the same a_i)
//   z_i  = tanh jet of a_i                          (computed by each of the TPP threads)
//   q'  += V'_i z_i                                 (each thread its own slice)
// and in the reverse sweep the adjoint of the row's output, V'_i . qbar, is completed
// the same way before the tanh-jet adjoint and pbar += U_i^T abar (each its slice).  As
// in the single-thread kernel the M-wide activations are never stored: each layer's
// rank-r input is kept per thread in a per-CTA global scratch area (L2-resident) and
// the reverse sweep rebuilds the pre-activations from it.
//
// The bias gradient has M entries per layer: the warps' sums of each block of 8 rows
// go to a small shared buffer, and after a barrier warp 0 adds the four warps' sums in
// warp order into one shared row, so the result is deterministic and the shared
// memory holds a single M-wide row per layer (about 64 KB at M = 4,000, L = 4).
#include "lrnr_internal.cuh"
#include "point_common.cuh"
#include "simt_common.cuh"

#include <algorithm>

namespace lrnr {
namespace {

constexpr int SNT = 128;   // threads per CTA
constexpr int RS = 16;     // rank entries per thread slice
constexpr int kWarps = SNT / 32;

// Shared memory (floats): the tile's s, one small row per warp (loss, dL/ds by padded
// rank, output-bias dL/db), the CTA's hidden-layer dL/db row (L x M), and the warps'
// 8-row bias sums (two buffers).
struct SlLayout {
  int s, wrow, pw, db, dbw, total;
  __host__ __device__ SlLayout(int L, int M, int RM) {
    s = 0;
    pw = 2 + (L + 1) * RM;
    wrow = (L + 1) * RM;
    db = wrow + kWarps * pw;
    dbw = db + ((L * M + 3) & ~3);
    total = dbw + 2 * kWarps * 8;
  }
};

__host__ __device__ inline size_t sl_store_floats(int L, int RM, int NPT) {
  return (size_t)(L > 1 ? L - 1 : 1) * 4 * RM * NPT;
}

__device__ __forceinline__ float2 sf2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Sum over the TPP threads of a point (consecutive lanes); every one gets the total.
template <int TPP>
__device__ __forceinline__ float point_sum(float v) {
#pragma unroll
  for (int off = 1; off < TPP; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// This thread's slice of a row W[0..N): entries [16 q, 16 q + 16) as pairs, zero past N.
template <int N>
__device__ __forceinline__ void load_slice(const float *__restrict__ W, int q, float2 (&w)[RS / 2]) {
  if constexpr (N >= RS) {
#pragma unroll
    for (int k = 0; k < RS; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(W + q * RS + k));
      w[k / 2] = make_float2(v.x, v.y);
      w[k / 2 + 1] = make_float2(v.z, v.w);
    }
  } else {
    // N = 2 (the input layer) or 1 (the output layer): only slice 0 holds entries
#pragma unroll
    for (int k = 0; k < RS / 2; ++k) w[k] = make_float2(0.0f, 0.0f);
    if (q == 0) {
      if constexpr (N == 2) w[0] = __ldg(reinterpret_cast<const float2 *>(W));
      else w[0] = make_float2(__ldg(W), 0.0f);
    }
  }
}

template <int TPP, int C>
__device__ __forceinline__ void slice_dot(const float2 (&w)[RS / 2], const float2 (&v)[C][RS / 2],
                                          float (&out)[C]) {
  float2 acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int kk = 0; kk < RS / 2; ++kk)
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = sf2(w[kk], v[c][kk], acc[c]);
#pragma unroll
  for (int c = 0; c < C; ++c) out[c] = point_sum<TPP>(acc[c].x + acc[c].y);
}

template <int RM, int TPP, int NI, int NO, int C>
__device__ __forceinline__ void sl_layer_fwd(const float *__restrict__ U, const float *__restrict__ b,
                                             const float *__restrict__ Vn, int M, int q,
                                             const float2 (&y)[C][RS / 2], float2 (&qn)[C][RS / 2]) {
#pragma unroll 2
  for (int i = 0; i < M; ++i) {
    float2 uw[RS / 2], vw[RS / 2];
    load_slice<NI>(U + (int64_t)i * RM, q, uw);
    load_slice<NO>(Vn + (int64_t)i * RM, q, vw);
    float a[C][1], av[C];
    slice_dot<TPP, C>(uw, y, av);
#pragma unroll
    for (int c = 0; c < C; ++c) a[c][0] = av[c];
    a[0][0] += __ldg(b + i);
    act_fwd<C, 1>(a);
#pragma unroll
    for (int kk = 0; kk < RS / 2; ++kk)
#pragma unroll
      for (int c = 0; c < C; ++c) qn[c][kk] = sf2(vw[kk], make_float2(a[c][0], a[c][0]), qn[c][kk]);
  }
}

// Reverse of one hidden layer: pb += U^T abar (this thread's slice) and the rows' bias
// gradients added into db_l[0..M) (shared, warp order).
template <int RM, int TPP, int NI, int NO, int C>
__device__ __forceinline__ void sl_layer_bwd(const float *__restrict__ U, const float *__restrict__ b,
                                             const float *__restrict__ Vn, int M, int q,
                                             const float2 (&y)[C][RS / 2],
                                             const float2 (&qb)[C][RS / 2], float2 (&pb)[C][RS / 2],
                                             float *db_l, float *dbw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0, blk = 0; i0 < M; i0 += 8, ++blk) {
    float ab0[8];
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) {
      const int i = i0 + ii;
      ab0[ii] = 0.0f;
      if (i < M) {
        float2 uw[RS / 2], vw[RS / 2];
        load_slice<NI>(U + (int64_t)i * RM, q, uw);
        load_slice<NO>(Vn + (int64_t)i * RM, q, vw);
        float av[C], wv[C], a[C][1], wb[C][1];
        slice_dot<TPP, C>(uw, y, av);
        slice_dot<TPP, C>(vw, qb, wv);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          a[c][0] = av[c];
          wb[c][0] = wv[c];
        }
        a[0][0] += __ldg(b + i);
        act_bwd<C, 1>(a, wb);
#pragma unroll
        for (int kk = 0; kk < RS / 2; ++kk)
#pragma unroll
          for (int c = 0; c < C; ++c)
            pb[c][kk] = sf2(uw[kk], make_float2(wb[c][0], wb[c][0]), pb[c][kk]);
        ab0[ii] = q == 0 ? wb[0][0] : 0.0f;   // one contribution per point
      }
    }
    // the warp's sums of the 8 rows, then (barrier) the warps' sums in warp order
    const float r = warp_reduce_scatter<8>(ab0);
    float *buf = dbw + (blk & 1) * kWarps * 8;
    if ((lane & 3) == 0) buf[warp * 8 + (lane >> 2)] = r;
    __syncthreads();
    if (threadIdx.x < 8 && i0 + (int)threadIdx.x < M) {
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += buf[w * 8 + threadIdx.x];
      db_l[i0 + threadIdx.x] += s;
    }
  }
}

// Sum v over the points of the warp that share this thread's slice index (lanes
// differing in the point bits) and add the totals into dst[0..RS) from the lanes of
// the warp's first point.
template <int TPP>
__device__ __forceinline__ void slice_accumulate(float (&v)[RS], float *dst) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < RS; ++k)
#pragma unroll
    for (int off = TPP; off < 32; off <<= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  if (lane < TPP)
#pragma unroll
    for (int k = 0; k < RS; ++k) dst[k] += v[k];
}

template <int RM, int TPP, int C>
__device__ void sl_tile(const KParams &p, const Tile &T, const float *__restrict__ s_s,
                        float *__restrict__ q_s, float *wrow, float *db_s, float *dbw) {
  constexpr int RP = RS / 2;
  constexpr int NPT = SNT / TPP;
  const int tid = threadIdx.x;
  const int pp = tid / TPP, q = tid % TPP;
  const int L = p.L, M = p.M;
  const int64_t LS = full_layer_floats(M, RM);
  const float *V0 = p.pack + L * LS;
  const float Uout = __ldg(V0 + 2 * R1);
  const float bout = __ldg(V0 + 2 * R1 + 1);

  const PointIn pt = load_point(p, T, pp);
  const float x = pt.x, t = pt.t;
  const float v00 = __ldg(V0 + 0), v01 = __ldg(V0 + 1), v10 = __ldg(V0 + R1), v11 = __ldg(V0 + R1 + 1);

  float2 qv[C][RP];
  auto input_jet = [&]() {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int kk = 0; kk < RP; ++kk) qv[c][kk] = make_float2(0.0f, 0.0f);
    if (q == 0) {
      qv[0][0] = make_float2(v00 * x + v10 * t, v01 * x + v11 * t);
      if constexpr (C >= 3) {
        qv[1][0] = make_float2(v10, v11);
        qv[2][0] = make_float2(v00, v01);
      }
    }
  };
  // this thread's slice of s^l, as pairs
  auto s_pair = [&](int l, int kk) {
    return make_float2(s_s[l * RM + q * RS + 2 * kk], s_s[l * RM + q * RS + 2 * kk + 1]);
  };
  auto slot = [&](int l, int c, int k) { return (((l - 1) * 4 + c) * RS + k) * SNT + tid; };
  input_jet();

  for (int l = 0; l < L; ++l) {
    const float *U = p.pack + l * LS;
    const float *b = U + (int64_t)M * RM;
    const float *Vn = b + pad4(M);
    if (p.grad && l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int kk = 0; kk < RP; ++kk) {
          q_s[slot(l, c, 2 * kk)] = qv[c][kk].x;
          q_s[slot(l, c, 2 * kk + 1)] = qv[c][kk].y;
        }
    }
    float2 y[C][RP];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int kk = 0; kk < RP; ++kk) {
        y[c][kk] = __fmul2_rn(qv[c][kk], s_pair(l, kk));
        qv[c][kk] = make_float2(0.0f, 0.0f);
      }
    if (l == 0 && l == L - 1) sl_layer_fwd<RM, TPP, R1, 1, C>(U, b, Vn, M, q, y, qv);
    else if (l == 0) sl_layer_fwd<RM, TPP, R1, RM, C>(U, b, Vn, M, q, y, qv);
    else if (l == L - 1) sl_layer_fwd<RM, TPP, RM, 1, C>(U, b, Vn, M, q, y, qv);
    else sl_layer_fwd<RM, TPP, RM, RM, C>(U, b, Vn, M, q, y, qv);
  }
  // the output layer's rank-1 input lives in slice 0: broadcast it to the point
  const int lead = (threadIdx.x & 31) & ~(TPP - 1);
  const float sL = s_s[L * RM];
  float qL[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < C; ++c) {
    qL[c] = __shfl_sync(0xffffffffu, qv[c][0].x, lead);
    u[c] = Uout * sL * qL[c];
  }
  u[0] += bout;

  float ub[4], lp;
  if (!residual_and_seeds(p, T, pt, pp, u, ub, lp, TPP, q == 0)) return;
  if (q != 0) lp = 0.0f;

  const int DB0 = partial_db0(L, RM);
  const int PW = 2 + (L + 1) * RM;
  {
    float dsL = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) dsL += Uout * ub[c] * qL[c];
    const float ls = warp_sum(lp);
    const float s0 = warp_sum(q == 0 ? dsL : 0.0f);
    const float s1 = warp_sum(q == 0 ? ub[0] : 0.0f);
    if ((tid & 31) == 0) {
      wrow[0] += ls;
      wrow[1 + L * RM] += s0;
      wrow[PW - 1] += s1;
    }
  }
  float2 qb[C][RP];
#pragma unroll
  for (int c = 0; c < C; ++c) {
#pragma unroll
    for (int kk = 0; kk < RP; ++kk) qb[c][kk] = make_float2(0.0f, 0.0f);
    if (q == 0) qb[c][0].x = sL * Uout * ub[c];
  }
  auto load_q = [&](int l) {
    if (l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int kk = 0; kk < RP; ++kk)
          qv[c][kk] = make_float2(q_s[slot(l, c, 2 * kk)], q_s[slot(l, c, 2 * kk + 1)]);
    } else {
      input_jet();
    }
  };
  for (int l = L - 1; l >= 0; --l) {
    const float *U = p.pack + l * LS;
    const float *b = U + (int64_t)M * RM;
    const float *Vn = b + pad4(M);
    load_q(l);
    float2 y[C][RP], pb[C][RP];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int kk = 0; kk < RP; ++kk) {
        y[c][kk] = __fmul2_rn(qv[c][kk], s_pair(l, kk));
        pb[c][kk] = make_float2(0.0f, 0.0f);
      }
    float *db_l = db_s + l * M;
    if (l == 0 && l == L - 1) sl_layer_bwd<RM, TPP, R1, 1, C>(U, b, Vn, M, q, y, qb, pb, db_l, dbw);
    else if (l == 0) sl_layer_bwd<RM, TPP, R1, RM, C>(U, b, Vn, M, q, y, qb, pb, db_l, dbw);
    else if (l == L - 1) sl_layer_bwd<RM, TPP, RM, 1, C>(U, b, Vn, M, q, y, qb, pb, db_l, dbw);
    else sl_layer_bwd<RM, TPP, RM, RM, C>(U, b, Vn, M, q, y, qb, pb, db_l, dbw);
    load_q(l);
    // dL/ds^l = sum_c pbar_c * q_c on this slice, summed over the warp's points
    float g[RS];
#pragma unroll
    for (int kk = 0; kk < RP; ++kk) {
      float2 d = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int c = 0; c < C; ++c) d = sf2(pb[c][kk], qv[c][kk], d);
      g[2 * kk] = d.x;
      g[2 * kk + 1] = d.y;
    }
    slice_accumulate<TPP>(g, wrow + 1 + l * RM + q * RS);
    if (l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int kk = 0; kk < RP; ++kk) qb[c][kk] = __fmul2_rn(pb[c][kk], s_pair(l, kk));
    }
  }
  (void)NPT;
}

template <int RM, int TPP>
__global__ void __launch_bounds__(SNT, 2) k_full_fp32_sl(const __grid_constant__ KParams p) {
  extern __shared__ __align__(16) float smem[];
  constexpr int NPT = SNT / TPP;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int L = p.L, M = p.M;
  const SlLayout lay(L, M, RM);
  float *s_s = smem + lay.s;
  float *wrow_s = smem + lay.wrow;
  float *db_s = smem + lay.db;
  float *dbw = smem + lay.dbw;
  float *q_s = p.scratch + (size_t)blockIdx.x * sl_store_floats(L, RM, NPT);
  if (p.step && blockIdx.x == 0 && tid == 0) atomicAdd((unsigned long long *)p.step, 1ull);
  const int ntiles = __ldg(p.tile_off + p.n_inst);
  const int DB0 = partial_db0(L, RM);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile T = decode_tile(p, tile);
    __syncthreads();
    for (int j = tid; j < (L + 1) * RM; j += SNT) {
      const int l = j / RM, k = j % RM;
      s_s[j] = (k < p.r[l]) ? __ldg(p.s + (int64_t)T.inst * p.sum_r + p.roff[l] + k) : 0.0f;
    }
    if (p.grad) {
      for (int j = tid; j < kWarps * lay.pw; j += SNT) wrow_s[j] = 0.0f;
      for (int j = tid; j < L * M; j += SNT) db_s[j] = 0.0f;
    }
    __syncthreads();
    float *wrow = wrow_s + warp * lay.pw;
    if (T.kind == KIND_INT)
      sl_tile<RM, TPP, 4>(p, T, s_s, q_s, wrow, db_s, dbw);
    else
      sl_tile<RM, TPP, 1>(p, T, s_s, q_s, wrow, db_s, dbw);
    if (p.grad) {
      __syncthreads();
      for (int j = tid; j < p.P; j += SNT) {
        float acc = 0.0f;
        if (j < DB0 || j == p.P - 1) {
          const int wj = j < DB0 ? j : lay.pw - 1;
#pragma unroll
          for (int w = 0; w < kWarps; ++w) acc += wrow_s[w * lay.pw + wj];
        } else {
          acc = db_s[j - DB0];
        }
        if (j == 0 && !isfinite(acc)) set_status(p.status, DEV_NONFINITE);
        p.partial[(int64_t)tile * p.P + j] = acc;
      }
    }
  }
}

template <int RM, int TPP>
cudaError_t launch_sl_t(const KParams &p, int grid, cudaStream_t st) {
  const SlLayout lay(p.L, p.M, RM);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_full_fp32_sl<RM, TPP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_full_fp32_sl<RM, TPP><<<std::max(1, grid), SNT, bytes, st>>>(p);
  return cudaGetLastError();
}

template <int RM, int TPP>
int sl_ctas_per_sm_t(const KParams &p) {
  const SlLayout lay(p.L, p.M, RM);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  if (cudaFuncSetAttribute(k_full_fp32_sl<RM, TPP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_full_fp32_sl<RM, TPP>, SNT, bytes) !=
      cudaSuccess)
    return 1;
  return std::max(1, per_sm);
}

}  // namespace

// Points per tile of the sliced kernel (128 threads, RM / 16 threads per point).
int full_fp32_sl_nt(int RM) { return SNT / (RM / RS); }

size_t full_fp32_sl_smem_bytes(int L, int M, int RM) {
  return (size_t)SlLayout(L, M, RM).total * sizeof(float);
}

size_t full_fp32_sl_scratch_floats(int L, int RM, int grid) {
  return sl_store_floats(L, RM, full_fp32_sl_nt(RM)) * (size_t)grid;
}

int full_fp32_sl_ctas_per_sm(const KParams &p) {
  if (p.RM == 32) return sl_ctas_per_sm_t<32, 2>(p);
  if (p.RM == 64) return sl_ctas_per_sm_t<64, 4>(p);
  return 1;
}

cudaError_t launch_full_fp32_sl(const KParams &p, int grid, cudaStream_t st) {
  if (!p.scratch && p.grad) return cudaErrorInvalidValue;
  if (p.nt != full_fp32_sl_nt(p.RM)) return cudaErrorInvalidValue;
  if (p.RM == 32) return launch_sl_t<32, 2>(p, grid, st);
  if (p.RM == 64) return launch_sl_t<64, 4>(p, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace lrnr
