// FastLRNR residual + adjoint, FP32 SIMT (kernel template) (Sec. 2.2 Eq. 2.8, Sec. 2.3).
//
// One thread per collocation point.  The reduced bases (Uhat, bhat, Vhat: a few KB
// per layer) and the tile's coefficients s live in shared memory and are read
// with warp-uniform (broadcast) loads.  Each layer streams over its rhat rows: for
// row i the thread forms the pre-activation jet a_i = Uhat_i . (s * zhat) (+ bhat_i)
// (four scalars, one per jet channel), pushes it through tanh and accumulates the
// next rank-r jet zhat' += Vhat_i w_i; the reverse sweep does the same per row for
// the adjoint.  Rank-r vectors are held as pairs of adjacent entries so that the
// products run on the packed two-lane FP32 FMA (two multiply-adds per instruction;
// each lane rounds exactly like a scalar fmaf).  Row loops are not unrolled, which
// keeps the kernel small enough for the instruction cache.  The forward keeps each
// hidden layer's input jet in a per-CTA global scratch area ([slot][thread],
// coalesced, L2-resident) so the reverse sweep can rebuild pre-activations without
// re-running the network.  Per-layer gradient pieces are summed over the warp and
// over the tile's warps in a fixed order, giving one partial row per tile.
#pragma once

#include <algorithm>

#include "lrnr_internal.cuh"
#include "point_common.cuh"
#include "simt_common.cuh"

namespace lrnr {

// Shared memory of one CTA (floats): the reduced bases, the tile's s, the staged
// pre-activation adjoints of the current layer [row][thread][channel], one partial
// row per warp and, when the kernel computes the tile schedule, the tile offsets.
struct FastLayout {
  int pack, s, ab, red, toff, scan, total;
  __host__ __device__ FastLayout(int L, int RM, int RH, int NT, int P, int fused_inst = 0) {
    pack = 0;
    s = (fast_pack_floats(L, RM, RH) + 3) & ~3;
    ab = (s + (L + 1) * RM + 3) & ~3;
    red = ab + 4 * RH * NT;
    toff = red + (NT / 32) * P;
    scan = toff + (fused_inst ? fused_inst + 1 : 0);
    total = scan + (fused_inst ? NT : 0);
  }
};

// Largest instance count for which the FastLRNR kernel computes its own tile offsets.
constexpr int kFastFusedInstMax = 4096;

// Floats of layer-input store per CTA (global scratch).
__host__ __device__ inline size_t fast_store_floats(int L, int RM, int NT) {
  return (size_t)(L > 1 ? L - 1 : 1) * 4 * RM * NT;
}

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

// Rank-r jet of C channels, RM entries each, held as RM/2 pairs.
template <int C, int RM>
struct Jet {
  float2 v[C][RM / 2];
};

// The input jet of hidden layer l: stored by the forward (l > 0) or rebuilt from
// the point (l == 0: zhat^0 = V^0^T z^0).
template <int RM, int C>
__device__ __forceinline__ void load_input(int l, const float2 *__restrict__ q_g, int NT, int tid,
                                           const float *V0, float x, float t, Jet<C, RM> &q) {
  if (l > 0) {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int h = 0; h < RM / 2; ++h) q.v[c][h] = q_g[(((l - 1) * 4 + c) * (RM / 2) + h) * NT + tid];
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int h = 0; h < RM / 2; ++h) q.v[c][h] = make_float2(0.0f, 0.0f);
    // R1 = 2: entries 0 and 1 form the first pair
    q.v[0][0] = make_float2(V0[0] * x + V0[R1] * t, V0[1] * x + V0[R1 + 1] * t);
    if constexpr (C >= 3) {
      q.v[1][0] = make_float2(V0[R1], V0[R1 + 1]);
      q.v[2][0] = make_float2(V0[0], V0[1]);
    }
  }
}

template <int RM, int C>
__device__ __forceinline__ void store_input(int l, float2 *__restrict__ q_g, int NT, int tid,
                                            const Jet<C, RM> &q) {
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int h = 0; h < RM / 2; ++h) q_g[(((l - 1) * 4 + c) * (RM / 2) + h) * NT + tid] = q.v[c][h];
}

// out[c] += W[0..NI) . v[c][0..NI), accumulated as even/odd partial sums.
template <int RM, int NI, int C>
__device__ __forceinline__ void row_dot(const float *__restrict__ W, const Jet<C, RM> &v,
                                        float (&out)[C]) {
  float2 acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = make_float2(out[c], 0.0f);
  if constexpr (NI % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NI; k += 4) {
      const float4 w = *reinterpret_cast<const float4 *>(W + k);
      const float2 w01 = make_float2(w.x, w.y), w23 = make_float2(w.z, w.w);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        acc[c] = f2fma(w01, v.v[c][k / 2], acc[c]);
        acc[c] = f2fma(w23, v.v[c][k / 2 + 1], acc[c]);
      }
    }
  } else if constexpr (NI == 2) {
    const float2 w01 = *reinterpret_cast<const float2 *>(W);
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = f2fma(w01, v.v[c][0], acc[c]);
  } else {   // NI == 1
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c].x = fmaf(W[0], v.v[c][0].x, acc[c].x);
  }
#pragma unroll
  for (int c = 0; c < C; ++c) out[c] = acc[c].x + acc[c].y;
}

// acc[c][0..NI) += W[0..NI) * v[c]
template <int RM, int NI, int C>
__device__ __forceinline__ void row_axpy(const float *__restrict__ W, const float (&v)[C],
                                         Jet<C, RM> &acc) {
  if constexpr (NI % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NI; k += 4) {
      const float4 w = *reinterpret_cast<const float4 *>(W + k);
      const float2 w01 = make_float2(w.x, w.y), w23 = make_float2(w.z, w.w);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float2 vc = splat(v[c]);
        acc.v[c][k / 2] = f2fma(w01, vc, acc.v[c][k / 2]);
        acc.v[c][k / 2 + 1] = f2fma(w23, vc, acc.v[c][k / 2 + 1]);
      }
    }
  } else if constexpr (NI == 2) {
    const float2 w01 = *reinterpret_cast<const float2 *>(W);
#pragma unroll
    for (int c = 0; c < C; ++c) acc.v[c][0] = f2fma(w01, splat(v[c]), acc.v[c][0]);
  } else {   // NI == 1
#pragma unroll
    for (int c = 0; c < C; ++c) acc.v[c][0].x = fmaf(W[0], v[c], acc.v[c][0].x);
  }
}

template <int RM, int C>
__device__ __forceinline__ void jet_scale(Jet<C, RM> &q, const float *__restrict__ sl) {
#pragma unroll
  for (int h = 0; h < RM / 2; ++h) {
    const float2 s2 = *reinterpret_cast<const float2 *>(sl + 2 * h);
#pragma unroll
    for (int c = 0; c < C; ++c) q.v[c][h] = f2mul(q.v[c][h], s2);
  }
}

template <int RM, int C>
__device__ __forceinline__ void jet_zero(Jet<C, RM> &q) {
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int h = 0; h < RM / 2; ++h) q.v[c][h] = make_float2(0.0f, 0.0f);
}

// tanh jet of one row, in place: a = (a0, a_t, a_x, a_xx) -> (z, z_t, z_x, z_xx).
template <int C>
__device__ __forceinline__ void jet_fwd(float (&a)[C]) {
  float z, d1, d2;
  tanh_d(a[0], z, d1, d2);
  if constexpr (C == 4) a[3] = d2 * a[2] * a[2] + d1 * a[3];
  if constexpr (C >= 3) {
    a[1] *= d1;
    a[2] *= d1;
  }
  a[0] = z;
}

// Adjoint of jet_fwd: given the pre-activation a and the output adjoint wb,
// overwrite wb with the pre-activation adjoint.
template <int C>
__device__ __forceinline__ void jet_bwd(const float (&a)[C], float (&wb)[C]) {
  float z, d1, d2;
  tanh_d(a[0], z, d1, d2);
  float ab0 = wb[0] * d1;
  if constexpr (C >= 3) ab0 += d2 * (wb[1] * a[1] + wb[2] * a[2]);
  if constexpr (C == 4) {
    const float d3 = d1 * (6.0f * z * z - 2.0f);
    ab0 += wb[3] * (d3 * a[2] * a[2] + d2 * a[3]);
    wb[2] = wb[2] * d1 + 2.0f * wb[3] * d2 * a[2];
    wb[3] = wb[3] * d1;
  } else if constexpr (C >= 3) {
    wb[2] = wb[2] * d1;
  }
  if constexpr (C >= 3) wb[1] = wb[1] * d1;
  wb[0] = ab0;
}

// One reduced layer forward: y (= s * zhat, input jet) -> qn (next rank-r jet).
template <int RM, int C, int NI, int NO>
__device__ __forceinline__ void layer_fwd(const float *__restrict__ Uh, const float *__restrict__ bh,
                                          const float *__restrict__ Vh, int nrows,
                                          const Jet<C, RM> &y, Jet<C, RM> &qn) {
#pragma unroll 1
  for (int i = 0; i < nrows; ++i) {
    float a[C];
    a[0] = bh[i];
#pragma unroll
    for (int c = 1; c < C; ++c) a[c] = 0.0f;
    row_dot<RM, NI, C>(Uh + i * RM, y, a);
    jet_fwd<C>(a);
    row_axpy<RM, NO, C>(Vh + i * RM, a, qn);
  }
}

// One reduced layer reverse, in two passes over the rows so that no more than two
// rank-r jets are live at once:
//   pass 1: rebuild a_i = Uhat_i . y (+ bhat_i), pull wb_i = Vhat_i . qb back through
//           the tanh jet, stage abar_i (all channels) in ab_s[row][thread][channel];
//   pass 2: pb = Uhat^T abar from the staged rows.
template <int RM, int C, int NI, int NO>
__device__ __forceinline__ void layer_bwd(const float *__restrict__ Uh, const float *__restrict__ bh,
                                          const float *__restrict__ Vh, int nrows,
                                          const Jet<C, RM> &y, const Jet<C, RM> &qb,
                                          float4 *ab_s, int NT) {
#pragma unroll 1
  for (int i = 0; i < nrows; ++i) {
    float a[C], wb[C];
    a[0] = bh[i];
#pragma unroll
    for (int c = 1; c < C; ++c) a[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) wb[c] = 0.0f;
    row_dot<RM, NI, C>(Uh + i * RM, y, a);
    row_dot<RM, NO, C>(Vh + i * RM, qb, wb);
    jet_bwd<C>(a, wb);
    float4 v = make_float4(wb[0], 0.0f, 0.0f, 0.0f);
    if constexpr (C == 4) v = make_float4(wb[0], wb[1], wb[2], wb[3]);
    ab_s[i * NT + threadIdx.x] = v;
  }
}

template <int RM, int C, int NI>
__device__ __forceinline__ void layer_bwd_pbar(const float *__restrict__ Uh, int nrows,
                                               const float4 *ab_s, int NT, Jet<C, RM> &pb) {
#pragma unroll 2
  for (int i = 0; i < nrows; ++i) {
    const float4 v = ab_s[i * NT + threadIdx.x];
    float ab[C];
    ab[0] = v.x;
    if constexpr (C == 4) { ab[1] = v.y; ab[2] = v.z; ab[3] = v.w; }
    row_axpy<RM, NI, C>(Uh + i * RM, ab, pb);
  }
}

template <int RM, int RH, int C>
__device__ void fast_tile(const KParams &p, const Tile &T, const float *__restrict__ w_s,
                          const float *__restrict__ s_s, float2 *__restrict__ q_g, float4 *ab_s,
                          float *red_w) {
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int L = p.L;
  const int LS = fast_layer_floats(RM, RH);
  const float *V0 = w_s + L * LS;
  const float Uout = w_s[L * LS + 2 * R1];
  const float bout = w_s[L * LS + 2 * R1 + 1];

  const PointIn pt = load_point(p, T, tid);
  const float x = pt.x, t = pt.t;

  // ---- forward: zhat^0 = V^0^T z^0, then the reduced layers (Eq. 2.8)
  Jet<C, RM> q;
  load_input<RM, C>(0, q_g, NT, tid, V0, x, t, q);
  for (int l = 0; l < L; ++l) {
    const float *Uh = w_s + l * LS;
    const float *bh = Uh + RH * RM;
    const float *Vh = bh + RH;
    if (p.grad && l > 0) store_input<RM, C>(l, q_g, NT, tid, q);
    Jet<C, RM> y = q;
    jet_scale<RM, C>(y, s_s + l * RM);
    jet_zero<RM, C>(q);
    const int nr = p.rh[l];
    if (l == 0 && l == L - 1) layer_fwd<RM, C, R1, 1>(Uh, bh, Vh, nr, y, q);
    else if (l == 0) layer_fwd<RM, C, R1, RM>(Uh, bh, Vh, nr, y, q);
    else if (l == L - 1) layer_fwd<RM, C, RM, 1>(Uh, bh, Vh, nr, y, q);
    else layer_fwd<RM, C, RM, RM>(Uh, bh, Vh, nr, y, q);
  }
  const float sL = s_s[L * RM];
  float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < C; ++c) u[c] = Uout * sL * q.v[c][0].x;
  u[0] += bout;

  // ---- residual, loss and seeds (Eq. 4.1, Eq. 3.5 / 3.6)
  float ub[4], lp;
  if (!residual_and_seeds(p, T, pt, tid, u, ub, lp)) return;

  // ---- reverse sweep (backpropagation through the FastLRNR, Sec. 2.3)
  const int DB0 = partial_db0(L, RM);
  Jet<C, RM> qb;
  {
    const float ls = warp_sum(lp);
    float dsL = 0.0f;
    jet_zero<RM, C>(qb);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float pbv = Uout * ub[c];
      dsL += pbv * q.v[c][0].x;
      qb.v[c][0].x = sL * pbv;
    }
    const float s0 = warp_sum(dsL);
    const float s1 = warp_sum(ub[0]);
    if ((tid & 31) == 0) {
      red_w[0] += ls;
      red_w[1 + L * RM] += s0;
      red_w[DB0 + L * RH] += s1;
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const float *Uh = w_s + l * LS;
    const float *bh = Uh + RH * RM;
    const float *Vh = bh + RH;
    const float *sl = s_s + l * RM;
    const int nr = p.rh[l];
    {
      Jet<C, RM> y;
      load_input<RM, C>(l, q_g, NT, tid, V0, x, t, y);
      jet_scale<RM, C>(y, sl);
      if (l == 0 && l == L - 1) layer_bwd<RM, C, R1, 1>(Uh, bh, Vh, nr, y, qb, ab_s, NT);
      else if (l == 0) layer_bwd<RM, C, R1, RM>(Uh, bh, Vh, nr, y, qb, ab_s, NT);
      else if (l == L - 1) layer_bwd<RM, C, RM, 1>(Uh, bh, Vh, nr, y, qb, ab_s, NT);
      else layer_bwd<RM, C, RM, RM>(Uh, bh, Vh, nr, y, qb, ab_s, NT);
    }
    Jet<C, RM> pb;
    jet_zero<RM, C>(pb);
    if (l == 0) layer_bwd_pbar<RM, C, R1>(Uh, nr, ab_s, NT, pb);
    else layer_bwd_pbar<RM, C, RM>(Uh, nr, ab_s, NT, pb);
    // dL/ds^l = sum_c pbar_c * zhat_c (input jet, reloaded) and dL/dbhat^l rows
    float g[RM + RH];
#pragma unroll
    for (int h = 0; h < RM / 2; ++h) {
      float2 d = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float2 qv;
        if (l > 0) {
          qv = q_g[(((l - 1) * 4 + c) * (RM / 2) + h) * NT + tid];
        } else {
          qv = make_float2(0.0f, 0.0f);
          if (h == 0) {
            if (c == 0) qv = make_float2(V0[0] * x + V0[R1] * t, V0[1] * x + V0[R1 + 1] * t);
            else if (c == 1) qv = make_float2(V0[R1], V0[R1 + 1]);
            else if (c == 2) qv = make_float2(V0[0], V0[1]);
          }
        }
        d = f2fma(pb.v[c][h], qv, d);
      }
      g[2 * h] = d.x;
      g[2 * h + 1] = d.y;
    }
#pragma unroll
    for (int i = 0; i < RH; ++i) g[RM + i] = (i < nr) ? ab_s[i * NT + tid].x : 0.0f;
    warp_accumulate<RM + RH>(g, red_w, [&](int j) {
      return j < RM ? 1 + l * RM + j : DB0 + l * RH + (j - RM);
    });
    if (l > 0) {
      qb = pb;
      jet_scale<RM, C>(qb, sl);
    }
  }
}

// MINB: resident CTAs per SM the register allocation is built for (3: at most 168
// registers per thread; 2: up to 255 registers, no spills).
template <int RM, int RH, int MINB>
__global__ void __launch_bounds__(128, MINB) k_fast(const __grid_constant__ KParams p) {
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int L = p.L;
  const FastLayout lay(L, RM, RH, NT, p.P, p.fused_tiles ? p.n_inst : 0);
  float *w_s = smem + lay.pack;
  float *s_s = smem + lay.s;
  float4 *ab_s = reinterpret_cast<float4 *>(smem + lay.ab);
  float *red_s = smem + lay.red;
  float2 *q_g = reinterpret_cast<float2 *>(p.scratch + (size_t)blockIdx.x * fast_store_floats(L, RM, NT));
  const int npack = fast_pack_floats(L, RM, RH);
  for (int i = tid; i < npack; i += NT) w_s[i] = __ldg(p.pack + i);
  if (p.step && blockIdx.x == 0 && tid == 0) atomicAdd((unsigned long long *)p.step, 1ull);
  const int32_t *toff = p.tile_off;
  if (p.fused_tiles) {
    int32_t *toff_s = reinterpret_cast<int32_t *>(smem + lay.toff);
    block_tile_offsets(p, toff_s, reinterpret_cast<int32_t *>(smem + lay.scan));
    toff = toff_s;
  }
  const int ntiles = p.fused_tiles ? toff[p.n_inst] : __ldg(p.tile_off + p.n_inst);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile T = decode_tile(p, tile, toff);
    __syncthreads();
    for (int j = tid; j < (L + 1) * RM; j += NT) {
      const int l = j / RM, k = j % RM;
      s_s[j] = (k < p.r[l]) ? __ldg(p.s + (int64_t)T.inst * p.sum_r + p.roff[l] + k) : 0.0f;
    }
    if (p.grad)
      for (int j = tid; j < (NT / 32) * p.P; j += NT) red_s[j] = 0.0f;
    __syncthreads();
    float *red_w = red_s + (tid >> 5) * p.P;
    if (T.kind == KIND_INT)
      fast_tile<RM, RH, 4>(p, T, w_s, s_s, q_g, ab_s, red_w);
    else
      fast_tile<RM, RH, 1>(p, T, w_s, s_s, q_g, ab_s, red_w);
    if (p.grad) {
      __syncthreads();
      for (int j = tid; j < p.P; j += NT) {
        float acc = 0.0f;
        for (int w = 0; w < NT / 32; ++w) acc += red_s[w * p.P + j];
        if (j == 0 && !isfinite(acc)) set_status(p.status, DEV_NONFINITE);
        p.partial[(int64_t)tile * p.P + j] = acc;
      }
    }
  }
}

template <int RM, int RH, int MINB>
cudaError_t launch_fast_v(const KParams &p, int grid_cap, cudaStream_t st) {
  const int NT = p.nt;
  const FastLayout lay(p.L, RM, RH, NT, p.P, p.fused_tiles ? p.n_inst : 0);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_fast<RM, RH, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_fast<RM, RH, MINB><<<std::max(1, grid_cap), NT, bytes, st>>>(p);
  return cudaGetLastError();
}

template <int RM, int RH, int MINB>
int fast_ctas_per_sm_v(const KParams &p) {
  const FastLayout lay(p.L, RM, RH, p.nt, p.P, p.fused_tiles ? p.n_inst : 0);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  if (cudaFuncSetAttribute(k_fast<RM, RH, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fast<RM, RH, MINB>, p.nt, bytes) !=
      cudaSuccess)
    return 1;
  return std::max(1, per_sm);
}

// p.fast_regs selects the register budget: 3 -> the 168-register build (3 CTAs per
// SM, some spills), else the 255-register build (2 CTAs per SM).
template <int RM, int RH>
cudaError_t launch_fast_t(const KParams &p, int grid_cap, cudaStream_t st) {
  return p.fast_regs == 3 ? launch_fast_v<RM, RH, 3>(p, grid_cap, st)
                          : launch_fast_v<RM, RH, 2>(p, grid_cap, st);
}

template <int RM, int RH>
int fast_ctas_per_sm_t(const KParams &p) {
  return p.fast_regs == 3 ? fast_ctas_per_sm_v<RM, RH, 3>(p) : fast_ctas_per_sm_v<RM, RH, 2>(p);
}

}  // namespace lrnr
