// FastLRNR residual + adjoint, FP32 SIMT (kernel template) (Sec. 2.2 Eq. 2.8, Sec. 2.3).
//
// One thread per collocation point.  The reduced bases (Uhat, bhat, Vhat: a few KB
// per layer) and the tile's coefficients s live in shared memory and are read
// with warp-uniform (broadcast) loads; every per-point quantity -- the jet of the
// reduced state zhat (value, d/dt, d/dx, d2/dx2) and its adjoint -- stays in
// registers.  The forward stores each hidden layer's input jet in shared memory
// ([slot][thread], conflict free) so the reverse sweep can rebuild the layer's
// pre-activation without re-running the network.  Per-layer gradient pieces are
// summed over the warp by recursive halving and over the tile's warps in a fixed
// order, giving one partial row per tile.
#pragma once

#include <algorithm>

#include "lrnr_internal.cuh"
#include "point_common.cuh"
#include "simt_common.cuh"

namespace lrnr {

// Shared memory of one CTA (floats): the reduced bases, the tile's s, the stored
// layer inputs [(l-1)*4 + c][k][thread], the adjoint staging [c][i][thread] and
// one partial row per warp.
struct FastLayout {
  int pack, s, q, ab, red, total;
  __host__ __device__ FastLayout(int L, int RM, int RH, int NT, int P) {
    pack = 0;
    s = (fast_pack_floats(L, RM, RH) + 3) & ~3;
    q = s + (L + 1) * RM;
    ab = q + (L > 1 ? (L - 1) : 0) * 4 * RM * NT;
    red = ab + 4 * RH * NT;
    total = red + (NT / 32) * P;
  }
};

// The input jet of hidden layer l: stored by the forward (l > 0) or rebuilt from
// the point (l == 0: zhat^0 = V^0^T z^0).
template <int RM, int C>
__device__ __forceinline__ void load_input(int l, const float *__restrict__ q_s, int NT, int tid,
                                           const float *V0, float x, float t, float (&q)[C][RM]) {
  if (l > 0) {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) q[c][k] = q_s[(((l - 1) * 4 + c) * RM + k) * NT + tid];
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) q[c][k] = 0.0f;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      q[0][k] = V0[k] * x + V0[R1 + k] * t;
      if constexpr (C >= 3) {
        q[1][k] = V0[R1 + k];
        q[2][k] = V0[k];
      }
    }
  }
}

// out[c] += W[0..NI) . v[c][0..NI)
template <int RM, int NI, int C>
__device__ __forceinline__ void row_dot(const float *__restrict__ W, const float (&v)[C][RM],
                                        float (&out)[C][1]) {
  if constexpr (NI % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NI; k += 4) {
      const float4 w = *reinterpret_cast<const float4 *>(W + k);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        out[c][0] = fmaf(w.x, v[c][k], out[c][0]);
        out[c][0] = fmaf(w.y, v[c][k + 1], out[c][0]);
        out[c][0] = fmaf(w.z, v[c][k + 2], out[c][0]);
        out[c][0] = fmaf(w.w, v[c][k + 3], out[c][0]);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NI; ++k)
#pragma unroll
      for (int c = 0; c < C; ++c) out[c][0] = fmaf(W[k], v[c][k], out[c][0]);
  }
}

// acc[c][0..NI) += W[0..NI) * v[c]
template <int RM, int NI, int C>
__device__ __forceinline__ void row_axpy(const float *__restrict__ W, const float (&v)[C][1],
                                         float (&acc)[C][RM]) {
  if constexpr (NI % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NI; k += 4) {
      const float4 w = *reinterpret_cast<const float4 *>(W + k);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        acc[c][k] = fmaf(w.x, v[c][0], acc[c][k]);
        acc[c][k + 1] = fmaf(w.y, v[c][0], acc[c][k + 1]);
        acc[c][k + 2] = fmaf(w.z, v[c][0], acc[c][k + 2]);
        acc[c][k + 3] = fmaf(w.w, v[c][0], acc[c][k + 3]);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NI; ++k)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c][k] = fmaf(W[k], v[c][0], acc[c][k]);
  }
}

template <int RM, int RH, int C>
__device__ void fast_tile(const KParams &p, const Tile &T, const float *__restrict__ w_s,
                          const float *__restrict__ s_s, float *__restrict__ q_s,
                          float *__restrict__ ab_s, float *red_w) {
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int L = p.L;
  const int LS = fast_layer_floats(RM, RH);
  const float *V0 = w_s + L * LS;
  const float Uout = w_s[L * LS + 2 * R1];
  const float bout = w_s[L * LS + 2 * R1 + 1];

  // ---- the point
  const PointIn pt = load_point(p, T, tid);
  const float x = pt.x, t = pt.t;

  // ---- forward: zhat^0 = V^0^T z^0, then the reduced layers (Eq. 2.8)
  float q[C][RM];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int k = 0; k < RM; ++k) q[c][k] = 0.0f;
#pragma unroll
  for (int k = 0; k < R1; ++k) {
    q[0][k] = V0[k] * x + V0[R1 + k] * t;
    if constexpr (C >= 3) {
      q[1][k] = V0[R1 + k];
      q[2][k] = V0[k];
    }
  }

  for (int l = 0; l < L; ++l) {
    const float *Uh = w_s + l * LS;
    const float *bh = Uh + RH * RM;
    const float *Vh = bh + RH;
    const float *sl = s_s + l * RM;
    if (p.grad && l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < RM; ++k) q_s[(((l - 1) * 4 + c) * RM + k) * NT + tid] = q[c][k];
    }
    float a[C][RH];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int i = 0; i < RH; ++i) a[c][i] = (c == 0) ? bh[i] : 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) q[c][k] *= sl[k];
    if (l == 0) mv_rows<RM, R1, RH, C>(Uh, q, a);
    else mv_rows<RM, RM, RH, C>(Uh, q, a);
    act_fwd<C, RH>(a);
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) q[c][k] = 0.0f;
    if (l == L - 1) mv_cols<RM, RH, 1, C, RH>(Vh, a, q);
    else mv_cols<RM, RH, RM, C, RH>(Vh, a, q);
  }
  const float sL = s_s[L * RM];
  float u[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) u[c] = 0.0f;
#pragma unroll
  for (int c = 0; c < C; ++c) u[c] = Uout * sL * q[c][0];
  u[0] += bout;

  // ---- residual, loss and seeds (Eq. 4.1, Eq. 3.5 / 3.6)
  float ub[4], lp;
  if (!residual_and_seeds(p, T, pt, tid, u, ub, lp)) return;

  // ---- reverse sweep (backpropagation through the FastLRNR, Sec. 2.3)
  const int DB0 = partial_db0(L, RM);
  {
    const float ls = warp_sum(lp);
    if ((tid & 31) == 0) red_w[0] += ls;
  }
  float qb[C][RM];
  {
    float dsL = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float pb = Uout * ub[c];
      dsL += pb * q[c][0];
#pragma unroll
      for (int k = 0; k < RM; ++k) qb[c][k] = 0.0f;
      qb[c][0] = sL * pb;
    }
    float v2[2] = {dsL, ub[0]};
    const float s0 = warp_sum(v2[0]);
    const float s1 = warp_sum(v2[1]);
    if ((tid & 31) == 0) {
      red_w[1 + L * RM] += s0;
      red_w[DB0 + L * RH] += s1;
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const float *Uh = w_s + l * LS;
    const float *bh = Uh + RH * RM;
    const float *Vh = bh + RH;
    const float *sl = s_s + l * RM;
    // y = s * (the layer's input jet)
    float y[C][RM];
    load_input<RM, C>(l, q_s, NT, tid, V0, x, t, y);
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) y[c][k] *= sl[k];
    // row by row: rebuild the pre-activation, pull back the output adjoint
    // wb = Vhat qb through tanh, stage abar in shared memory
    float g[RM + RH];
#pragma unroll
    for (int i = 0; i < RH; ++i) {
      float a[C][1], wb[C][1];
#pragma unroll
      for (int c = 0; c < C; ++c) { a[c][0] = (c == 0) ? bh[i] : 0.0f; wb[c][0] = 0.0f; }
      if (l == 0) row_dot<RM, R1, C>(Uh + i * RM, y, a);
      else row_dot<RM, RM, C>(Uh + i * RM, y, a);
      if (l == L - 1) row_dot<RM, 1, C>(Vh + i * RM, qb, wb);
      else row_dot<RM, RM, C>(Vh + i * RM, qb, wb);
      act_bwd<C, 1>(a, wb);
#pragma unroll
      for (int c = 0; c < C; ++c) ab_s[(c * RH + i) * NT + tid] = wb[c][0];
      g[RM + i] = wb[0][0];
    }
    // pbar = Uhat^T abar
    float pb[C][RM];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) pb[c][k] = 0.0f;
#pragma unroll
    for (int i = 0; i < RH; ++i) {
      float ab[C][1];
#pragma unroll
      for (int c = 0; c < C; ++c) ab[c][0] = ab_s[(c * RH + i) * NT + tid];
      if (l == 0) row_axpy<RM, R1, C>(Uh + i * RM, ab, pb);
      else row_axpy<RM, RM, C>(Uh + i * RM, ab, pb);
    }
    // dL/ds^l = sum_c pbar_c * q_c
    load_input<RM, C>(l, q_s, NT, tid, V0, x, t, y);
#pragma unroll
    for (int k = 0; k < RM; ++k) {
      float d = 0.0f;
#pragma unroll
      for (int c = 0; c < C; ++c) d = fmaf(pb[c][k], y[c][k], d);
      g[k] = d;
    }
    warp_accumulate<RM + RH>(g, red_w, [&](int j) {
      return j < RM ? 1 + l * RM + j : DB0 + l * RH + (j - RM);
    });
    if (l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < RM; ++k) qb[c][k] = pb[c][k] * sl[k];
    }
  }
}

template <int RM, int RH>
__global__ void __launch_bounds__(128) k_fast(const __grid_constant__ KParams p) {
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int L = p.L;
  const FastLayout lay(L, RM, RH, NT, p.P);
  float *w_s = smem + lay.pack;
  float *s_s = smem + lay.s;
  float *q_s = smem + lay.q;
  float *ab_s = smem + lay.ab;
  float *red_s = smem + lay.red;
  const int npack = fast_pack_floats(L, RM, RH);
  for (int i = tid; i < npack; i += NT) w_s[i] = __ldg(p.pack + i);
  if (p.step && blockIdx.x == 0 && tid == 0) atomicAdd((unsigned long long *)p.step, 1ull);
  const int ntiles = __ldg(p.tile_off + p.n_inst);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile T = decode_tile(p, tile);
    __syncthreads();
    for (int j = tid; j < (L + 1) * RM; j += NT) {
      const int l = j / RM, k = j % RM;
      s_s[j] = (k < p.r[l]) ? __ldg(p.s + (int64_t)T.inst * p.sum_r + p.roff[l] + k) : 0.0f;
    }
    if (p.grad)
      for (int j = tid; j < (NT / 32) * p.P; j += NT) red_s[j] = 0.0f;
    __syncthreads();
    float *red_w = red_s + (tid >> 5) * p.P;
    if (T.kind == KIND_INT) {
      if (p.grad && __ldg(p.nu + T.inst) == 0.0f)
        fast_tile<RM, RH, 3>(p, T, w_s, s_s, q_s, ab_s, red_w);
      else
        fast_tile<RM, RH, 4>(p, T, w_s, s_s, q_s, ab_s, red_w);
    } else {
      fast_tile<RM, RH, 1>(p, T, w_s, s_s, q_s, ab_s, red_w);
    }
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

template <int RM, int RH>
cudaError_t launch_fast_t(const KParams &p, int grid_cap, cudaStream_t st) {
  const int NT = p.nt;
  const FastLayout lay(p.L, RM, RH, NT, p.P);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_fast<RM, RH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fast<RM, RH>, NT, bytes);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(grid_cap, std::max(1, per_sm) * sms));
  k_fast<RM, RH><<<grid, NT, bytes, st>>>(p);
  return cudaGetLastError();
}

}  // namespace lrnr
