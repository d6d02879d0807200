// FastLRNR residual + adjoint, FP32 SIMT (kernel template) (Sec. 2.2 Eq. 2.8, Sec. 2.3).
//
// One thread per collocation point.  The reduced bases (Uhat, bhat, Vhat: a few KB
// per layer) and the tile's coefficients s live in shared memory and are read
// with warp-uniform (broadcast) loads.  Each layer streams over its rhat rows in
// blocks of four: for row i the thread forms the pre-activation jet
// a_i = Uhat_i . (s * zhat) (+ bhat_i) (four scalars, one per jet channel), pushes it
// through tanh and accumulates the next rank-r jet zhat' += Vhat_i w_i; the reverse
// sweep does the same per row for the adjoint.  Rank-r vectors are held as pairs of adjacent entries so that the
// products run on the packed two-lane FP32 FMA (two multiply-adds per instruction;
// each lane rounds exactly like a scalar fmaf).  Only the four rows of a block are
// unrolled, which keeps the kernel small enough for the instruction cache.  The forward keeps each
// hidden layer's input jet in a per-CTA global scratch area ([slot][thread],
// coalesced, L2-resident) so the reverse sweep can rebuild pre-activations without
// re-running the network.  Per-layer gradient pieces are summed over the warp and
// over the tile's warps in a fixed order, giving one partial row per tile.
#pragma once

#include <algorithm>

#include "lrnr_internal.cuh"
#include "point_common.cuh"
#include "simt_common.cuh"
#include "fused_reduce.cuh"

namespace lrnr {

// Shared memory of one CTA (floats): the reduced bases, the tile's s, the tile's
// scaled input bases Uhat diag(s^l) per layer, the staged pre-activation adjoints
// of the current layer [row][thread] (float4: the four channels), the staging
// buffer of the next reverse layer's input jet [channel][quad][thread] (float4), one
// partial row per warp and, when the kernel computes the tile schedule, the tile
// offsets.
struct FastLayout {
  int pack, s, us, ab, qb, red, toff, scan, misc, total;
  __host__ __device__ FastLayout(int L, int RM, int RH, int NT, int P, int fused_inst = 0) {
    pack = 0;
    s = (fast_pack_floats(L, RM, RH) + 3) & ~3;
    us = (s + (L + 1) * RM + 3) & ~3;
    ab = us + L * RH * RM;
    qb = ab + 4 * RH * NT;
    red = qb + 4 * RM * NT;
    toff = red + (NT / 32) * P;
    scan = toff + (fused_inst ? fused_inst + 1 : 0);
    misc = scan + (fused_inst ? NT : 0);   // per-warp sums and a flag of the fused reduction
    total = misc + NT / 32 + 4;
  }
};

// Largest instance count for which the FastLRNR kernel computes its own tile offsets.
constexpr int kFastFusedInstMax = 4096;

// Floats of the per-CTA global scratch of the gradient sweep: the layer-input store
// ((L-1) layers x 4 channels x RM x NT) followed by the activation store (L layers x
// RH rows x NT float4: tanh value and the three pre-activation derivative channels).
__host__ __device__ inline size_t fast_input_store_floats(int L, int RM, int NT) {
  return (size_t)(L > 1 ? L - 1 : 1) * 4 * RM * NT;
}
__host__ __device__ inline size_t fast_store_floats(int L, int RM, int RH, int NT) {
  return fast_input_store_floats(L, RM, NT) + (size_t)L * RH * 4 * NT;
}

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

// Rank-r jet of C channels, RM entries each, held as RM/2 pairs.
template <int C, int RM>
struct Jet {
  float2 v[C][RM / 2];
};

// The input jet of the first hidden layer, zhat^0 = V^0^T z^0 with z^0 = (x, t)
// and its derivative channels.
template <int RM, int C>
__device__ __forceinline__ void input_jet(const float *V0, float x, float t, Jet<C, RM> &q) {
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

// Layer-input store of the forward (hidden layer l > 0), per CTA in global memory:
// [l-1][channel][quad][thread] float4, four rank entries per float4.
template <int RM, int C>
__device__ __forceinline__ void store_input(int l, float4 *__restrict__ q_g, int NT, int tid,
                                            const Jet<C, RM> &q) {
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int h = 0; h < RM / 4; ++h)
      q_g[(((l - 1) * 4 + c) * (RM / 4) + h) * NT + tid] =
          make_float4(q.v[c][2 * h].x, q.v[c][2 * h].y, q.v[c][2 * h + 1].x, q.v[c][2 * h + 1].y);
}

// Start copying the thread's stored input jet of layer l into the staging buffer
// (cp.async, L2 -> shared memory without registers); each thread copies and later
// reads only its own entries.
template <int RM, int C>
__device__ __forceinline__ void prefetch_input(int l, const float4 *__restrict__ q_g, float4 *q_b,
                                               int NT, int tid) {
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int h = 0; h < RM / 4; ++h) {
      const float4 *src = q_g + (((l - 1) * 4 + c) * (RM / 4) + h) * NT + tid;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(q_b + (c * (RM / 4) + h) * NT + tid);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Wait for the thread's copies and read the staged jet.
template <int RM, int C>
__device__ __forceinline__ void load_staged(const float4 *q_b, int NT, int tid, Jet<C, RM> &q) {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int h = 0; h < RM / 4; ++h) {
      const float4 v = q_b[(c * (RM / 4) + h) * NT + tid];
      q.v[c][2 * h] = make_float2(v.x, v.y);
      q.v[c][2 * h + 1] = make_float2(v.z, v.w);
    }
}

// Rows are processed in blocks of RB: one block's dot products are RB * C
// independent accumulation chains and its tanh jets RB independent chains, which
// the scheduler interleaves (at two warps per scheduler a single row's dependent
// chain would leave the FMA pipe idle).  Rows past rhat are zero in the pack, so a
// block may run past the last selected row: its pre-activation is zero and its
// outgoing weights are zero.
constexpr int RB = 4;

// out[r][c] += W_r[0..NI) . v[c][0..NI) for the RB rows W_r = W + r * RM, each
// accumulated as even/odd partial sums.
template <int RM, int NI, int C>
__device__ __forceinline__ void block_dot(const float *__restrict__ W, const Jet<C, RM> &v,
                                          float (&out)[RB][C]) {
  if constexpr (NI == 1) {
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) out[r][c] = fmaf(W[r * RM], v.v[c][0].x, out[r][c]);
  } else {
    static_assert(NI == 2 || NI % 4 == 0, "input rank");
    float2 acc[RB][C];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[r][c] = make_float2(out[r][c], 0.0f);
    if constexpr (NI == 2) {
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const float2 w = *reinterpret_cast<const float2 *>(W + r * RM);
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = f2fma(w, v.v[c][0], acc[r][c]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NI; k += 4) {
        float4 w[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) w[r] = *reinterpret_cast<const float4 *>(W + r * RM + k);
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int c = 0; c < C; ++c)
            acc[r][c] = f2fma(make_float2(w[r].x, w[r].y), v.v[c][k / 2], acc[r][c]);
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int c = 0; c < C; ++c)
            acc[r][c] = f2fma(make_float2(w[r].z, w[r].w), v.v[c][k / 2 + 1], acc[r][c]);
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) out[r][c] = acc[r][c].x + acc[r][c].y;
  }
}

// acc[c][0..NO) += sum over the RB rows (in row order) of W_r[0..NO) * z[r][c].
template <int RM, int NO, int C>
__device__ __forceinline__ void block_axpy(const float *__restrict__ W, const float (&z)[RB][C],
                                           Jet<C, RM> &acc) {
  if constexpr (NO == 1) {
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) acc.v[c][0].x = fmaf(W[r * RM], z[r][c], acc.v[c][0].x);
  } else if constexpr (NO == 2) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const float2 w = *reinterpret_cast<const float2 *>(W + r * RM);
#pragma unroll
      for (int c = 0; c < C; ++c) acc.v[c][0] = f2fma(w, splat(z[r][c]), acc.v[c][0]);
    }
  } else {
    static_assert(NO % 4 == 0, "output rank");
#pragma unroll
    for (int k = 0; k < NO; k += 4) {
      float4 w[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) w[r] = *reinterpret_cast<const float4 *>(W + r * RM + k);
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float2 zz = splat(z[r][c]);
          acc.v[c][k / 2] = f2fma(make_float2(w[r].x, w[r].y), zz, acc.v[c][k / 2]);
          acc.v[c][k / 2 + 1] = f2fma(make_float2(w[r].z, w[r].w), zz, acc.v[c][k / 2 + 1]);
        }
    }
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

// tanh jet of one row, in place: a = (a0, a_t, a_x, a_xx) -> (z, z_t, z_x, z_xx); `keep`
// receives what the adjoint needs: (z, a_t, a_x, a_xx).
template <int C>
__device__ __forceinline__ void jet_fwd(float (&a)[C], float4 &keep) {
  float z, d1, d2;
  tanh_d(a[0], z, d1, d2);
  keep = make_float4(z, 0.0f, 0.0f, 0.0f);
  if constexpr (C == 4) keep = make_float4(z, a[1], a[2], a[3]);
  if constexpr (C == 4) a[3] = d2 * a[2] * a[2] + d1 * a[3];
  if constexpr (C >= 3) {
    a[1] *= d1;
    a[2] *= d1;
  }
  a[0] = z;
}

// Adjoint of jet_fwd from its kept values k = (z, a_t, a_x, a_xx) and the output
// adjoint wb: overwrite wb with the pre-activation adjoint.
template <int C>
__device__ __forceinline__ void jet_bwd(const float4 &k, float (&wb)[C]) {
  static_assert(C == 1 || C == 4, "jet channels");
  const float z = k.x;
  const float d1 = 1.0f - z * z;
  float ab0 = wb[0] * d1;
  if constexpr (C == 4) {
    const float d2 = -2.0f * z * d1;
    const float d3 = d1 * (6.0f * z * z - 2.0f);
    ab0 += d2 * (wb[1] * k.y + wb[2] * k.z);
    ab0 += wb[3] * (d3 * k.z * k.z + d2 * k.w);
    wb[2] = wb[2] * d1 + 2.0f * wb[3] * d2 * k.z;
    wb[3] = wb[3] * d1;
    wb[1] = wb[1] * d1;
  }
  wb[0] = ab0;
}

// One reduced layer forward: q (input jet; the bases are pre-scaled by s) -> qn
// (next rank-r jet).  With a_g, each row's kept values go to the activation store
// a_g[row][thread].
template <int RM, int C, int NI, int NO>
__device__ __forceinline__ void layer_fwd(const float *__restrict__ Us, const float *__restrict__ bh,
                                          const float *__restrict__ Vh, int nrows,
                                          const Jet<C, RM> &y, Jet<C, RM> &qn,
                                          float4 *__restrict__ a_g, int NT) {
#pragma unroll 1
  for (int i = 0; i < nrows; i += RB) {
    float a[RB][C];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      a[r][0] = bh[i + r];
#pragma unroll
      for (int c = 1; c < C; ++c) a[r][c] = 0.0f;
    }
    block_dot<RM, NI, C>(Us + i * RM, y, a);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      float4 keep;
      jet_fwd<C>(a[r], keep);
      if (a_g) a_g[(i + r) * NT + threadIdx.x] = keep;
    }
    block_axpy<RM, NO, C>(Vh + i * RM, a, qn);
  }
}

// One reduced layer reverse, in two passes over the rows so that no more than two
// rank-r jets are live at once:
//   pass 1: pull wb_i = Vhat_i . qb back through the tanh jet using the values the
//           forward kept (read one block ahead), stage abar_i (all channels) in
//           ab_s[row][thread];
//   pass 2: pb = Uhat^T abar from the staged rows.
template <int RM, int C, int NO>
__device__ __forceinline__ void layer_bwd(const float *__restrict__ Vh, int nrows,
                                          const float4 *__restrict__ a_g, const Jet<C, RM> &qb,
                                          float4 *ab_s, int NT) {
#pragma unroll 1
  for (int i = 0; i < nrows; i += RB) {
    float4 cur[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) cur[r] = a_g[(i + r) * NT + threadIdx.x];
    float wb[RB][C];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) wb[r][c] = 0.0f;
    block_dot<RM, NO, C>(Vh + i * RM, qb, wb);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      jet_bwd<C>(cur[r], wb[r]);
      float4 v = make_float4(wb[r][0], 0.0f, 0.0f, 0.0f);
      if constexpr (C == 4) v = make_float4(wb[r][0], wb[r][1], wb[r][2], wb[r][3]);
      ab_s[(i + r) * NT + threadIdx.x] = v;
    }
  }
}

template <int RM, int C, int NI>
__device__ __forceinline__ void layer_bwd_pbar(const float *__restrict__ Uh, int nrows,
                                               const float4 *ab_s, int NT, Jet<C, RM> &pb) {
#pragma unroll 1
  for (int i = 0; i < nrows; i += RB) {
    float ab[RB][C];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const float4 v = ab_s[(i + r) * NT + threadIdx.x];
      ab[r][0] = v.x;
      if constexpr (C == 4) { ab[r][1] = v.y; ab[r][2] = v.z; ab[r][3] = v.w; }
    }
    block_axpy<RM, NI, C>(Uh + i * RM, ab, pb);
  }
}

template <int RM, int RH, int C>
__device__ void fast_tile(const KParams &p, const Tile &T, const float *__restrict__ w_s,
                          const float *__restrict__ us_s, const float *__restrict__ s_s,
                          float4 *__restrict__ q_g, float4 *__restrict__ a_g, float4 *q_b,
                          float4 *ab_s, float *red_w) {
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int L = p.L;
  const int LS = fast_layer_floats(RM, RH);
  const float *V0 = w_s + L * LS;
  const float Uout = w_s[L * LS + 2 * R1];
  const float bout = w_s[L * LS + 2 * R1 + 1];

  const PointIn pt = load_point(p, T, tid);
  const float x = pt.x, t = pt.t;

  // ---- forward: zhat^0 = V^0^T z^0, then the reduced layers (Eq. 2.8) with the
  // tile's scaled bases Uhat diag(s^l)
  Jet<C, RM> q;
  input_jet<RM, C>(V0, x, t, q);
  for (int l = 0; l < L; ++l) {
    const float *Us = us_s + l * RH * RM;
    const float *bh = w_s + l * LS + RH * RM;
    const float *Vh = bh + RH;
    if (p.grad && l > 0) store_input<RM, C>(l, q_g, NT, tid, q);
    Jet<C, RM> qn;
    jet_zero<RM, C>(qn);
    const int nr = p.rh[l];
    float4 *al = p.grad ? a_g + (size_t)l * RH * NT : nullptr;
    if (l == 0 && l == L - 1) layer_fwd<RM, C, R1, 1>(Us, bh, Vh, nr, q, qn, al, NT);
    else if (l == 0) layer_fwd<RM, C, R1, RM>(Us, bh, Vh, nr, q, qn, al, NT);
    else if (l == L - 1) layer_fwd<RM, C, RM, 1>(Us, bh, Vh, nr, q, qn, al, NT);
    else layer_fwd<RM, C, RM, RM>(Us, bh, Vh, nr, q, qn, al, NT);
    q = qn;
  }
  const float sL = s_s[L * RM];
  float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < C; ++c) u[c] = Uout * sL * q.v[c][0].x;
  u[0] += bout;

  // ---- residual, loss and seeds (Eq. 4.1, Eq. 3.5 / 3.6)
  float ub[4], lp;
  if (!residual_and_seeds(p, T, pt, tid, u, ub, lp)) return;
  if (L > 1) prefetch_input<RM, C>(L - 1, q_g, q_b, NT, tid);

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
    const float *Vh = Uh + RH * RM + RH;
    const float *sl = s_s + l * RM;
    const int nr = p.rh[l];
    const float4 *al = a_g + (size_t)l * RH * NT;
    if (l == L - 1) layer_bwd<RM, C, 1>(Vh, nr, al, qb, ab_s, NT);
    else layer_bwd<RM, C, RM>(Vh, nr, al, qb, ab_s, NT);
    Jet<C, RM> pb;
    jet_zero<RM, C>(pb);
    if (l == 0) layer_bwd_pbar<RM, C, R1>(Uh, nr, ab_s, NT, pb);
    else layer_bwd_pbar<RM, C, RM>(Uh, nr, ab_s, NT, pb);
    // the layer's input jet (unscaled), read only now so that it is not live through
    // the two passes (no spills at 255 registers); then the next layer's input jet
    // is prefetched into the staging buffer
    Jet<C, RM> y;
    if (l > 0) {
      load_staged<RM, C>(q_b, NT, tid, y);
      if (l > 1) prefetch_input<RM, C>(l - 1, q_g, q_b, NT, tid);
    } else {
      input_jet<RM, C>(V0, x, t, y);
    }
    // dL/ds^l = sum_c pbar_c * zhat_c and the dL/dbhat^l rows
    float g[RM + RH];
#pragma unroll
    for (int h = 0; h < RM / 2; ++h) {
      float2 d = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int c = 0; c < C; ++c) d = f2fma(pb.v[c][h], y.v[c][h], d);
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
// FR: the variant with the fixed-order reduction (and Adam) inside the kernel; a
// separate instantiation, so that the kernel for large batches carries none of it.
template <int RM, int RH, int MINB, bool FR>
__global__ void __launch_bounds__(128, MINB) k_fast(const __grid_constant__ KParams p) {
  static_assert(RH % RB == 0, "row blocks");
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int L = p.L;
  const FastLayout lay(L, RM, RH, NT, p.P, p.fused_tiles ? p.n_inst : 0);
  float *w_s = smem + lay.pack;
  float *s_s = smem + lay.s;
  float *us_s = smem + lay.us;
  float4 *ab_s = reinterpret_cast<float4 *>(smem + lay.ab);
  float4 *q_b = reinterpret_cast<float4 *>(smem + lay.qb);
  float *red_s = smem + lay.red;
  float *store = p.scratch + (size_t)blockIdx.x * fast_store_floats(L, RM, RH, NT);
  float4 *q_g = reinterpret_cast<float4 *>(store);
  float4 *a_g = reinterpret_cast<float4 *>(store + fast_input_store_floats(L, RM, NT));
  const int npack = fast_pack_floats(L, RM, RH);
  for (int i = tid; i < npack; i += NT) w_s[i] = __ldg(p.pack + i);
  // Adam step number: the fused reduction reads the counter here and advances it
  // once every instance is done; otherwise block 0 advances it for the next kernel
  if (!FR && p.step && blockIdx.x == 0 && tid == 0) atomicAdd((unsigned long long *)p.step, 1ull);
  const int64_t kstep = (FR && p.step) ? *p.step + 1 : 0;
  float *wsum = smem + lay.misc;
  int *flag = reinterpret_cast<int *>(smem + lay.misc + NT / 32);
  const int32_t *toff = p.tile_off;
  if (p.fused_tiles) {
    int32_t *toff_s = reinterpret_cast<int32_t *>(smem + lay.toff);
    block_tile_offsets(p, toff_s, reinterpret_cast<int32_t *>(smem + lay.scan));
    toff = toff_s;
  }
  const int ntiles = p.fused_tiles ? toff[p.n_inst] : __ldg(p.tile_off + p.n_inst);
  if constexpr (FR) {
    // instances without points have no tile: finish them here
    for (int i = blockIdx.x; i < p.n_inst; i += gridDim.x)
      if (toff[i] == toff[i + 1]) fast_finish_instance(p, i, toff, red_s, wsum, kstep);
  }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // the CTA's last tile: the kernel that reduces the partial rows may be scheduled
    // now (it waits on the device for this grid to complete)
    if (tile + (int)gridDim.x >= ntiles) asm volatile("griddepcontrol.launch_dependents;");
    const Tile T = decode_tile(p, tile, toff);
    __syncthreads();
    for (int j = tid; j < (L + 1) * RM; j += NT) {
      const int l = j / RM, k = j % RM;
      s_s[j] = (k < p.r[l]) ? __ldg(p.s + (int64_t)T.inst * p.sum_r + p.roff[l] + k) : 0.0f;
    }
    if (p.grad)
      for (int j = tid; j < (NT / 32) * p.P; j += NT) red_s[j] = 0.0f;
    __syncthreads();
    {
      const int LS = fast_layer_floats(RM, RH);
      for (int j = tid; j < L * RH * RM; j += NT) {
        const int l = j / (RH * RM), ik = j % (RH * RM);
        us_s[j] = w_s[l * LS + ik] * s_s[l * RM + ik % RM];
      }
    }
    __syncthreads();
    float *red_w = red_s + (tid >> 5) * p.P;
    if (T.kind == KIND_INT)
      fast_tile<RM, RH, 4>(p, T, w_s, us_s, s_s, q_g, a_g, q_b, ab_s, red_w);
    else
      fast_tile<RM, RH, 1>(p, T, w_s, us_s, s_s, q_g, a_g, q_b, ab_s, red_w);
    if (p.grad) {
      __syncthreads();
      for (int j = tid; j < p.P; j += NT) {
        float acc = 0.0f;
        for (int w = 0; w < NT / 32; ++w) acc += red_s[w * p.P + j];
        if (j == 0 && !isfinite(acc)) set_status(p.status, DEV_NONFINITE);
        p.partial[(int64_t)tile * p.P + j] = acc;
      }
      // every read of the layer stores is behind the barrier above
      l2_discard(store, fast_store_floats(L, RM, RH, NT) * sizeof(float));
      if constexpr (FR) fast_tile_done(p, tile, ntiles, toff, red_s, wsum, flag, kstep);
    }
  }
}

template <int RM, int RH, int MINB, bool FR>
cudaError_t launch_fast_v(const KParams &p, int grid_cap, cudaStream_t st) {
  const int NT = p.nt;
  const FastLayout lay(p.L, RM, RH, NT, p.P, p.fused_tiles ? p.n_inst : 0);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_fast<RM, RH, MINB, FR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_fast<RM, RH, MINB, FR><<<std::max(1, grid_cap), NT, bytes, st>>>(p);
  return cudaGetLastError();
}

template <int RM, int RH, int MINB>
int fast_ctas_per_sm_v(const KParams &p) {
  const FastLayout lay(p.L, RM, RH, p.nt, p.P, p.fused_tiles ? p.n_inst : 0);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  if (cudaFuncSetAttribute(k_fast<RM, RH, MINB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fast<RM, RH, MINB, false>, p.nt, bytes) !=
      cudaSuccess)
    return 1;
  return std::max(1, per_sm);
}

// p.fast_regs selects the register budget: 3 -> the 168-register build (3 CTAs per
// SM, some spills), else the 255-register build (2 CTAs per SM).
template <int RM, int RH>
cudaError_t launch_fast_t(const KParams &p, int grid_cap, cudaStream_t st) {
  if (p.fused_red) return launch_fast_v<RM, RH, 2, true>(p, grid_cap, st);
  return p.fast_regs == 3 ? launch_fast_v<RM, RH, 3, false>(p, grid_cap, st)
                          : launch_fast_v<RM, RH, 2, false>(p, grid_cap, st);
}

template <int RM, int RH>
int fast_ctas_per_sm_t(const KParams &p) {
  return p.fast_regs == 3 ? fast_ctas_per_sm_v<RM, RH, 3>(p) : fast_ctas_per_sm_v<RM, RH, 2>(p);
}

}  // namespace lrnr
