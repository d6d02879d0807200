// Full-width LRNR residual + adjoint, FP32 SIMT (Sec. 2.1 Eq. 2.1-2.2, Sec. 2.3).
//
// The plain FP32 path: one thread per collocation point, the M-wide hidden state
// is never materialised.  A layer walks its M rows; for row i it forms the
// pre-activation jet a_i = U_i . (s * q) (+ b_i), pushes it through tanh and
// accumulates the next layer's rank-r input q' += V'_i z_i.  Bases are read from
// global memory with warp-uniform addresses (one L1 broadcast per warp).  The
// reverse sweep rebuilds each row's pre-activation from the stored rank-r input
// (C x r floats per point per layer) instead of keeping M-wide activations.
#include "lrnr_internal.cuh"
#include "point_common.cuh"
#include "simt_common.cuh"

#include <algorithm>

namespace lrnr {
namespace {

// Shared memory (floats): the tile's s and one partial row per warp.  The rank-r
// layer inputs are kept in a per-CTA global scratch area ([slot][thread], L2-resident).
template <int RM, int NT>
struct FullLayout {
  int s, red, total;
  __host__ __device__ FullLayout(int L, int P) {
    s = 0;
    red = s + (L + 1) * RM;
    total = red + (NT / 32) * P;
  }
};

__host__ __device__ inline size_t full_store_floats(int L, int RM, int NT) {
  return (size_t)(L > 1 ? L - 1 : 1) * 4 * RM * NT;
}

// Rank-r jets are held as RM/2 pairs per channel so that the products run on the
// packed FP32 FMA (two lanes of arithmetic per instruction).
__device__ __forceinline__ float2 ff2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fm2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Row W[0..N) as pairs (N a multiple of 4, or 2, or 1; nothing past N is read).
template <int RM, int N>
__device__ __forceinline__ void load_row2(const float *__restrict__ W, float2 (&w)[RM / 2]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int k = 0; k < N; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(W + k));
      w[k / 2] = make_float2(v.x, v.y);
      w[k / 2 + 1] = make_float2(v.z, v.w);
    }
  } else if constexpr (N == 2) {
    w[0] = __ldg(reinterpret_cast<const float2 *>(W));
  } else {
    w[0] = make_float2(__ldg(W), 0.0f);
  }
}

// One hidden layer forward: y = s * q (input jet) -> qn (next rank-r input).  Per row
// the pre-activation is an even/odd pair of partial dot products added at the end.
template <int RM, int NI, int NO, int C>
__device__ __forceinline__ void layer_fwd(const float *__restrict__ U, const float *__restrict__ b,
                                          const float *__restrict__ Vn, int M,
                                          const float2 (&y)[C][RM / 2], float2 (&qn)[C][RM / 2]) {
  static_assert(NI % 2 == 0, "input rank is padded to pairs");
#pragma unroll 2
  for (int i = 0; i < M; ++i) {
    float2 uw[RM / 2], vw[RM / 2];
    load_row2<RM, NI>(U + (int64_t)i * RM, uw);
    load_row2<RM, NO>(Vn + (int64_t)i * RM, vw);
    float2 acc[C];
    acc[0] = make_float2(__ldg(b + i), 0.0f);
#pragma unroll
    for (int c = 1; c < C; ++c) acc[c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int kk = 0; kk < NI / 2; ++kk)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = ff2(uw[kk], y[c][kk], acc[c]);
    float a[C][1];
#pragma unroll
    for (int c = 0; c < C; ++c) a[c][0] = acc[c].x + acc[c].y;
    act_fwd<C, 1>(a);
    if constexpr (NO == 1) {
#pragma unroll
      for (int c = 0; c < C; ++c) qn[c][0].x = fmaf(vw[0].x, a[c][0], qn[c][0].x);
    } else {
#pragma unroll
      for (int jj = 0; jj < NO / 2; ++jj)
#pragma unroll
        for (int c = 0; c < C; ++c) qn[c][jj] = ff2(vw[jj], make_float2(a[c][0], a[c][0]), qn[c][jj]);
    }
  }
}

// One hidden layer reverse: given y = s * q (input), qb (adjoint of the output
// rank-r vector), accumulate pb = U^T abar and the bias gradient rows into red_db.
template <int RM, int NI, int NO, int C>
__device__ __forceinline__ void layer_bwd(const float *__restrict__ U, const float *__restrict__ b,
                                          const float *__restrict__ Vn, int M,
                                          const float2 (&y)[C][RM / 2],
                                          const float2 (&qb)[C][RM / 2], float2 (&pb)[C][RM / 2],
                                          float *red_db) {
  static_assert(NI % 2 == 0, "input rank is padded to pairs");
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < M; i0 += 8) {
    float ab0[8];
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) {
      const int i = i0 + ii;
      ab0[ii] = 0.0f;
      if (i < M) {
        float2 uw[RM / 2], vw[RM / 2];
        load_row2<RM, NI>(U + (int64_t)i * RM, uw);
        load_row2<RM, NO>(Vn + (int64_t)i * RM, vw);
        float2 acc[C], accw[C];
        acc[0] = make_float2(__ldg(b + i), 0.0f);
#pragma unroll
        for (int c = 1; c < C; ++c) acc[c] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < C; ++c) accw[c] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int kk = 0; kk < NI / 2; ++kk)
#pragma unroll
          for (int c = 0; c < C; ++c) acc[c] = ff2(uw[kk], y[c][kk], acc[c]);
        float a[C][1], wb[C][1];
        if constexpr (NO == 1) {
#pragma unroll
          for (int c = 0; c < C; ++c) wb[c][0] = vw[0].x * qb[c][0].x;
        } else {
#pragma unroll
          for (int jj = 0; jj < NO / 2; ++jj)
#pragma unroll
            for (int c = 0; c < C; ++c) accw[c] = ff2(vw[jj], qb[c][jj], accw[c]);
#pragma unroll
          for (int c = 0; c < C; ++c) wb[c][0] = accw[c].x + accw[c].y;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) a[c][0] = acc[c].x + acc[c].y;
        act_bwd<C, 1>(a, wb);
#pragma unroll
        for (int kk = 0; kk < NI / 2; ++kk)
#pragma unroll
          for (int c = 0; c < C; ++c)
            pb[c][kk] = ff2(uw[kk], make_float2(wb[c][0], wb[c][0]), pb[c][kk]);
        ab0[ii] = wb[0][0];
      }
    }
    const float r = warp_reduce_scatter<8>(ab0);
    if ((lane & 3) == 0 && i0 + (lane >> 2) < M) red_db[i0 + (lane >> 2)] += r;
  }
}

template <int RM, int NT, int C>
__device__ void full_tile(const KParams &p, const Tile &T, const float *__restrict__ s_s,
                          float *__restrict__ q_s, float *red_w) {
  constexpr int RP = RM / 2;
  const int tid = threadIdx.x;
  const int L = p.L, M = p.M;
  const int64_t LS = full_layer_floats(M, RM);
  const float *V0 = p.pack + L * LS;
  const float Uout = __ldg(V0 + 2 * R1);
  const float bout = __ldg(V0 + 2 * R1 + 1);

  const PointIn pt = load_point(p, T, tid);
  const float x = pt.x, t = pt.t;
  float v00 = __ldg(V0 + 0), v01 = __ldg(V0 + 1), v10 = __ldg(V0 + R1), v11 = __ldg(V0 + R1 + 1);

  float2 q[C][RP];
  auto input_jet = [&]() {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int kk = 0; kk < RP; ++kk) q[c][kk] = make_float2(0.0f, 0.0f);
    q[0][0] = make_float2(v00 * x + v10 * t, v01 * x + v11 * t);
    if constexpr (C >= 3) {
      q[1][0] = make_float2(v10, v11);
      q[2][0] = make_float2(v00, v01);
    }
  };
  auto s_pair = [&](int l, int kk) {
    return make_float2(s_s[l * RM + 2 * kk], s_s[l * RM + 2 * kk + 1]);
  };
  auto slot = [&](int l, int c, int k) { return (((l - 1) * 4 + c) * RM + k) * NT + tid; };
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
          q_s[slot(l, c, 2 * kk)] = q[c][kk].x;
          q_s[slot(l, c, 2 * kk + 1)] = q[c][kk].y;
        }
    }
    float2 y[C][RP];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int kk = 0; kk < RP; ++kk) {
        y[c][kk] = fm2(q[c][kk], s_pair(l, kk));
        q[c][kk] = make_float2(0.0f, 0.0f);
      }
    if (l == 0 && l == L - 1) layer_fwd<RM, R1, 1, C>(U, b, Vn, M, y, q);
    else if (l == 0) layer_fwd<RM, R1, RM, C>(U, b, Vn, M, y, q);
    else if (l == L - 1) layer_fwd<RM, RM, 1, C>(U, b, Vn, M, y, q);
    else layer_fwd<RM, RM, RM, C>(U, b, Vn, M, y, q);
  }
  const float sL = s_s[L * RM];
  float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < C; ++c) u[c] = Uout * sL * q[c][0].x;
  u[0] += bout;

  float ub[4], lp;
  if (!residual_and_seeds(p, T, pt, tid, u, ub, lp)) return;

  const int DB0 = partial_db0(L, RM);
  {
    const float ls = warp_sum(lp);
    if ((tid & 31) == 0) red_w[0] += ls;
  }
  float2 qb[C][RP];
  {
    float dsL = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float pbv = Uout * ub[c];
      dsL += pbv * q[c][0].x;
#pragma unroll
      for (int kk = 0; kk < RP; ++kk) qb[c][kk] = make_float2(0.0f, 0.0f);
      qb[c][0].x = sL * pbv;
    }
    const float s0 = warp_sum(dsL);
    const float s1 = warp_sum(ub[0]);
    if ((tid & 31) == 0) {
      red_w[1 + L * RM] += s0;
      red_w[DB0 + L * M] += s1;
    }
  }
  // the layer's input jet q is read from the store twice (for s * q before the
  // layer, for dL/ds after it) instead of being held through the layer
  auto load_q = [&](int l) {
    if (l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int kk = 0; kk < RP; ++kk)
          q[c][kk] = make_float2(q_s[slot(l, c, 2 * kk)], q_s[slot(l, c, 2 * kk + 1)]);
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
        y[c][kk] = fm2(q[c][kk], s_pair(l, kk));
        pb[c][kk] = make_float2(0.0f, 0.0f);
      }
    float *red_db = red_w + DB0 + l * M;
    if (l == 0 && l == L - 1) layer_bwd<RM, R1, 1, C>(U, b, Vn, M, y, qb, pb, red_db);
    else if (l == 0) layer_bwd<RM, R1, RM, C>(U, b, Vn, M, y, qb, pb, red_db);
    else if (l == L - 1) layer_bwd<RM, RM, 1, C>(U, b, Vn, M, y, qb, pb, red_db);
    else layer_bwd<RM, RM, RM, C>(U, b, Vn, M, y, qb, pb, red_db);
    load_q(l);
    float g[RM];
#pragma unroll
    for (int kk = 0; kk < RP; ++kk) {
      float2 d = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int c = 0; c < C; ++c) d = ff2(pb[c][kk], q[c][kk], d);
      g[2 * kk] = d.x;
      g[2 * kk + 1] = d.y;
    }
    warp_accumulate<RM>(g, red_w, [&](int j) { return 1 + l * RM + j; });
    if (l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int kk = 0; kk < RP; ++kk) qb[c][kk] = fm2(pb[c][kk], s_pair(l, kk));
    }
  }
}

template <int RM, int NT>
__global__ void __launch_bounds__(NT) k_full_fp32(const __grid_constant__ KParams p) {
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x;
  const int L = p.L;
  const FullLayout<RM, NT> lay(L, p.P);
  float *s_s = smem + lay.s;
  float *q_s = p.scratch + (size_t)blockIdx.x * full_store_floats(L, RM, NT);
  float *red_s = smem + lay.red;
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
    if (T.kind == KIND_INT)
      full_tile<RM, NT, 4>(p, T, s_s, q_s, red_w);
    else
      full_tile<RM, NT, 1>(p, T, s_s, q_s, red_w);
    if (p.grad) {
      __syncthreads();
      for (int j = tid; j < p.P; j += NT) {
        float acc = 0.0f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) acc += red_s[w * p.P + j];
        if (j == 0 && !isfinite(acc)) set_status(p.status, DEV_NONFINITE);
        p.partial[(int64_t)tile * p.P + j] = acc;
      }
    }
  }
}

template <int RM, int NT>
cudaError_t launch_full_t(const KParams &p, int grid, cudaStream_t st) {
  const FullLayout<RM, NT> lay(p.L, p.P);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_full_fp32<RM, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_full_fp32<RM, NT><<<std::max(1, grid), NT, bytes, st>>>(p);
  return cudaGetLastError();
}

template <int RM, int NT>
int ctas_per_sm_t(const KParams &p) {
  const FullLayout<RM, NT> lay(p.L, p.P);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  if (cudaFuncSetAttribute(k_full_fp32<RM, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_full_fp32<RM, NT>, NT, bytes) !=
      cudaSuccess)
    return 1;
  return std::max(1, per_sm);
}

}  // namespace

size_t full_fp32_smem_bytes(int L, int RM, int NT, int P) {
  return (size_t)((L + 1) * RM + (NT / 32) * P) * sizeof(float);
}

size_t full_fp32_scratch_floats(int L, int RM, int NT, int grid) {
  return full_store_floats(L, RM, NT) * (size_t)grid;
}

int full_fp32_choose_nt(int L, int RM, int P) {
  for (int nt : {64, 32}) {
    if (full_fp32_smem_bytes(L, RM, nt, P) <= (size_t)kSmemBudget) return nt;
  }
  return 0;
}

int full_fp32_ctas_per_sm(const KParams &p) {
  if (p.RM >= 32) return full_fp32_sl_ctas_per_sm(p);
  if (p.nt == 64) {
    if (p.RM == 8) return ctas_per_sm_t<8, 64>(p);
    if (p.RM == 16) return ctas_per_sm_t<16, 64>(p);
  } else if (p.nt == 32) {
    if (p.RM == 8) return ctas_per_sm_t<8, 32>(p);
    if (p.RM == 16) return ctas_per_sm_t<16, 32>(p);
  }
  return 1;
}

// Padded ranks 8 and 16: one thread per point (this file); 32 and 64: the sliced
// kernel, RM / 16 threads per point.
cudaError_t launch_full_fp32(const KParams &p, int grid, cudaStream_t st) {
  if (p.RM >= 32) return launch_full_fp32_sl(p, grid, st);
  if (!p.scratch && p.grad) return cudaErrorInvalidValue;
  if (p.nt == 64) {
    if (p.RM == 8) return launch_full_t<8, 64>(p, grid, st);
    if (p.RM == 16) return launch_full_t<16, 64>(p, grid, st);
  } else if (p.nt == 32) {
    if (p.RM == 8) return launch_full_t<8, 32>(p, grid, st);
    if (p.RM == 16) return launch_full_t<16, 32>(p, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lrnr
