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

template <int RM, int NI>
__device__ __forceinline__ void load_row(const float *__restrict__ W, float (&w)[RM]) {
  if constexpr (NI % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NI; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(W + k));
      w[k] = v.x; w[k + 1] = v.y; w[k + 2] = v.z; w[k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NI; ++k) w[k] = __ldg(W + k);
  }
}

// One hidden layer forward: q (input jet, overwritten with s * q) -> qn.
template <int RM, int NI, int NO, int C>
__device__ __forceinline__ void layer_fwd(const float *__restrict__ U, const float *__restrict__ b,
                                          const float *__restrict__ Vn, int M,
                                          const float (&y)[C][RM], float (&qn)[C][RM]) {
#pragma unroll 2
  for (int i = 0; i < M; ++i) {
    float uw[RM], vw[RM];
    load_row<RM, NI>(U + (int64_t)i * RM, uw);
    load_row<RM, NO>(Vn + (int64_t)i * RM, vw);
    float a[C][1];
    a[0][0] = __ldg(b + i);
#pragma unroll
    for (int c = 1; c < C; ++c) a[c][0] = 0.0f;
#pragma unroll
    for (int k = 0; k < NI; ++k)
#pragma unroll
      for (int c = 0; c < C; ++c) a[c][0] = fmaf(uw[k], y[c][k], a[c][0]);
    act_fwd<C, 1>(a);
#pragma unroll
    for (int j = 0; j < NO; ++j)
#pragma unroll
      for (int c = 0; c < C; ++c) qn[c][j] = fmaf(vw[j], a[c][0], qn[c][j]);
  }
}

// One hidden layer reverse: given y = s * q (input), qb (adjoint of the output
// rank-r vector), accumulate pb = U^T abar and the bias gradient rows into red_w.
template <int RM, int NI, int NO, int C>
__device__ __forceinline__ void layer_bwd(const float *__restrict__ U, const float *__restrict__ b,
                                          const float *__restrict__ Vn, int M,
                                          const float (&y)[C][RM], const float (&qb)[C][RM],
                                          float (&pb)[C][RM], float *red_db) {
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < M; i0 += 8) {
    float ab0[8];
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) {
      const int i = i0 + ii;
      ab0[ii] = 0.0f;
      if (i < M) {
        float uw[RM], vw[RM];
        load_row<RM, NI>(U + (int64_t)i * RM, uw);
        load_row<RM, NO>(Vn + (int64_t)i * RM, vw);
        float a[C][1], wb[C][1];
        a[0][0] = __ldg(b + i);
#pragma unroll
        for (int c = 1; c < C; ++c) a[c][0] = 0.0f;
#pragma unroll
        for (int c = 0; c < C; ++c) wb[c][0] = 0.0f;
#pragma unroll
        for (int k = 0; k < NI; ++k)
#pragma unroll
          for (int c = 0; c < C; ++c) a[c][0] = fmaf(uw[k], y[c][k], a[c][0]);
#pragma unroll
        for (int j = 0; j < NO; ++j)
#pragma unroll
          for (int c = 0; c < C; ++c) wb[c][0] = fmaf(vw[j], qb[c][j], wb[c][0]);
        act_bwd<C, 1>(a, wb);
#pragma unroll
        for (int k = 0; k < NI; ++k)
#pragma unroll
          for (int c = 0; c < C; ++c) pb[c][k] = fmaf(uw[k], wb[c][0], pb[c][k]);
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
  const int tid = threadIdx.x;
  const int L = p.L, M = p.M;
  const int64_t LS = full_layer_floats(M, RM);
  const float *V0 = p.pack + L * LS;
  const float Uout = __ldg(V0 + 2 * R1);
  const float bout = __ldg(V0 + 2 * R1 + 1);

  const PointIn pt = load_point(p, T, tid);
  const float x = pt.x, t = pt.t;
  float v00 = __ldg(V0 + 0), v01 = __ldg(V0 + 1), v10 = __ldg(V0 + R1), v11 = __ldg(V0 + R1 + 1);

  float q[C][RM];
  auto input_jet = [&]() {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) q[c][k] = 0.0f;
    q[0][0] = v00 * x + v10 * t;
    q[0][1] = v01 * x + v11 * t;
    if constexpr (C >= 3) {
      q[1][0] = v10; q[1][1] = v11;
      q[2][0] = v00; q[2][1] = v01;
    }
  };
  input_jet();

  for (int l = 0; l < L; ++l) {
    const float *U = p.pack + l * LS;
    const float *b = U + (int64_t)M * RM;
    const float *Vn = b + pad4(M);
    if (p.grad && l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < RM; ++k) q_s[(((l - 1) * 4 + c) * RM + k) * NT + tid] = q[c][k];
    }
    float y[C][RM];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) { y[c][k] = q[c][k] * s_s[l * RM + k]; q[c][k] = 0.0f; }
    if (l == 0 && l == L - 1) layer_fwd<RM, R1, 1, C>(U, b, Vn, M, y, q);
    else if (l == 0) layer_fwd<RM, R1, RM, C>(U, b, Vn, M, y, q);
    else if (l == L - 1) layer_fwd<RM, RM, 1, C>(U, b, Vn, M, y, q);
    else layer_fwd<RM, RM, RM, C>(U, b, Vn, M, y, q);
  }
  const float sL = s_s[L * RM];
  float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < C; ++c) u[c] = Uout * sL * q[c][0];
  u[0] += bout;

  float ub[4], lp;
  if (!residual_and_seeds(p, T, pt, tid, u, ub, lp)) return;

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
      const float pbv = Uout * ub[c];
      dsL += pbv * q[c][0];
#pragma unroll
      for (int k = 0; k < RM; ++k) qb[c][k] = 0.0f;
      qb[c][0] = sL * pbv;
    }
    const float s0 = warp_sum(dsL);
    const float s1 = warp_sum(ub[0]);
    if ((tid & 31) == 0) {
      red_w[1 + L * RM] += s0;
      red_w[DB0 + L * M] += s1;
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const float *U = p.pack + l * LS;
    const float *b = U + (int64_t)M * RM;
    const float *Vn = b + pad4(M);
    if (l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < RM; ++k) q[c][k] = q_s[(((l - 1) * 4 + c) * RM + k) * NT + tid];
    } else {
      input_jet();
    }
    float y[C][RM], pb[C][RM];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int k = 0; k < RM; ++k) { y[c][k] = q[c][k] * s_s[l * RM + k]; pb[c][k] = 0.0f; }
    float *red_db = red_w + DB0 + l * M;
    if (l == 0 && l == L - 1) layer_bwd<RM, R1, 1, C>(U, b, Vn, M, y, qb, pb, red_db);
    else if (l == 0) layer_bwd<RM, R1, RM, C>(U, b, Vn, M, y, qb, pb, red_db);
    else if (l == L - 1) layer_bwd<RM, RM, 1, C>(U, b, Vn, M, y, qb, pb, red_db);
    else layer_bwd<RM, RM, RM, C>(U, b, Vn, M, y, qb, pb, red_db);
    float g[RM];
#pragma unroll
    for (int k = 0; k < RM; ++k) {
      float d = 0.0f;
#pragma unroll
      for (int c = 0; c < C; ++c) d = fmaf(pb[c][k], q[c][k], d);
      g[k] = d;
    }
    warp_accumulate<RM>(g, red_w, [&](int j) { return 1 + l * RM + j; });
    if (l > 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < RM; ++k) qb[c][k] = pb[c][k] * s_s[l * RM + k];
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
  if (p.nt == 64) {
    if (p.RM == 8) return ctas_per_sm_t<8, 64>(p);
    if (p.RM == 16) return ctas_per_sm_t<16, 64>(p);
    if (p.RM == 32) return ctas_per_sm_t<32, 64>(p);
  } else if (p.nt == 32) {
    if (p.RM == 8) return ctas_per_sm_t<8, 32>(p);
    if (p.RM == 16) return ctas_per_sm_t<16, 32>(p);
    if (p.RM == 32) return ctas_per_sm_t<32, 32>(p);
  }
  return 1;
}

cudaError_t launch_full_fp32(const KParams &p, int grid, cudaStream_t st) {
  if (!p.scratch && p.grad) return cudaErrorInvalidValue;
  if (p.nt == 64) {
    if (p.RM == 8) return launch_full_t<8, 64>(p, grid, st);
    if (p.RM == 16) return launch_full_t<16, 64>(p, grid, st);
    if (p.RM == 32) return launch_full_t<32, 64>(p, grid, st);
  } else if (p.nt == 32) {
    if (p.RM == 8) return launch_full_t<8, 32>(p, grid, st);
    if (p.RM == 16) return launch_full_t<16, 32>(p, grid, st);
    if (p.RM == 32) return launch_full_t<32, 32>(p, grid, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lrnr
