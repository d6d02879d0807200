// SIMT building blocks shared by the FP32 kernels: small register-blocked
// matrix-vector products against shared/global weights, the tanh jet (value,
// d/dt, d/dx, d2/dx2) and its adjoint, and warp reductions into a partial row.
#pragma once

#include "lrnr_internal.cuh"

namespace lrnr {

// a[c][i] (+)= sum_k W[i*RM + k] * y[c][k],  i < NO, k < NI
template <int RM, int NI, int NO, int C>
__device__ __forceinline__ void mv_rows(const float *__restrict__ W, const float (&y)[C][RM],
                                        float (&a)[C][NO]) {
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    if constexpr (NI % 4 == 0) {
#pragma unroll
      for (int k = 0; k < NI; k += 4) {
        const float4 w = *reinterpret_cast<const float4 *>(W + i * RM + k);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          a[c][i] = fmaf(w.x, y[c][k + 0], a[c][i]);
          a[c][i] = fmaf(w.y, y[c][k + 1], a[c][i]);
          a[c][i] = fmaf(w.z, y[c][k + 2], a[c][i]);
          a[c][i] = fmaf(w.w, y[c][k + 3], a[c][i]);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < NI; ++k) {
        const float w = W[i * RM + k];
#pragma unroll
        for (int c = 0; c < C; ++c) a[c][i] = fmaf(w, y[c][k], a[c][i]);
      }
    }
  }
}

// o[c][k] (+)= sum_i W[i*RM + k] * v[c][i],  i < NR, k < NK
template <int RM, int NR, int NK, int C, int NV>
__device__ __forceinline__ void mv_cols(const float *__restrict__ W, const float (&v)[C][NV],
                                        float (&o)[C][RM]) {
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    if constexpr (NK % 4 == 0) {
#pragma unroll
      for (int k = 0; k < NK; k += 4) {
        const float4 w = *reinterpret_cast<const float4 *>(W + i * RM + k);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          o[c][k + 0] = fmaf(w.x, v[c][i], o[c][k + 0]);
          o[c][k + 1] = fmaf(w.y, v[c][i], o[c][k + 1]);
          o[c][k + 2] = fmaf(w.z, v[c][i], o[c][k + 2]);
          o[c][k + 3] = fmaf(w.w, v[c][i], o[c][k + 3]);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const float w = W[i * RM + k];
#pragma unroll
        for (int c = 0; c < C; ++c) o[c][k] = fmaf(w, v[c][i], o[c][k]);
      }
    }
  }
}

template <int C, int N>
__device__ __forceinline__ void act_fwd(float (&a)[C][N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float z, d1, d2;
    tanh_d(a[0][i], z, d1, d2);
    if constexpr (C == 4) a[3][i] = d2 * a[2][i] * a[2][i] + d1 * a[3][i];
    if constexpr (C >= 3) {
      a[1][i] = d1 * a[1][i];
      a[2][i] = d1 * a[2][i];
    }
    a[0][i] = z;
  }
}

// Given the pre-activation jet a and the output adjoint wb, overwrite wb with the
// pre-activation adjoint (chain rule of act_fwd, reversed).
template <int C, int N>
__device__ __forceinline__ void act_bwd(const float (&a)[C][N], float (&wb)[C][N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float z, d1, d2;
    tanh_d(a[0][i], z, d1, d2);
    float ab0 = wb[0][i] * d1;
    if constexpr (C >= 3) ab0 += d2 * (wb[1][i] * a[1][i] + wb[2][i] * a[2][i]);
    if constexpr (C == 4) {
      const float d3 = d1 * (6.0f * z * z - 2.0f);
      ab0 += wb[3][i] * (d3 * a[2][i] * a[2][i] + d2 * a[3][i]);
      wb[2][i] = wb[2][i] * d1 + 2.0f * wb[3][i] * d2 * a[2][i];
      wb[3][i] = wb[3][i] * d1;
    } else if constexpr (C >= 3) {
      wb[2][i] = wb[2][i] * d1;
    }
    if constexpr (C >= 3) wb[1][i] = wb[1][i] * d1;
    wb[0][i] = ab0;
  }
}

// Reduce NV values over the warp and add them to the warp's row of red_s at the
// positions given by slot(j).
template <int NV, typename SlotFn>
__device__ __forceinline__ void warp_accumulate(const float (&v)[NV], float *red_w, SlotFn slot) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int base = 0; base < NV; base += 32) {
    float t[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) t[j] = (base + j < NV) ? v[base + j] : 0.0f;
    const float r = warp_reduce_scatter<32>(t);
    if (base + lane < NV) red_w[slot(base + lane)] += r;
  }
}

}  // namespace lrnr
