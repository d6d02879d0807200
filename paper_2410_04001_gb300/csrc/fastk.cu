// FastLRNR residual + adjoint in FP32 for ranks above the rank-r jet kernel (padded
// rank 32 or 64, as in the convection-diffusion-reaction network r = (1, 49, 30, 25, 1)
// of Sec. 4) with reduced widths rhat <= 16 (Sec. 2.2 Eq. 2.8, Sec. 2.3).
//
// The reduced layers compose through rhat-dimensional states.  With w^l the tanh jet
// of the pre-activation a^l of hidden layer l (rhat_l rows):
//   a^0 = K^0 z^0 + bhat^0,       K^0 = Uhat^0 diag(s^0) V^0^T          (rhat_0 x 2)
//   a^l = K^l w^{l-1} + bhat^l,   K^l = Uhat^l diag(s^l) Vhat^{l-1 T}   (rhat_l x rhat_{l-1})
//   u   = k . w^{L-1} + b^L,      k   = U^L s^L Vhat^{L-1 T}            (1 x rhat_{L-1})
// where Vhat^{l-1} is the reduced output basis of layer l-1, so a point carries jets of
// rhat entries instead of rank-r jets; the maps K are formed once per tile from s.
// The gradient in s goes through the same factorisation:
//   dL/ds^l_k = sum_{i,j} Uhat^l_{ik} Vhat^{l-1}_{jk} G^l_{ij},
//   G^l = sum over the tile's points and jet channels of abar^l (outer) w^{l-1},
// and dL/ds^L_0 = U^L sum_j Vhat^{L-1}_{j0} g_j with g = sum of ubar_c w^{L-1}_c.  Each
// point adds its rhat x rhat products to G (summed over the warp by reduce-scatter,
// then over the warps in a fixed order), and the rank-r projection runs once per
// tile.  The partial row per tile has the layout of the rank-r kernel's, so the same
// reductions follow: a separate fixed-order reduction for large batches, or (FR) the
// group-ticket reduction and Adam inside this kernel when the batch's tiles fit in
// one round of the grid, which with the tile offsets computed here makes a small
// SPInProp step a single launch.
#include "lrnr_internal.cuh"
#include "point_common.cuh"
#include "simt_common.cuh"
#include "fused_reduce.cuh"

namespace lrnr {
namespace {

constexpr int KT = 128;   // threads (points) per tile

// Shared memory (floats): the reduced pack, s, the maps K (L blocks of RH x RH; K^0 in
// columns 0..1 of block 0) and k, the per-warp G accumulators (L blocks of RH x RH and
// g), one partial row per warp, the tile offsets and their scan when the kernel
// computes them (fused_inst instances), and the per-warp sums and flag of the fused
// reduction.
struct KfLayout {
  int pack, s, K, kout, G, red, toff, scan, misc, total;
  __host__ __device__ KfLayout(int L, int RM, int RH, int P, int fused_inst) {
    pack = 0;
    s = (fast_pack_floats(L, RM, RH) + 3) & ~3;
    K = (s + (L + 1) * RM + 3) & ~3;
    kout = K + L * RH * RH;
    G = (kout + RH + 3) & ~3;
    const int gw = L * RH * RH + RH;
    red = G + (KT / 32) * gw;
    toff = red + (KT / 32) * P;
    scan = toff + (fused_inst ? fused_inst + 1 : 0);
    misc = scan + (fused_inst ? KT : 0);
    total = misc + KT / 32 + 1;
  }
  __host__ __device__ static int g_floats(int L, int RH) { return L * RH * RH + RH; }
};

// Per-CTA global store of the reverse sweep: the layer inputs w^{l-1} (l >= 1, four
// channels of RH) and each row's kept jet values (tanh value, a_t, a_x, a_xx).
__host__ __device__ inline size_t fastk_store_floats(int L, int RH) {
  return (size_t)(L > 1 ? L - 1 : 1) * 4 * RH * KT + (size_t)L * RH * 4 * KT;
}

// Add this thread's values v[0..N) (N a multiple of 32) into dst[0..N) as warp sums.
template <int N>
__device__ __forceinline__ void warp_add_rows(float (&v)[N], float *dst) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < N; b += 32) {
    float t[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) t[j] = v[b + j];
    const float r = warp_reduce_scatter<32>(t);
    dst[b + lane] += r;
  }
}

template <int RM, int RH, int C>
__device__ void fastk_tile(const KParams &p, const Tile &T, const float *__restrict__ w_s,
                           const float *__restrict__ K_s, const float *__restrict__ kout_s,
                           float *__restrict__ G_w, float4 *__restrict__ q_g,
                           float4 *__restrict__ a_g, float *red_w) {
  const int tid = threadIdx.x;
  const int L = p.L;
  const int LS = fast_layer_floats(RM, RH);
  const float bout = w_s[L * LS + 2 * R1 + 1];
  const PointIn pt = load_point(p, T, tid);
  const float x = pt.x, t = pt.t;
  // the input jet z^0 = (x, t) and its channels (d/dt, d/dx, d2/dx2)
  auto input_jet = [&](float (&w)[C][RH]) {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int j = 0; j < RH; ++j) w[c][j] = 0.0f;
    w[0][0] = x;
    w[0][1] = t;
    if constexpr (C == 4) {
      w[1][1] = 1.0f;
      w[2][0] = 1.0f;
    }
  };
  auto in_slot = [&](int l, int c, int j) { return (((l - 1) * 4 + c) * RH + j) * KT + tid; };

  float w[C][RH];
  input_jet(w);
  for (int l = 0; l < L; ++l) {
    const float *K = K_s + l * RH * RH;
    const float *bh = w_s + l * LS + RH * RM;
    const int nin = l == 0 ? R1 : RH;
    if (p.grad && l > 0) {
      float *qs = reinterpret_cast<float *>(q_g);
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < RH; ++j) qs[in_slot(l, c, j)] = w[c][j];
    }
    float a[C][RH];
#pragma unroll
    for (int i = 0; i < RH; ++i) {
#pragma unroll
      for (int c = 0; c < C; ++c) a[c][i] = c == 0 ? bh[i] : 0.0f;
#pragma unroll
      for (int j = 0; j < RH; ++j) {
        if (j >= nin) break;
        const float kij = K[i * RH + j];
#pragma unroll
        for (int c = 0; c < C; ++c) a[c][i] = fmaf(kij, w[c][j], a[c][i]);
      }
    }
#pragma unroll
    for (int i = 0; i < RH; ++i) {
      float z, d1, d2;
      tanh_d(a[0][i], z, d1, d2);
      float4 keep = make_float4(z, 0.0f, 0.0f, 0.0f);
      if constexpr (C == 4) {
        keep = make_float4(z, a[1][i], a[2][i], a[3][i]);
        w[3][i] = d2 * a[2][i] * a[2][i] + d1 * a[3][i];
        w[1][i] = d1 * a[1][i];
        w[2][i] = d1 * a[2][i];
      }
      w[0][i] = z;
      if (p.grad) a_g[(l * RH + i) * KT + tid] = keep;
    }
  }
  float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < RH; ++j) acc = fmaf(kout_s[j], w[c][j], acc);
    u[c] = acc;
  }
  u[0] += bout;

  float ub[4], lp;
  if (!residual_and_seeds(p, T, pt, tid, u, ub, lp)) return;

  const int DB0 = partial_db0(L, RM);
  {
    const float ls = warp_sum(lp);
    const float s1 = warp_sum(ub[0]);
    if ((tid & 31) == 0) {
      red_w[0] += ls;
      red_w[DB0 + L * RH] += s1;
    }
    // g_j = sum_c ubar_c w^{L-1}_{c,j} (for dL/ds of the output layer)
    float gv[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float acc = 0.0f;
      if (j < RH) {
#pragma unroll
        for (int c = 0; c < C; ++c) acc = fmaf(ub[c], w[c][j], acc);
      }
      gv[j] = acc;
    }
    const int lane = tid & 31;
    const float r = warp_reduce_scatter<32>(gv);
    if (lane < RH) G_w[L * RH * RH + lane] += r;
  }
  // output adjoint of the last hidden layer's state
  float wb[C][RH];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int j = 0; j < RH; ++j) wb[c][j] = ub[c] * kout_s[j];

  for (int l = L - 1; l >= 0; --l) {
    const float *K = K_s + l * RH * RH;
    const int nin = l == 0 ? R1 : RH;
    // abar of the rows from the kept jet values (the chain rule of the tanh jet)
#pragma unroll
    for (int i = 0; i < RH; ++i) {
      const float4 k = a_g[(l * RH + i) * KT + tid];
      float v[C];
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = wb[c][i];
      const float z = k.x;
      const float d1 = 1.0f - z * z;
      float ab0 = v[0] * d1;
      if constexpr (C == 4) {
        const float d2 = -2.0f * z * d1;
        const float d3 = d1 * (6.0f * z * z - 2.0f);
        ab0 += d2 * (v[1] * k.y + v[2] * k.z);
        ab0 += v[3] * (d3 * k.z * k.z + d2 * k.w);
        wb[2][i] = v[2] * d1 + 2.0f * v[3] * d2 * k.z;
        wb[3][i] = v[3] * d1;
        wb[1][i] = v[1] * d1;
      }
      wb[0][i] = ab0;
    }
    // dL/dbhat^l rows
    {
      float g[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) g[i] = i < RH ? wb[0][i] : 0.0f;
      const float r = warp_reduce_scatter<32>(g);
      const int lane = tid & 31;
      if (lane < RH) red_w[DB0 + l * RH + lane] += r;
    }
    // the layer's input w^{l-1} (z^0 for the first layer)
    float wp[C][RH];
    if (l > 0) {
      const float *qs = reinterpret_cast<const float *>(q_g);
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < RH; ++j) wp[c][j] = qs[in_slot(l, c, j)];
    } else {
      input_jet(wp);
    }
    // G^l += sum_c abar_c (outer) w^{l-1}_c, in chunks of 32 entries
    float *Gl = G_w + l * RH * RH;
#pragma unroll
    for (int b = 0; b < RH * RH; b += 32) {
      float gv[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int i = (b + e) / RH, j = (b + e) % RH;
        float acc = 0.0f;
        if (j < nin) {
#pragma unroll
          for (int c = 0; c < C; ++c) acc = fmaf(wb[c][i], wp[c][j], acc);
        }
        gv[e] = acc;
      }
      const float r = warp_reduce_scatter<32>(gv);
      Gl[b + (tid & 31)] += r;
    }
    // wbar^{l-1} = K^l^T abar
    if (l > 0) {
      float nb[C][RH];
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < RH; ++j) nb[c][j] = 0.0f;
#pragma unroll
      for (int i = 0; i < RH; ++i)
#pragma unroll
        for (int j = 0; j < RH; ++j) {
          const float kij = K[i * RH + j];
#pragma unroll
          for (int c = 0; c < C; ++c) nb[c][j] = fmaf(kij, wb[c][i], nb[c][j]);
        }
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < RH; ++j) wb[c][j] = nb[c][j];
    }
  }
}

// FR: the variant with the fixed-order reduction and Adam inside the kernel (group
// tickets), for batches whose tiles fit in one round of the grid.
template <int RM, int RH, bool FR>
__global__ void __launch_bounds__(KT, 2) k_fastk(const __grid_constant__ KParams p) {
  static_assert(RH == 8 || RH == 16, "reduced width");
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x;
  const int L = p.L;
  const KfLayout lay(L, RM, RH, p.P, p.fused_tiles ? p.n_inst : 0);
  float *w_s = smem + lay.pack;
  float *s_s = smem + lay.s;
  float *K_s = smem + lay.K;
  float *kout_s = smem + lay.kout;
  float *G_s = smem + lay.G;
  float *red_s = smem + lay.red;
  const int GW = KfLayout::g_floats(L, RH);
  float *store = p.scratch + (size_t)blockIdx.x * fastk_store_floats(L, RH);
  float4 *q_g = reinterpret_cast<float4 *>(store);
  float4 *a_g = reinterpret_cast<float4 *>(store + (size_t)(L > 1 ? L - 1 : 1) * 4 * RH * KT);
  const int LS = fast_layer_floats(RM, RH);
  const int npack = fast_pack_floats(L, RM, RH);
  for (int i = tid; i < npack; i += KT) w_s[i] = __ldg(p.pack + i);
  // Adam step number: the fused reduction reads the counter here and advances it
  // once every instance is done; otherwise block 0 advances it for the next kernel
  if (!FR && p.step && blockIdx.x == 0 && tid == 0) atomicAdd((unsigned long long *)p.step, 1ull);
  const int64_t kstep = (FR && p.step) ? *p.step + 1 : 0;
  float *wsum = smem + lay.misc;
  int *flag = reinterpret_cast<int *>(smem + lay.misc + KT / 32);
  __syncthreads();   // the pack is read by every thread below
  const float *V0 = w_s + L * LS;
  const float Uout = V0[2 * R1];
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
    const Tile T = decode_tile(p, tile, toff);
    __syncthreads();
    for (int j = tid; j < (L + 1) * RM; j += KT) {
      const int l = j / RM, k = j % RM;
      s_s[j] = (k < p.r[l]) ? __ldg(p.s + (int64_t)T.inst * p.sum_r + p.roff[l] + k) : 0.0f;
    }
    if (p.grad) {
      for (int j = tid; j < (KT / 32) * p.P; j += KT) red_s[j] = 0.0f;
      for (int j = tid; j < (KT / 32) * GW; j += KT) G_s[j] = 0.0f;
    }
    __syncthreads();
    // the maps K^l and k for this instance's coefficients
    for (int e = tid; e < L * RH * RH + RH; e += KT) {
      float acc = 0.0f;
      if (e < L * RH * RH) {
        const int l = e / (RH * RH), i = (e / RH) % RH, j = e % RH;
        const float *Uh = w_s + l * LS + i * RM;
        const float *sl = s_s + l * RM;
        if (l == 0) {
          if (j < R1)
            for (int k = 0; k < R1; ++k) acc = fmaf(Uh[k] * sl[k], V0[j * R1 + k], acc);
        } else {
          // four partial sums over the rank (RM is a multiple of 4)
          const float *Vp = w_s + (l - 1) * LS + RH * RM + RH + j * RM;
          float a4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 2
          for (int k = 0; k < RM; k += 4)
#pragma unroll
            for (int q = 0; q < 4; ++q) a4[q] = fmaf(Uh[k + q] * sl[k + q], Vp[k + q], a4[q]);
          acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
        }
        K_s[e] = acc;
      } else {
        const int j = e - L * RH * RH;
        const float *Vp = w_s + (L - 1) * LS + RH * RM + RH + j * RM;
        kout_s[j] = Uout * s_s[L * RM] * Vp[0];
      }
    }
    __syncthreads();
    float *red_w = red_s + (tid >> 5) * p.P;
    float *G_w = G_s + (tid >> 5) * GW;
    if (T.kind == KIND_INT)
      fastk_tile<RM, RH, 4>(p, T, w_s, K_s, kout_s, G_w, q_g, a_g, red_w);
    else
      fastk_tile<RM, RH, 1>(p, T, w_s, K_s, kout_s, G_w, q_g, a_g, red_w);
    if (p.grad) {
      __syncthreads();
      // the warps' G added in order into warp 0's block
      for (int e = tid; e < GW; e += KT) {
        float g = G_s[e];
#pragma unroll
        for (int w = 1; w < KT / 32; ++w) g += G_s[w * GW + e];
        G_s[e] = g;
      }
      __syncthreads();
      // dL/ds from the tile's G, projected through the bases (two partial sums per
      // entry); written into warp 0's partial row, whose dL/ds entries are otherwise zero
      for (int e = tid; e < (L + 1) * RM; e += KT) {
        const int l = e / RM, k = e % RM;
        if (k >= p.r[l]) continue;
        float acc0 = 0.0f, acc1 = 0.0f;
        if (l == 0) {
          const float *Uh = w_s;
#pragma unroll
          for (int i = 0; i < RH; ++i) {
            const float *Gi = G_s + i * RH;
            const float ui = Uh[i * RM + k];
            acc0 = fmaf(ui * V0[k], Gi[0], acc0);
            acc1 = fmaf(ui * V0[R1 + k], Gi[1], acc1);
          }
        } else if (l < L) {
          const float *Uh = w_s + l * LS;
          const float *Vp = w_s + (l - 1) * LS + RH * RM + RH + k;
          const float *Gl = G_s + l * RH * RH;
          for (int i = 0; i < RH; ++i) {
            const float ui = Uh[i * RM + k];
            float h0 = 0.0f, h1 = 0.0f;
#pragma unroll
            for (int j = 0; j < RH; j += 2) {
              h0 = fmaf(Vp[j * RM], Gl[i * RH + j], h0);
              h1 = fmaf(Vp[(j + 1) * RM], Gl[i * RH + j + 1], h1);
            }
            acc0 = fmaf(ui, h0, acc0);
            acc1 = fmaf(ui, h1, acc1);
          }
        } else {
          const float *Vp = w_s + (L - 1) * LS + RH * RM + RH + k;
          const float *g = G_s + L * RH * RH;
#pragma unroll
          for (int j = 0; j < RH; j += 2) {
            acc0 = fmaf(Vp[j * RM], g[j], acc0);
            acc1 = fmaf(Vp[(j + 1) * RM], g[j + 1], acc1);
          }
          acc0 *= Uout;
          acc1 *= Uout;
        }
        red_s[1 + l * RM + k] += acc0 + acc1;
      }
      __syncthreads();
      for (int j = tid; j < p.P; j += KT) {
        float acc = 0.0f;
        for (int w = 0; w < KT / 32; ++w) acc += red_s[w * p.P + j];
        if (j == 0 && !isfinite(acc)) set_status(p.status, DEV_NONFINITE);
        p.partial[(int64_t)tile * p.P + j] = acc;
      }
      l2_discard(store, fastk_store_floats(L, RH) * sizeof(float));
      if constexpr (FR) fast_tile_done(p, tile, ntiles, toff, red_s, wsum, flag, kstep);
    }
  }
}

template <int RM, int RH, bool FR>
cudaError_t launch_fastk_v(const KParams &p, int grid, cudaStream_t st) {
  const KfLayout lay(p.L, RM, RH, p.P, p.fused_tiles ? p.n_inst : 0);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_fastk<RM, RH, FR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_fastk<RM, RH, FR><<<std::max(1, grid), KT, bytes, st>>>(p);
  return cudaGetLastError();
}

template <int RM, int RH>
cudaError_t launch_fastk_t(const KParams &p, int grid, cudaStream_t st) {
  return p.fused_red ? launch_fastk_v<RM, RH, true>(p, grid, st)
                     : launch_fastk_v<RM, RH, false>(p, grid, st);
}

template <int RM, int RH>
int fastk_ctas_per_sm_t(const KParams &p) {
  const KfLayout lay(p.L, RM, RH, p.P, p.fused_tiles ? p.n_inst : 0);
  const size_t bytes = (size_t)lay.total * sizeof(float);
  if (cudaFuncSetAttribute(k_fastk<RM, RH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fastk<RM, RH, false>, KT, bytes) !=
      cudaSuccess)
    return 1;
  return std::max(1, per_sm);
}

}  // namespace

bool fastk_supported(int L, int RM, int RH, int P, int fused_inst) {
  if ((RM != 32 && RM != 64) || (RH != 8 && RH != 16) || L < 1) return false;
  const KfLayout lay(L, RM, RH, P, fused_inst);
  return (size_t)lay.total * sizeof(float) <= (size_t)kSmemBudget;
}

int fastk_nt() { return KT; }

size_t fastk_scratch_floats(int L, int RH, int grid) {
  return fastk_store_floats(L, RH) * (size_t)grid;
}

int fastk_ctas_per_sm(const KParams &p) {
  if (p.RM == 32) return p.RH == 8 ? fastk_ctas_per_sm_t<32, 8>(p) : fastk_ctas_per_sm_t<32, 16>(p);
  return p.RH == 8 ? fastk_ctas_per_sm_t<64, 8>(p) : fastk_ctas_per_sm_t<64, 16>(p);
}

cudaError_t launch_fastk(const KParams &p, int grid, cudaStream_t st) {
  if (p.nt != KT || (!p.scratch && p.grad)) return cudaErrorInvalidValue;
  if (p.RM == 32 && p.RH == 8) return launch_fastk_t<32, 8>(p, grid, st);
  if (p.RM == 32 && p.RH == 16) return launch_fastk_t<32, 16>(p, grid, st);
  if (p.RM == 64 && p.RH == 8) return launch_fastk_t<64, 8>(p, grid, st);
  if (p.RM == 64 && p.RH == 16) return launch_fastk_t<64, 16>(p, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace lrnr
