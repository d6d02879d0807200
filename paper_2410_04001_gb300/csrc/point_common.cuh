// Per-point pieces shared by every tile kernel: reading the collocation point of a
// tile slot, and forming the CDR residual / boundary residual, the point's share of
// the loss and the adjoint seeds of the output jet (Sec. 4 Eq. 4.1; Sec. 3.2
// Eq. 3.5 and 3.6).
#pragma once

#include "lrnr_internal.cuh"

namespace lrnr {

struct PointIn {
  bool act;     // slot holds a real point
  float x, t;
  int side;     // periodic tiles: 0 = (0, t), 1 = (2pi, t)
};

__device__ __forceinline__ PointIn load_point(const KParams &p, const Tile &T, int slot) {
  PointIn pt;
  pt.side = 0;
  if (T.kind == KIND_BC) {
    const int pr = slot >> 1;
    pt.side = slot & 1;
    pt.act = pr < T.count;
    pt.t = pt.act ? __ldg(p.t_bc + T.first + pr) : 0.5f;
    pt.x = pt.side ? TWO_PI_F : 0.0f;
  } else {
    pt.act = slot < T.count;
    const int64_t g = T.first + slot;
    if (T.kind == KIND_INT) {
      pt.x = pt.act ? __ldg(p.x_int + g) : 1.0f;
      pt.t = pt.act ? __ldg(p.t_int + g) : 0.5f;
    } else {
      pt.x = pt.act ? __ldg(p.x_ic + g) : 1.0f;
      pt.t = 0.0f;
    }
  }
  return pt;
}

// Denominator of the MSE mean of point class k (0 interior, 1 initial, 2 periodic)
// of instance inst (Eq. 3.5): the caller's count when the batch carries one (a shard
// of an instance's points is normalised by the count of the whole instance, so that
// the shards' losses and gradients add up to the instance's), else the class's own
// count in this batch.
__device__ __forceinline__ float mse_count(const KParams &p, int inst, int k, const int64_t *off) {
  return (float)(p.norm ? __ldg(p.norm + 3 * (int64_t)inst + k)
                        : __ldg(off + inst + 1) - __ldg(off + inst));
}

// Given the output jet u = (u, u_t, u_x, u_xx) of the point in `slot`: in
// evaluation mode write the requested outputs (when `write`) and return false; in
// gradient mode return true with the point's loss share in lp and the seeds
// d loss / d u_c in ub.  Periodic tiles pair slots (2j, 2j+1) of one warp, held by
// lanes pair_xor apart (1 when a thread holds a point, TPP when TPP consecutive
// threads share one), so every lane of the warp must call this.
__device__ __forceinline__ bool residual_and_seeds(const KParams &p, const Tile &T,
                                                   const PointIn &pt, int slot, const float (&u)[4],
                                                   float (&ub)[4], float &lp, int pair_xor = 1,
                                                   bool write = true) {
  const int inst = T.inst;
  const float beta = __ldg(p.beta + inst), nu = __ldg(p.nu + inst), rho = __ldg(p.rho + inst);
  ub[0] = ub[1] = ub[2] = ub[3] = 0.0f;
  lp = 0.0f;
  const bool mse = p.loss == LRNR_LOSS_MSE;
  if (T.kind == KIND_INT) {
    const float R = u[1] + beta * u[2] - nu * u[3] - rho * u[0] * (1.0f - u[0]);
    if (!p.grad) {
      if (pt.act && write) {
        const int64_t g = T.first + slot;
        if (p.u) p.u[g] = u[0];
        if (p.ut) p.ut[g] = u[1];
        if (p.ux) p.ux[g] = u[2];
        if (p.uxx) p.uxx[g] = u[3];
        if (p.res) p.res[g] = R;
      }
      return false;
    }
    const float n = mse_count(p, inst, 0, p.int_off);
    float gR;
    if (mse) { lp = p.w[0] * R * R / n; gR = 2.0f * p.w[0] * R / n; }
    else { lp = p.w[0] * fabsf(R); gR = p.w[0] * (float)((R > 0.0f) - (R < 0.0f)); }
    if (!pt.act) { lp = 0.0f; gR = 0.0f; }
    ub[0] = -rho * (1.0f - 2.0f * u[0]) * gR;
    ub[1] = gR;
    ub[2] = beta * gR;
    ub[3] = -nu * gR;
  } else if (T.kind == KIND_IC) {
    const float B = u[0] - sinf(pt.x);
    if (!p.grad) {
      if (pt.act && write && p.res_ic) p.res_ic[T.first + slot] = B;
      return false;
    }
    const float n = mse_count(p, inst, 1, p.ic_off);
    float gB;
    if (mse) { lp = p.w[1] * B * B / n; gB = 2.0f * p.w[1] * B / n; }
    else { lp = p.w[1] * fabsf(B); gB = p.w[1] * (float)((B > 0.0f) - (B < 0.0f)); }
    if (!pt.act) { lp = 0.0f; gB = 0.0f; }
    ub[0] = gB;
  } else {
    const float uo = __shfl_xor_sync(0xffffffffu, u[0], pair_xor);
    const float B = pt.side ? (uo - u[0]) : (u[0] - uo);
    if (!p.grad) {
      if (pt.act && write && pt.side == 0 && p.res_bc) p.res_bc[T.first + (slot >> 1)] = B;
      return false;
    }
    const float n = mse_count(p, inst, 2, p.bc_off);
    float gB;
    if (mse) { lp = p.w[2] * B * B / n; gB = 2.0f * p.w[2] * B / n; }
    else { lp = p.w[2] * fabsf(B); gB = p.w[2] * (float)((B > 0.0f) - (B < 0.0f)); }
    if (!pt.act) { lp = 0.0f; gB = 0.0f; }
    if (pt.side) lp = 0.0f;
    ub[0] = pt.side ? -gB : gB;
  }
  return true;
}

}  // namespace lrnr
