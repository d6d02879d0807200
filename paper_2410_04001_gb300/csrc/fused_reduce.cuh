// Fixed-order reduction and Adam inside a FastLRNR tile kernel (KParams::fused_red):
// each tile's partial row is summed with the rest of its group of kRedGroup tiles by
// the CTA that completes the group (ticket), and each instance by the CTA that
// completes its last group, so the sums run in tile order whatever the CTAs' timing.
// No CTA waits on another.  Used by the rank-r and the reduced-coordinate kernels,
// which share the partial-row layout (loss, dL/ds by padded rank, dL/dbhat).
#pragma once
#include "lrnr_internal.cuh"
#include "simt_common.cuh"

namespace lrnr {

// Instance owning tile t: the largest i with toff[i] <= t.
__device__ __forceinline__ int instance_of_tile(const int32_t *toff, int n_inst, int t) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Entry j summed over rows a..b-1 of a row matrix with row length P, in row order.
// The rows were written by other CTAs, so they are read through L2; the loads of a
// chunk of up to kRedGroup rows are all issued before the additions.
__device__ __forceinline__ float rows_sum(const float *src, int P, int j, int a, int b) {
  float acc = 0.0f;
  for (int c = a; c < b; c += kRedGroup) {
    float v[kRedGroup];
#pragma unroll
    for (int k = 0; k < kRedGroup; ++k)
      v[k] = (c + k < b) ? __ldcg(src + (int64_t)(c + k) * P + j) : 0.0f;
#pragma unroll
    for (int k = 0; k < kRedGroup; ++k) acc += v[k];
  }
  return acc;
}

// Finish instance i: add its group rows in group order, then either write loss,
// dL/ds and dL/db (scattered to the EIM rows; dL/db zeroed beforehand by the host),
// or apply Adam to the instance's s (Sec. 4) with the l1 locality subgradient of
// Eq. 3.7 and write the loss.  An instance without tiles has a zero gradient.  In
// Adam mode the CTA finishing the last instance advances the step counter.  All
// threads of the CTA; `buf` holds P floats, `wsum` NT/32 floats (shared memory).
static __device__ void fast_finish_instance(const KParams &p, int i, const int32_t *toff,
                                            float *buf, float *wsum, int64_t kstep) {
  const int tid = threadIdx.x, NT = blockDim.x, P = p.P;
  const int t0 = toff[i], t1 = toff[i + 1];
  for (int j = tid; j < P; j += NT)
    buf[j] = t1 > t0 ? rows_sum(p.gpart, P, j, t0 / kRedGroup + i, (t1 - 1) / kRedGroup + i + 1)
                     : 0.0f;
  __syncthreads();
  const int DB0 = partial_db0(p.L, p.RM);
  if (!p.adam_s) {
    for (int j = tid; j < P; j += NT) {
      const float v = buf[j];
      if (j == 0) {
        if (p.loss_out) p.loss_out[i] = v;
      } else if (j < DB0) {
        const int l = (j - 1) / p.RM, k = (j - 1) % p.RM;
        if (k < p.r[l]) p.dL_ds[(int64_t)i * p.sum_r + p.roff[l] + k] = v;
      } else if (p.dL_db) {
        const int jj = j - DB0;
        float *db = p.dL_db + (int64_t)i * p.sum_m;
        if (jj == p.L * p.RH) {
          db[p.L * p.M] = v;
        } else if (jj < p.L * p.RH) {
          const int row = p.rows[jj];   // [l][RH]: jj = l * RH + slot
          if (row >= 0) db[(jj / p.RH) * p.M + row] = v;
        }
      }
    }
    __syncthreads();
    return;
  }
  const float bc1 = 1.0f - powf(p.b1, (float)kstep);
  const float bc2 = 1.0f - powf(p.b2, (float)kstep);
  float loc = 0.0f;
  for (int j = 1 + tid; j < DB0; j += NT) {
    const int l = (j - 1) / p.RM, k = (j - 1) % p.RM;
    if (k >= p.r[l]) continue;
    const int64_t o = (int64_t)i * p.sum_r + p.roff[l] + k;
    const float sv = p.adam_s[o];
    float gr = buf[j];
    if (p.anchor) {
      const float d = sv - p.anchor[o];
      loc += p.lam * fabsf(d);
      gr += p.lam * (float)((d > 0.0f) - (d < 0.0f));
    }
    const float mv = p.b1 * p.adam_m[o] + (1.0f - p.b1) * gr;
    const float vv = p.b2 * p.adam_v[o] + (1.0f - p.b2) * gr * gr;
    p.adam_m[o] = mv;
    p.adam_v[o] = vv;
    p.adam_s[o] = sv - p.lr * (mv / bc1) / (sqrtf(vv / bc2) + p.eps);
  }
  loc = warp_sum(loc);
  if ((tid & 31) == 0) wsum[tid >> 5] = loc;
  __syncthreads();
  if (tid == 0) {
    float lt = 0.0f;
    for (int w = 0; w < NT / 32; ++w) lt += wsum[w];
    if (p.loss_out) p.loss_out[i] = buf[0] + lt;
    __threadfence();
    int *tk = p.tickets + p.n_groups + p.n_inst;
    if (atomicAdd(tk, 1) == p.n_inst - 1) {
      *tk = 0;
      *p.step = kstep;
    }
  }
  __syncthreads();
}

// After a tile's partial row is written (all threads): take the tile's group
// ticket.  The CTA completing the group sums the group's rows of each instance it
// holds, in tile order, into that instance's group row gpart[g + i], and takes the
// instance's ticket; the CTA completing an instance's last group finishes it.
// Tickets are reset by the CTA that completes them, ready for the next launch.
static __device__ void fast_tile_done(const KParams &p, int tile, int ntiles, const int32_t *toff,
                                      float *buf, float *wsum, int *flag, int64_t kstep) {
  const int tid = threadIdx.x, NT = blockDim.x, P = p.P;
  const int g = tile / kRedGroup;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const int gsize = min(kRedGroup, ntiles - g * kRedGroup);
    const int last = atomicAdd(p.tickets + g, 1) == gsize - 1;
    if (last) p.tickets[g] = 0;
    flag[0] = last;
  }
  __syncthreads();
  if (!flag[0]) return;
  __threadfence();
  const int ta = g * kRedGroup, tb = min(ntiles, ta + kRedGroup);
  const int i0 = instance_of_tile(toff, p.n_inst, ta);
  const int i1 = instance_of_tile(toff, p.n_inst, tb - 1);
  for (int i = i0; i <= i1; ++i) {
    const int a = max(ta, toff[i]), b = min(tb, toff[i + 1]);
    if (a >= b) continue;   // an instance without tiles (finished at kernel start)
    for (int j = tid; j < P; j += NT)
      p.gpart[(int64_t)(g + i) * P + j] = rows_sum(p.partial, P, j, a, b);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const int ng = (toff[i + 1] - 1) / kRedGroup - toff[i] / kRedGroup + 1;
      const int last = atomicAdd(p.tickets + p.n_groups + i, 1) == ng - 1;
      if (last) p.tickets[p.n_groups + i] = 0;
      flag[0] = last;
    }
    __syncthreads();
    if (flag[0]) {
      __threadfence();
      fast_finish_instance(p, i, toff, buf, wsum, kstep);
    }
    __syncthreads();
  }
}

}  // namespace lrnr
