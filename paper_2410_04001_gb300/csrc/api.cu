// C ABI of liblrnr.so: argument validation, model and workspace management, and
// the launch sequences of each entry point.  See include/lrnr.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lrnr_internal.cuh"

namespace lrnr {
cudaError_t launch_eim_reduce_f64(const double *Xi, const int32_t *rows, int rh, int M,
                                  const double *U, const double *b, const double *Vn, int rin,
                                  int rout, double *out, int *status, cudaStream_t st);
cudaError_t launch_snapshots_f64(const double *w64, int L, int M, const int *r_dev,
                                 const int64_t *offs_dev, int layer, int64_t n_pts,
                                 const double *x, const double *t, int n_s, const double *s,
                                 int sum_r, double *out, cudaStream_t st);
int full_tc_supported(int L, int M, int RM, int NC, int prec);
size_t full_tc_pack_bytes(int L, int M, int RM, int NC, int tf32);
void full_tc_pack(int L, int M, int RM, int NC, const std::vector<std::vector<double>> &U,
                  const std::vector<std::vector<double>> &V, const std::vector<std::vector<double>> &b,
                  const int *r, std::vector<unsigned char> &out, int tf32);
int full_tc_nt();
int full_tc_nc(int RM, int prec);
size_t full_tc_scratch_floats(int L, int RM, int grid);
cudaError_t launch_adam_update(int n_inst, int sum_r, const float *g, float *s, float *m, float *v,
                               int64_t *step, float lr, float b1, float b2, float eps, float lam,
                               const float *anchor, const float *loss_in, float *loss_out,
                               cudaStream_t st);
}  // namespace lrnr

using namespace lrnr;

struct lrnr_model {
  int device = 0;
  int num_sms = 1;
  int L = 0, M = 0;
  int r[LMAX + 1] = {0};
  int roff[LMAX + 2] = {0};
  int sum_r = 0, sum_m = 0;
  int RM = 8;
  std::vector<std::vector<double>> U, V, b;   // host FP64 bases
  float *full_pack = nullptr;                  // FP32, full form
  double *w64 = nullptr;                       // FP64 bases (snapshots)
  int *r_dev = nullptr;
  int64_t *offs_dev = nullptr;
  void *tc_pack = nullptr;                     // tensor-core operand pack (full form)
  void *tc16_pack = nullptr;                   // the same in 16-column chunks (split-BF16, rank 32)
  void *ftc_pack = nullptr;                    // tensor-core pack of the reduced network
  void *tf_pack = nullptr;                     // the same two packs in TF32
  void *ftf_pack = nullptr;
  float *fastk_pack = nullptr;                 // FP32 reduced pack for ranks 32 / 64 (fastk.cu)
  int ftc_nc = 16;                             // its chunk width (32 at rank 64)
  // reduced layers (host, FP64): Uh [rh][r_l], bh [rh], Vh [rh][r_{l+1}], rows [rh]
  int rhat[LMAX] = {0};
  std::vector<std::vector<double>> Uh, bh, Vh;
  std::vector<std::vector<int32_t>> rows;
  bool fast_dirty = true;
  int fRM = 0, fRH = 0;
  float *fast_pack = nullptr;
  int32_t *rows_dev = nullptr;
  int *status_dev = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // optional CUDA-event timing of the tile kernels (one event pair per launch);
  // pairs recorded while a stream was being captured belong to the CUDA graph and
  // are re-recorded by each replay, so they are kept until timing is reset
  bool timing = false;
  std::vector<cudaEvent_t> ev_start, ev_stop;
  size_t ev_used = 0;
  std::vector<cudaEvent_t> cap_start, cap_stop;
  // launch-shape overrides per (form, precision): points per tile, CTAs per SM cap
  uint32_t wait_limit = 1u << 20;              // mbarrier poll cap of the tensor-core kernel
  int tune_nt[2][4] = {{0}};
  int tune_cta[2][4] = {{0}};
  // tickets of the two-level Adam reduction and of the FastLRNR kernel's fused
  // reduction (zero between calls; every ticket is reset by the CTA completing it)
  int *adam_cnt = nullptr;
  int adam_cnt_n = 0;
};

namespace {

lrnr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LRNR_OK;
  if (e == cudaErrorMemoryAllocation) return LRNR_ENOMEM;
  return LRNR_ECUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

int pad_rank(int r) { return r <= 8 ? 8 : (r <= 16 ? 16 : (r <= 32 ? 32 : 64)); }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

// Available (RM, RH) instantiations of the FastLRNR kernel, cheapest first.
const int kFastPairs[][2] = {{8, 8}, {16, 8}, {8, 16}, {16, 16}};

int64_t max_tiles(int64_t n_int, int64_t n_ic, int64_t n_bc, int n_inst, int nt) {
  return (n_int + nt - 1) / nt + (n_ic + nt - 1) / nt + (n_bc + nt / 2 - 1) / (nt / 2) +
         3 * (int64_t)n_inst;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Precisions that run on the tensor cores.
bool tc_prec(lrnr_precision prec) {
  return prec == LRNR_BF16 || prec == LRNR_BF16X3 || prec == LRNR_TF32;
}

lrnr_status ensure_ws(lrnr_model *m, size_t need, cudaStream_t st) {
  if (m->ws_bytes >= need) return LRNR_OK;
  if (capturing(st)) return LRNR_ENOTREADY;
  if (m->ws) {
    CK(cudaStreamSynchronize(st));
    CK(cudaFree(m->ws));
    m->ws = nullptr;
    m->ws_bytes = 0;
  }
  CK(cudaMalloc(&m->ws, need));
  m->ws_bytes = need;
  return LRNR_OK;
}

// Zeroed ticket counters, at least n of them (grown outside stream capture only).
lrnr_status ensure_tickets(lrnr_model *m, int64_t n, cudaStream_t st) {
  if (m->adam_cnt_n >= n) return LRNR_OK;
  if (capturing(st)) return LRNR_ENOTREADY;
  if (n > INT32_MAX) return LRNR_EINVAL;
  if (m->adam_cnt) {
    if (st) CK(cudaStreamSynchronize(st));
    else CK(cudaDeviceSynchronize());
    CK(cudaFree(m->adam_cnt));
    m->adam_cnt = nullptr;
    m->adam_cnt_n = 0;
  }
  CK(cudaMalloc(&m->adam_cnt, sizeof(int) * (size_t)n));
  CK(cudaMemset(m->adam_cnt, 0, sizeof(int) * (size_t)n));
  m->adam_cnt_n = (int)n;
  return LRNR_OK;
}

lrnr_status build_fast_pack(lrnr_model *m) {
  if (!m->fast_dirty) return LRNR_OK;
  int need_rh = 0;
  for (int l = 0; l < m->L; ++l) {
    if (m->rhat[l] <= 0) return LRNR_ENOTREADY;
    need_rh = std::max(need_rh, m->rhat[l]);
  }
  int RMp = 0, RHp = 0;
  for (auto &pr : kFastPairs)
    if (pr[0] >= m->RM && pr[1] >= need_rh) { RMp = pr[0]; RHp = pr[1]; break; }
  // no FP32 instantiation for these ranks: only the tensor-core form of the reduced
  // network is built (RM = the model's padded rank)
  const bool fp32_ok = RMp != 0;
  if (!fp32_ok) {
    RMp = m->RM;
    RHp = need_rh <= 8 ? 8 : (need_rh <= 16 ? 16 : 32);
  }
  const int L = m->L;
  const int LS = fast_layer_floats(RMp, RHp);
  std::vector<float> pk((size_t)fast_pack_floats(L, RMp, RHp), 0.0f);
  std::vector<int32_t> rw((size_t)L * RHp, -1);
  for (int l = 0; l < L; ++l) {
    const int rh = m->rhat[l], rin = m->r[l], rout = m->r[l + 1];
    float *Uh = pk.data() + (size_t)l * LS, *bh = Uh + RHp * RMp, *Vh = bh + RHp;
    for (int a = 0; a < rh; ++a) {
      for (int k = 0; k < rin; ++k) Uh[a * RMp + k] = (float)m->Uh[l][(size_t)a * rin + k];
      bh[a] = (float)m->bh[l][a];
      for (int k = 0; k < rout; ++k) Vh[a * RMp + k] = (float)m->Vh[l][(size_t)a * rout + k];
      rw[(size_t)l * RHp + a] = m->rows[l][a];
    }
  }
  float *tail = pk.data() + (size_t)L * LS;
  for (int k = 0; k < m->r[0]; ++k) {
    tail[k] = (float)m->V[0][k];                  // V^0 row x
    tail[R1 + k] = (float)m->V[0][m->r[0] + k];   // V^0 row t
  }
  tail[2 * R1] = (float)m->U[L][0];
  tail[2 * R1 + 1] = (float)m->b[L][0];
  if (m->fast_pack) cudaFree(m->fast_pack);
  if (m->fastk_pack) cudaFree(m->fastk_pack);
  if (m->rows_dev) cudaFree(m->rows_dev);
  m->fast_pack = nullptr;
  m->fastk_pack = nullptr;
  m->rows_dev = nullptr;
  if (fp32_ok) {
    CK(cudaMalloc(&m->fast_pack, pk.size() * sizeof(float)));
    CK(cudaMemcpy(m->fast_pack, pk.data(), pk.size() * sizeof(float), cudaMemcpyHostToDevice));
  } else if ((RMp == 32 || RMp == 64) && RHp <= 16) {
    // ranks above the rank-r jet kernel: the same pack for the reduced-coordinate kernel
    CK(cudaMalloc(&m->fastk_pack, pk.size() * sizeof(float)));
    CK(cudaMemcpy(m->fastk_pack, pk.data(), pk.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  CK(cudaMalloc(&m->rows_dev, rw.size() * sizeof(int32_t)));
  CK(cudaMemcpy(m->rows_dev, rw.data(), rw.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  m->fRM = RMp;
  m->fRH = RHp;
  // The reduced network is itself an LRNR of width RHp with bases (Uhat, Vhat, bhat)
  // (Eq. 2.8): pack it for the tensor-core kernel in 16-column chunks, rows past
  // rhat zero (they contribute nothing and get a zero dL/db).
  if (m->ftc_pack) cudaFree(m->ftc_pack);
  if (m->ftf_pack) cudaFree(m->ftf_pack);
  m->ftc_pack = nullptr;
  m->ftf_pack = nullptr;
  const int RMt = std::max(16, RMp);
  m->ftc_nc = RMt <= 32 ? 16 : 32;
  if (full_tc_supported(L, RHp, RMt, m->ftc_nc, LRNR_BF16)) {
    std::vector<std::vector<double>> Ur(L + 1), Vr(L + 1), br(L + 1);
    Vr[0] = m->V[0];
    Ur[L] = m->U[L];
    br[L] = m->b[L];
    for (int l = 0; l < L; ++l) {
      const int rh = m->rhat[l], rin = m->r[l], rout = m->r[l + 1];
      Ur[l].assign((size_t)RHp * rin, 0.0);
      br[l].assign(RHp, 0.0);
      Vr[l + 1].assign((size_t)RHp * rout, 0.0);
      for (int a = 0; a < rh; ++a) {
        for (int k = 0; k < rin; ++k) Ur[l][(size_t)a * rin + k] = m->Uh[l][(size_t)a * rin + k];
        br[l][a] = m->bh[l][a];
        for (int k = 0; k < rout; ++k) Vr[l + 1][(size_t)a * rout + k] = m->Vh[l][(size_t)a * rout + k];
      }
    }
    std::vector<unsigned char> tp;
    full_tc_pack(L, RHp, RMt, m->ftc_nc, Ur, Vr, br, m->r, tp, 0);
    CK(cudaMalloc(&m->ftc_pack, tp.size()));
    CK(cudaMemcpy(m->ftc_pack, tp.data(), tp.size(), cudaMemcpyHostToDevice));
    if (full_tc_supported(L, RHp, RMt, m->ftc_nc, LRNR_TF32)) {
      full_tc_pack(L, RHp, RMt, m->ftc_nc, Ur, Vr, br, m->r, tp, 1);
      CK(cudaMalloc(&m->ftf_pack, tp.size()));
      CK(cudaMemcpy(m->ftf_pack, tp.data(), tp.size(), cudaMemcpyHostToDevice));
    }
  }
  m->fast_dirty = false;
  return LRNR_OK;
}

lrnr_status check_batch(const lrnr_model *m, const lrnr_batch *bt) {
  if (!bt || bt->n_inst < 1 || bt->n_int < 0 || bt->n_ic < 0 || bt->n_bc < 0) return LRNR_EINVAL;
  if (!bt->beta || !bt->nu || !bt->rho || !bt->int_off || !bt->ic_off || !bt->bc_off)
    return LRNR_EINVAL;
  if (bt->n_int > 0 && (!bt->x_int || !bt->t_int)) return LRNR_EINVAL;
  if (bt->n_ic > 0 && !bt->x_ic) return LRNR_EINVAL;
  if (bt->n_bc > 0 && !bt->t_bc) return LRNR_EINVAL;
  (void)m;
  return LRNR_OK;
}

// Common set-up of a residual / gradient pass.
struct Pass {
  KParams p;
  int grid_cap;
  int nb_entries;     // partial entries beyond dL/ds (dL/db block)
  float *gsum = nullptr;   // Adam group rows (spinprop_step)
};

lrnr_status prepare(lrnr_model *m, lrnr_form form, lrnr_precision prec, const lrnr_batch *bt,
                    bool grad, const float *s, cudaStream_t st, Pass &ps, bool adam = false) {
  lrnr_status rc = check_batch(m, bt);
  if (rc != LRNR_OK) return rc;
  if (!s) return LRNR_EINVAL;
  KParams &p = ps.p;
  std::memset(&p, 0, sizeof(p));
  p.L = m->L;
  p.M = m->M;
  p.n_inst = bt->n_inst;
  for (int l = 0; l <= m->L; ++l) p.r[l] = m->r[l];
  for (int l = 0; l <= m->L + 1; ++l) p.roff[l] = m->roff[l];
  p.sum_r = m->sum_r;
  p.beta = bt->beta; p.nu = bt->nu; p.rho = bt->rho; p.s = s;
  p.int_off = bt->int_off; p.ic_off = bt->ic_off; p.bc_off = bt->bc_off;
  p.x_int = bt->x_int; p.t_int = bt->t_int; p.x_ic = bt->x_ic; p.t_bc = bt->t_bc;
  p.tot[0] = bt->n_int; p.tot[1] = bt->n_ic; p.tot[2] = bt->n_bc;
  p.norm = bt->norm;
  p.grad = grad ? 1 : 0;
  p.status = m->status_dev;
  if (form == LRNR_FAST && tc_prec(prec)) {
    // the reduced network on the tensor cores: an LRNR of width RH
    rc = build_fast_pack(m);
    if (rc != LRNR_OK) return rc;
    if (!(prec == LRNR_TF32 ? m->ftf_pack : m->ftc_pack) ||
        !full_tc_supported(m->L, m->fRH, std::max(16, m->fRM), m->ftc_nc, prec))
      return LRNR_ENOTSUP;
    p.RM = std::max(16, m->fRM);
    p.RH = m->fRH;
    p.M = m->fRH;
    for (int l = 0; l < m->L; ++l) p.rh[l] = m->rhat[l];
    p.pack = nullptr;
    p.nt = full_tc_nt();
    ps.nb_entries = m->L * p.RH + 1;
  } else if (form == LRNR_FAST) {
    if (prec != LRNR_FP32) return LRNR_ENOTSUP;
    rc = build_fast_pack(m);
    if (rc != LRNR_OK) return rc;
    p.RM = m->fRM;
    p.RH = m->fRH;
    for (int l = 0; l < m->L; ++l) p.rh[l] = m->rhat[l];
    if (!m->fast_pack) {
      // ranks above the rank-r jet kernel (padded 32 / 64): the reduced-coordinate
      // kernel, when the reduced width allows it
      const int P = partial_len(m->L, p.RM, m->L * p.RH + 1);
      if (!m->fastk_pack || !fastk_supported(m->L, p.RM, p.RH, P, 0)) return LRNR_ENOTSUP;
      p.fastk = 1;
      p.pack = m->fastk_pack;
      // the kernel computes its tile offsets when they fit in shared memory
      p.fused_tiles =
          bt->n_inst <= 4096 && fastk_supported(m->L, p.RM, p.RH, P, bt->n_inst) ? 1 : 0;
      p.nt = fastk_nt();
    } else {
      p.pack = m->fast_pack;
      p.fused_tiles = bt->n_inst <= 4096 ? 1 : 0;   // the kernel computes its tile offsets
      p.nt = fast_choose_nt(m->L, p.RM, p.RH, partial_len(m->L, p.RM, m->L * p.RH + 1));
      if (!p.nt) return LRNR_ENOTSUP;
      const int tn = m->tune_nt[LRNR_FAST][prec];
      if (tn && fast_smem_bytes(m->L, p.RM, p.RH, tn, partial_len(m->L, p.RM, m->L * p.RH + 1)) <=
                    (size_t)kSmemBudget)
        p.nt = tn;
    }
    ps.nb_entries = m->L * p.RH + 1;
  } else if (form == LRNR_FULL) {
    p.RM = m->RM;
    p.RH = 0;
    if (prec == LRNR_FP32) {
      p.pack = m->full_pack;
      if (p.RM >= 32) {
        // padded ranks 32 / 64: RM / 16 threads share a point (full_fp32_sliced.cu)
        if (full_fp32_sl_smem_bytes(m->L, m->M, p.RM) > (size_t)kSmemBudget) return LRNR_ENOTSUP;
        p.nt = full_fp32_sl_nt(p.RM);
      } else {
        p.nt = full_fp32_choose_nt(m->L, p.RM, partial_len(m->L, p.RM, m->L * m->M + 1));
        if (!p.nt) return LRNR_ENOTSUP;
        const int tn = m->tune_nt[LRNR_FULL][prec];
        if ((tn == 32 || tn == 64) &&
            full_fp32_smem_bytes(m->L, p.RM, tn, partial_len(m->L, p.RM, m->L * m->M + 1)) <=
                (size_t)kSmemBudget)
          p.nt = tn;
      }
    } else if (tc_prec(prec)) {
      p.RM = std::max(16, m->RM);   // tensor-core tiles need K and N of at least 16
      const int nc = full_tc_nc(p.RM, prec);
      const void *pk = prec == LRNR_TF32 ? m->tf_pack : (nc == 16 ? m->tc16_pack : m->tc_pack);
      if (!pk || !full_tc_supported(m->L, m->M, p.RM, nc, prec)) return LRNR_ENOTSUP;
      p.pack = nullptr;
      p.nt = full_tc_nt();
    } else {
      return LRNR_ENOTSUP;
    }
    ps.nb_entries = m->L * m->M + 1;
  } else {
    return LRNR_EINVAL;
  }
  p.P = grad ? partial_len(m->L, p.RM, ps.nb_entries - 1) : 0;
  const int64_t tiles = max_tiles(bt->n_int, bt->n_ic, bt->n_bc, bt->n_inst, p.nt);
  if (tiles > INT32_MAX / 2) return LRNR_EINVAL;
  const bool tc = tc_prec(prec);
  ps.grid_cap = (int)std::min<int64_t>(tiles, INT32_MAX);
  size_t scr_bytes = 0;
  if (tc) {
    // one CTA per SM with 32-column chunks, two with 16-column chunks (reduced form)
    const int per_sm = (form == LRNR_FAST && m->ftc_nc == 16) ? 2 : 1;
    ps.grid_cap = (int)std::min<int64_t>(tiles, per_sm * (int64_t)m->num_sms);
    scr_bytes = full_tc_scratch_floats(m->L, p.RM, ps.grid_cap) * sizeof(float);
  } else if (form == LRNR_FAST) {
    // the FastLRNR kernel keeps layer inputs in a per-CTA scratch: size the grid first
    // 255-register build (2 CTAs/SM) unless the tuning asks for 3 CTAs per SM
    p.fast_regs = m->tune_cta[LRNR_FAST][prec] >= 3 ? 3 : 2;
    int per_sm = fast_ctas_per_sm(p);
    if (m->tune_cta[LRNR_FAST][prec] > 0) per_sm = std::min(per_sm, m->tune_cta[LRNR_FAST][prec]);
    ps.grid_cap = (int)std::min<int64_t>(tiles, (int64_t)per_sm * m->num_sms);
    if (grad)
      scr_bytes = (p.fastk ? fastk_scratch_floats(m->L, p.RH, ps.grid_cap)
                           : fast_scratch_floats(m->L, p.RM, p.RH, p.nt, ps.grid_cap)) *
                  sizeof(float);
  } else {
    // the FP32 full-width kernel also keeps layer inputs in a per-CTA scratch
    int per_sm = full_fp32_ctas_per_sm(p);
    if (m->tune_cta[LRNR_FULL][prec] > 0) per_sm = std::min(per_sm, m->tune_cta[LRNR_FULL][prec]);
    ps.grid_cap = (int)std::min<int64_t>(tiles, (int64_t)per_sm * m->num_sms);
    if (grad)
      scr_bytes = (p.RM >= 32 ? full_fp32_sl_scratch_floats(m->L, p.RM, ps.grid_cap)
                              : full_fp32_scratch_floats(m->L, p.RM, p.nt, ps.grid_cap)) *
                  sizeof(float);
  }
  // Batches whose tiles fit in one round of the FastLRNR grid (2 CTAs per SM) are
  // reduced inside the kernel (group rows + tickets): one launch instead of two.
  const bool fused_red = grad && form == LRNR_FAST && prec == LRNR_FP32 &&
                         tiles <= 2 * (int64_t)m->num_sms;
  if (fused_red) {
    p.fast_regs = 2;
    ps.grid_cap = (int)std::min<int64_t>(tiles, 2 * (int64_t)m->num_sms);
    scr_bytes = (p.fastk ? fastk_scratch_floats(m->L, p.RH, ps.grid_cap)
                         : fast_scratch_floats(m->L, p.RM, p.RH, p.nt, ps.grid_cap)) *
                sizeof(float);
  }
  const int64_t n_groups = (tiles + kRedGroup - 1) / kRedGroup;
  const size_t off_part = align256(sizeof(int32_t) * (size_t)(bt->n_inst + 1));
  const size_t part_bytes = grad ? align256((size_t)tiles * p.P * sizeof(float)) : 0;
  const size_t scr_al = align256(scr_bytes);
  const size_t adam_bytes =
      adam && !fused_red ? align256(adam_group_floats(bt->n_inst, m->L, p.RM) * sizeof(float)) : 0;
  const size_t gpart_bytes =
      fused_red ? align256((size_t)(n_groups + bt->n_inst) * p.P * sizeof(float)) : 0;
  rc = ensure_ws(m, off_part + part_bytes + scr_al + adam_bytes + gpart_bytes, st);
  if (rc != LRNR_OK) return rc;
  if (fused_red || adam) {
    rc = ensure_tickets(m, fused_red ? n_groups + bt->n_inst + 1 : bt->n_inst, st);
    if (rc != LRNR_OK) return rc;
  }
  char *ws = static_cast<char *>(m->ws);
  p.tile_off = reinterpret_cast<int32_t *>(ws);
  p.partial = reinterpret_cast<float *>(ws + off_part);
  p.scratch = scr_bytes ? reinterpret_cast<float *>(ws + off_part + part_bytes) : nullptr;
  ps.gsum = adam_bytes ? reinterpret_cast<float *>(ws + off_part + part_bytes + scr_al) : nullptr;
  if (fused_red) {
    p.fused_red = 1;
    p.n_groups = (int)n_groups;
    p.gpart = reinterpret_cast<float *>(ws + off_part + part_bytes + scr_al + adam_bytes);
    p.tickets = m->adam_cnt;
    p.rows = m->rows_dev;
    p.sum_m = m->sum_m;
  }
  p.max_wait = m->wait_limit;
  p.loss = LRNR_LOSS_MSE;
  p.w[0] = p.w[1] = p.w[2] = 1.0f;
  return LRNR_OK;
}

lrnr_status run_main(lrnr_model *m, lrnr_form form, lrnr_precision prec, Pass &ps,
                     cudaStream_t st) {
  KParams &p = ps.p;
  if (!p.fused_tiles) CK(launch_tile_offsets(p, const_cast<int32_t *>(p.tile_off), st));
  cudaEvent_t e1 = nullptr, e2 = nullptr;
  const bool cap = m->timing && capturing(st);
  if (cap) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    m->cap_start.push_back(a);
    m->cap_stop.push_back(b);
    e1 = a;
    e2 = b;
    CK(cudaEventRecordWithFlags(e1, st, cudaEventRecordExternal));
  } else if (m->timing) {
    if (m->ev_used == m->ev_start.size()) {
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      m->ev_start.push_back(a);
      m->ev_stop.push_back(b);
    }
    e1 = m->ev_start[m->ev_used];
    e2 = m->ev_stop[m->ev_used];
    ++m->ev_used;
    CK(cudaEventRecord(e1, st));
  }
  if (tc_prec(prec)) {
    const bool fast = form == LRNR_FAST;
    const int nc = fast ? m->ftc_nc : full_tc_nc(p.RM, prec);
    const void *pk = prec == LRNR_TF32 ? (fast ? m->ftf_pack : m->tf_pack)
                                       : (fast ? m->ftc_pack : (nc == 16 ? m->tc16_pack : m->tc_pack));
    CK(launch_full_tc(p, pk, (int)prec, nc, ps.grid_cap, st));
  } else if (form == LRNR_FAST) {
    CK(launch_fast(p, ps.grid_cap, st));
  } else {
    CK(launch_full_fp32(p, ps.grid_cap, st));
  }
  if (e2) CK(cap ? cudaEventRecordWithFlags(e2, st, cudaEventRecordExternal) : cudaEventRecord(e2, st));
  return LRNR_OK;
}

}  // namespace

extern "C" {

const char *lrnr_status_string(lrnr_status s) {
  switch (s) {
    case LRNR_OK: return "ok";
    case LRNR_EINVAL: return "invalid argument";
    case LRNR_ENOMEM: return "device allocation failed";
    case LRNR_ECUDA: return "CUDA error";
    case LRNR_ESINGULAR: return "singular interpolation block P^T Xi";
    case LRNR_EEARLYSTOP: return "EIM stopped early";
    case LRNR_ETIMEOUT: return "device wait reached its iteration cap";
    case LRNR_ENOTREADY: return "not ready (FastLRNR layers not selected, or workspace too small while capturing)";
    case LRNR_ENONFINITE: return "non-finite value met by a kernel";
    case LRNR_ENOTSUP: return "form / precision not supported for this model";
    case LRNR_ETOOBIG: return "batch exceeds the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

lrnr_status lrnr_build(int L, int M, const int *r, const double *const *U, const double *const *V,
                       const double *const *b, lrnr_model **out) {
  if (!out) return LRNR_EINVAL;
  *out = nullptr;
  if (L < 1 || L > LMAX || M < 1 || M > 4096 || !r || !U || !V || !b) return LRNR_EINVAL;
  if (r[0] < 1 || r[0] > R1 || r[L] != 1) return LRNR_EINVAL;
  for (int l = 1; l < L; ++l)
    if (r[l] < 1 || r[l] > RMAX) return LRNR_EINVAL;
  for (int l = 0; l <= L; ++l)
    if (!U[l] || !V[l] || !b[l]) return LRNR_EINVAL;
  lrnr_model *m = new (std::nothrow) lrnr_model();
  if (!m) return LRNR_ENOMEM;
  cudaGetDevice(&m->device);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  m->L = L;
  m->M = M;
  int rmid = 1;
  for (int l = 0; l <= L; ++l) {
    m->r[l] = r[l];
    m->roff[l + 1] = m->roff[l] + r[l];
    if (l > 0 && l < L) rmid = std::max(rmid, r[l]);
  }
  m->sum_r = m->roff[L + 1];
  m->sum_m = L * M + 1;
  m->RM = pad_rank(rmid);
  m->U.resize(L + 1);
  m->V.resize(L + 1);
  m->b.resize(L + 1);
  m->Uh.resize(L);
  m->bh.resize(L);
  m->Vh.resize(L);
  m->rows.resize(L);
  auto width = [&](int l) { return l < 0 ? 2 : (l < L ? M : 1); };
  for (int l = 0; l <= L; ++l) {
    const int mo = width(l), mi = width(l - 1);
    m->U[l].assign(U[l], U[l] + (size_t)mo * r[l]);
    m->V[l].assign(V[l], V[l] + (size_t)mi * r[l]);
    m->b[l].assign(b[l], b[l] + mo);
    for (double v : m->U[l]) if (!std::isfinite(v)) { delete m; return LRNR_EINVAL; }
    for (double v : m->V[l]) if (!std::isfinite(v)) { delete m; return LRNR_EINVAL; }
    for (double v : m->b[l]) if (!std::isfinite(v)) { delete m; return LRNR_EINVAL; }
  }
  // FP32 full pack
  const int RM = m->RM;
  const int64_t LS = full_layer_floats(M, RM);
  std::vector<float> pk((size_t)full_pack_floats(L, M, RM), 0.0f);
  for (int l = 0; l < L; ++l) {
    float *Ul = pk.data() + l * LS, *bl = Ul + (size_t)M * RM, *Vn = bl + pad4(M);
    const int rin = r[l], rout = r[l + 1];
    for (int i = 0; i < M; ++i) {
      for (int k = 0; k < rin; ++k) Ul[(size_t)i * RM + k] = (float)m->U[l][(size_t)i * rin + k];
      bl[i] = (float)m->b[l][i];
      for (int k = 0; k < rout; ++k) Vn[(size_t)i * RM + k] = (float)m->V[l + 1][(size_t)i * rout + k];
    }
  }
  float *tail = pk.data() + L * LS;
  for (int k = 0; k < r[0]; ++k) {
    tail[k] = (float)m->V[0][k];
    tail[R1 + k] = (float)m->V[0][r[0] + k];
  }
  tail[2 * R1] = (float)m->U[L][0];
  tail[2 * R1 + 1] = (float)m->b[L][0];
  // FP64 bases for snapshots
  std::vector<double> w64;
  std::vector<int64_t> offs;
  for (int l = 0; l <= L; ++l) {
    offs.push_back((int64_t)w64.size());
    w64.insert(w64.end(), m->U[l].begin(), m->U[l].end());
    offs.push_back((int64_t)w64.size());
    w64.insert(w64.end(), m->V[l].begin(), m->V[l].end());
    offs.push_back((int64_t)w64.size());
    w64.insert(w64.end(), m->b[l].begin(), m->b[l].end());
  }
  cudaError_t e = cudaSuccess;
  auto fail = [&](cudaError_t err) {
    lrnr_destroy(m);
    return cuda_status(err);
  };
  if ((e = cudaMalloc(&m->full_pack, pk.size() * sizeof(float))) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(m->full_pack, pk.data(), pk.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->w64, w64.size() * sizeof(double))) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(m->w64, w64.data(), w64.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->r_dev, sizeof(int) * (L + 1))) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(m->r_dev, m->r, sizeof(int) * (L + 1), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->offs_dev, sizeof(int64_t) * offs.size())) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(m->offs_dev, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->status_dev, sizeof(int))) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(m->status_dev, 0, sizeof(int))) != cudaSuccess) return fail(e);
  if (full_tc_supported(L, M, std::max(16, RM), 32, LRNR_BF16)) {
    std::vector<unsigned char> tp;
    full_tc_pack(L, M, std::max(16, RM), 32, m->U, m->V, m->b, m->r, tp, 0);
    if ((e = cudaMalloc(&m->tc_pack, tp.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(m->tc_pack, tp.data(), tp.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  }
  if (full_tc_supported(L, M, std::max(16, RM), 16, LRNR_BF16X3) &&
      full_tc_nc(std::max(16, RM), LRNR_BF16X3) == 16) {
    std::vector<unsigned char> tp;
    full_tc_pack(L, M, std::max(16, RM), 16, m->U, m->V, m->b, m->r, tp, 0);
    if ((e = cudaMalloc(&m->tc16_pack, tp.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(m->tc16_pack, tp.data(), tp.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  }
  if (full_tc_supported(L, M, std::max(16, RM), 32, LRNR_TF32)) {
    std::vector<unsigned char> tp;
    full_tc_pack(L, M, std::max(16, RM), 32, m->U, m->V, m->b, m->r, tp, 1);
    if ((e = cudaMalloc(&m->tf_pack, tp.size())) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(m->tf_pack, tp.data(), tp.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  }
  *out = m;
  return LRNR_OK;
}

lrnr_status lrnr_snapshots(lrnr_model *m, int layer, int64_t n_pts, const double *x,
                           const double *t, int n_s, const double *s, double *out,
                           void *stream) {
  if (!m || layer < 0 || layer >= m->L || n_pts < 0 || n_s < 0) return LRNR_EINVAL;
  if (n_pts * (int64_t)n_s == 0) return LRNR_OK;
  if (!x || !t || !s || !out) return LRNR_EINVAL;
  if (n_pts * (int64_t)n_s > INT32_MAX) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  CK(launch_snapshots_f64(m->w64, m->L, m->M, m->r_dev, m->offs_dev, layer, n_pts, x, t, n_s, s,
                          m->sum_r, out, static_cast<cudaStream_t>(stream)));
  return LRNR_OK;
}

lrnr_status fastlrnr_select_rows(lrnr_model *m, int layer, const double *snapshots, int64_t K,
                                 int rhat, double tol, const int32_t *rows_in,
                                 const double *Xi_in, int32_t *rows_out, double *Xi_out,
                                 int *rhat_used, void *stream) {
  if (!m || layer < 0 || layer >= m->L || rhat < 1 || rhat > RHMAX || rhat > m->M) return LRNR_EINVAL;
  if (!(tol >= 0.0)) return LRNR_EINVAL;
  if (!rows_in && (!snapshots || K < 1)) return LRNR_EINVAL;
  if (rows_in && !Xi_in) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int M = m->M;
  int32_t *rows_d = nullptr;
  double *Xi_d = nullptr, *R = nullptr, *colmax = nullptr, *outb = nullptr;
  int *est = nullptr;
  lrnr_status rc = LRNR_OK;
  int used = rhat;
  const int rin = m->r[layer], rout = m->r[layer + 1];
  std::vector<double> hb((size_t)rhat * (rin + 1 + rout));
  std::vector<int32_t> hrows(rhat);
  auto cleanup = [&]() {
    if (rows_d) cudaFree(rows_d);
    if (Xi_d) cudaFree(Xi_d);
    if (R) cudaFree(R);
    if (colmax) cudaFree(colmax);
    if (outb) cudaFree(outb);
    if (est) cudaFree(est);
  };
#define CKC(call)                            \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) {                 \
      rc = cuda_status(e_);                  \
      cleanup();                             \
      return rc;                             \
    }                                        \
  } while (0)
  CKC(cudaMalloc(&rows_d, sizeof(int32_t) * rhat));
  CKC(cudaMalloc(&Xi_d, sizeof(double) * (size_t)M * rhat));
  CKC(cudaMalloc(&outb, sizeof(double) * hb.size()));
  CKC(cudaMemsetAsync(m->status_dev, 0, sizeof(int), st));
  if (!rows_in) {
    CKC(cudaMalloc(&R, sizeof(double) * (size_t)M * K));
    CKC(cudaMalloc(&colmax, sizeof(double) * (size_t)K));
    CKC(cudaMalloc(&est, sizeof(int) * 2));
    CKC(cudaMemcpyAsync(R, snapshots, sizeof(double) * (size_t)M * K, cudaMemcpyDeviceToDevice, st));
    CKC(launch_eim_greedy(R, M, K, rhat, tol, rows_d, Xi_d, est, colmax, nullptr, m->status_dev, st));
    int hst[2];
    CKC(cudaMemcpyAsync(hst, est, sizeof(hst), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    used = hst[0] ? hst[1] : rhat;
  } else {
    CKC(cudaMemcpyAsync(rows_d, rows_in, sizeof(int32_t) * rhat, cudaMemcpyDeviceToDevice, st));
    CKC(cudaMemcpyAsync(Xi_d, Xi_in, sizeof(double) * (size_t)M * rhat, cudaMemcpyDeviceToDevice, st));
  }
  int dst = 0;
  CKC(cudaMemcpyAsync(&dst, m->status_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKC(cudaStreamSynchronize(st));
  if (dst == DEV_NONFINITE) { cleanup(); return LRNR_ENONFINITE; }
  if (used < 1) { cleanup(); if (rhat_used) *rhat_used = 0; return LRNR_ESINGULAR; }
  CKC(cudaMemcpy(hrows.data(), rows_d, sizeof(int32_t) * used, cudaMemcpyDeviceToHost));
  {
    std::vector<char> seen(M, 0);
    for (int a = 0; a < used; ++a) {
      if (hrows[a] < 0 || hrows[a] >= M || seen[hrows[a]]) { cleanup(); return LRNR_EINVAL; }
      seen[hrows[a]] = 1;
    }
  }
  const double *Ul = m->w64;  // offsets below
  int64_t offs[3];
  CKC(cudaMemcpy(offs, m->offs_dev + 3 * layer, sizeof(offs), cudaMemcpyDeviceToHost));
  int64_t offn[3];
  CKC(cudaMemcpy(offn, m->offs_dev + 3 * (layer + 1), sizeof(offn), cudaMemcpyDeviceToHost));
  CKC(launch_eim_reduce_f64(Xi_d, rows_d, used, M, Ul + offs[0], Ul + offs[2], Ul + offn[1], rin,
                            rout, outb, m->status_dev, st));
  CKC(cudaMemcpyAsync(&dst, m->status_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKC(cudaStreamSynchronize(st));
  if (dst == DEV_SINGULAR) { cleanup(); return LRNR_ESINGULAR; }
  const size_t nb = (size_t)used * (rin + 1 + rout);
  CKC(cudaMemcpy(hb.data(), outb, sizeof(double) * nb, cudaMemcpyDeviceToHost));
  for (double v : std::vector<double>(hb.begin(), hb.begin() + nb))
    if (!std::isfinite(v)) { cleanup(); return LRNR_ESINGULAR; }
  m->Uh[layer].assign(hb.begin(), hb.begin() + (size_t)used * rin);
  m->bh[layer].assign(hb.begin() + (size_t)used * rin, hb.begin() + (size_t)used * (rin + 1));
  m->Vh[layer].assign(hb.begin() + (size_t)used * (rin + 1), hb.begin() + nb);
  m->rows[layer].assign(hrows.begin(), hrows.begin() + used);
  m->rhat[layer] = used;
  m->fast_dirty = true;
  {
    // once every hidden layer has reduced bases, build the FastLRNR pack here so
    // later calls (and graph captures) allocate nothing for it
    bool all = true;
    for (int l = 0; l < m->L; ++l) all = all && m->rhat[l] > 0;
    if (all) {
      rc = build_fast_pack(m);
      if (rc != LRNR_OK && rc != LRNR_ENOTSUP) { cleanup(); return rc; }
      rc = LRNR_OK;
    }
  }
  if (rows_out) CKC(cudaMemcpyAsync(rows_out, rows_d, sizeof(int32_t) * used, cudaMemcpyDeviceToDevice, st));
  if (Xi_out) CKC(cudaMemcpyAsync(Xi_out, Xi_d, sizeof(double) * (size_t)M * used, cudaMemcpyDeviceToDevice, st));
  CKC(cudaStreamSynchronize(st));
  if (rhat_used) *rhat_used = used;
  cleanup();
#undef CKC
  return LRNR_OK;
}

lrnr_status lrnr_residual(lrnr_model *m, lrnr_form form, lrnr_precision prec, const lrnr_batch *bt,
                          float *u, float *u_t, float *u_x, float *u_xx, float *res, float *res_ic,
                          float *res_bc, void *stream) {
  if (!m) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Pass ps;
  lrnr_status rc = prepare(m, form, prec, bt, false, bt ? bt->s : nullptr, st, ps);
  if (rc != LRNR_OK) return rc;
  ps.p.u = u; ps.p.ut = u_t; ps.p.ux = u_x; ps.p.uxx = u_xx; ps.p.res = res;
  ps.p.res_ic = res_ic; ps.p.res_bc = res_bc;
  return run_main(m, form, prec, ps, st);
}

lrnr_status lrnr_residual_grad(lrnr_model *m, lrnr_form form, lrnr_precision prec,
                               const lrnr_batch *bt, lrnr_loss loss, const float *w,
                               float *loss_out, float *dL_ds, float *dL_db, void *stream) {
  if (!m || !loss_out || !dL_ds) return LRNR_EINVAL;
  if (loss != LRNR_LOSS_MSE && loss != LRNR_LOSS_L1) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Pass ps;
  lrnr_status rc = prepare(m, form, prec, bt, true, bt ? bt->s : nullptr, st, ps);
  if (rc != LRNR_OK) return rc;
  ps.p.loss = loss;
  if (w) { ps.p.w[0] = w[0]; ps.p.w[1] = w[1]; ps.p.w[2] = w[2]; }
  if (dL_db) CK(cudaMemsetAsync(dL_db, 0, sizeof(float) * (size_t)bt->n_inst * m->sum_m, st));
  if (ps.p.fused_red) {
    ps.p.loss_out = loss_out;
    ps.p.dL_ds = dL_ds;
    ps.p.dL_db = dL_db;
    return run_main(m, form, prec, ps, st);
  }
  rc = run_main(m, form, prec, ps, st);
  if (rc != LRNR_OK) return rc;
  const int DB0 = partial_db0(m->L, ps.p.RM);
  const int n_needed = dL_db ? ps.p.P : DB0;
  KParams pr = ps.p;
  pr.M = m->M;   // dL/db is laid out by the full width (the reduced tensor-core pass ran with M = RH)
  CK(launch_reduce(pr, n_needed, form == LRNR_FAST, m->rows_dev, pr.RH, loss_out, dL_ds,
                   dL_db, m->sum_m, m->num_sms, st));
  return LRNR_OK;
}

lrnr_status spinprop_step(lrnr_model *m, lrnr_form form, lrnr_precision prec, const lrnr_batch *bt,
                          lrnr_loss loss, const float *w, float *s_inout, float *adam_m,
                          float *adam_v, int64_t *step, int n_steps, float lr, float beta1,
                          float beta2, float eps, float lambda_loc, const float *s_anchor,
                          float *loss_out, void *stream) {
  if (!m || !s_inout || !adam_m || !adam_v || !step || n_steps < 0) return LRNR_EINVAL;
  if (loss != LRNR_LOSS_MSE && loss != LRNR_LOSS_L1) return LRNR_EINVAL;
  if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f) || !(lambda_loc >= 0.0f))
    return LRNR_EINVAL;
  DeviceGuard g(m->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Pass ps;
  lrnr_status rc = prepare(m, form, prec, bt, true, s_inout, st, ps, true);
  if (rc != LRNR_OK) return rc;
  ps.p.loss = loss;
  if (w) { ps.p.w[0] = w[0]; ps.p.w[1] = w[1]; ps.p.w[2] = w[2]; }
  ps.p.step = step;
  if (ps.p.fused_red) {
    // one kernel per step: residual, adjoint, reduction and Adam
    KParams &p = ps.p;
    p.loss_out = loss_out;
    p.adam_s = s_inout;
    p.adam_m = adam_m;
    p.adam_v = adam_v;
    p.lr = lr;
    p.b1 = beta1;
    p.b2 = beta2;
    p.eps = eps;
    p.lam = s_anchor ? lambda_loc : 0.0f;
    p.anchor = s_anchor;
    for (int k = 0; k < n_steps; ++k) {
      rc = run_main(m, form, prec, ps, st);
      if (rc != LRNR_OK) return rc;
    }
    return LRNR_OK;
  }
  for (int k = 0; k < n_steps; ++k) {
    rc = run_main(m, form, prec, ps, st);
    if (rc != LRNR_OK) return rc;
    CK(launch_reduce_adam(ps.p, s_inout, adam_m, adam_v, step, lr, beta1, beta2, eps, lambda_loc,
                          s_anchor, loss_out, ps.gsum, m->adam_cnt, m->num_sms, st));
  }
  return LRNR_OK;
}

}  // extern "C"

namespace lrnr {
// Parameters of a FastLRNR FP32 gradient pass that uses caller-provided scratch
// instead of the model workspace (for lrnr_residual_grad_noalloc).  Allocates
// nothing: the reduced pack must already exist.
lrnr_status noalloc_fast_params(lrnr_model *m, const lrnr_batch *bt, lrnr_loss loss,
                                const float *w, KParams &p, const int32_t **rows, int *sum_m,
                                int *device) {
  lrnr_status rc = check_batch(m, bt);
  if (rc != LRNR_OK) return rc;
  if (!bt->s) return LRNR_EINVAL;
  if (m->fast_dirty) return LRNR_ENOTREADY;
  if (!m->fast_pack) return LRNR_ENOTSUP;   // ranks above the FP32 instantiations
  std::memset(&p, 0, sizeof(p));
  p.L = m->L;
  p.M = m->M;
  p.n_inst = bt->n_inst;
  for (int l = 0; l <= m->L; ++l) p.r[l] = m->r[l];
  for (int l = 0; l <= m->L + 1; ++l) p.roff[l] = m->roff[l];
  p.sum_r = m->sum_r;
  p.beta = bt->beta; p.nu = bt->nu; p.rho = bt->rho; p.s = bt->s;
  p.int_off = bt->int_off; p.ic_off = bt->ic_off; p.bc_off = bt->bc_off;
  p.x_int = bt->x_int; p.t_int = bt->t_int; p.x_ic = bt->x_ic; p.t_bc = bt->t_bc;
  p.tot[0] = bt->n_int; p.tot[1] = bt->n_ic; p.tot[2] = bt->n_bc;
  p.norm = bt->norm;
  p.grad = 1;
  p.status = m->status_dev;
  p.RM = m->fRM;
  p.RH = m->fRH;
  p.pack = m->fast_pack;
  for (int l = 0; l < m->L; ++l) p.rh[l] = m->rhat[l];
  p.P = partial_len(m->L, p.RM, m->L * p.RH);
  // the tile size and wait cap lrnr_residual_grad uses (including an lrnr_set_tuning
  // override that fits the kernel's shared memory), so both give identical results
  const int Pfit = partial_len(m->L, p.RM, m->L * p.RH + 1);
  p.nt = fast_choose_nt(m->L, p.RM, p.RH, Pfit);
  if (!p.nt) return LRNR_ENOTSUP;
  const int tn = m->tune_nt[LRNR_FAST][LRNR_FP32];
  if (tn && fast_smem_bytes(m->L, p.RM, p.RH, tn, Pfit) <= (size_t)kSmemBudget) p.nt = tn;
  p.fast_regs = m->tune_cta[LRNR_FAST][LRNR_FP32] >= 3 ? 3 : 2;
  p.loss = loss;
  p.w[0] = p.w[1] = p.w[2] = 1.0f;
  if (w) { p.w[0] = w[0]; p.w[1] = w[1]; p.w[2] = w[2]; }
  p.max_wait = m->wait_limit;
  *rows = m->rows_dev;
  *sum_m = m->sum_m;
  *device = m->device;
  return LRNR_OK;
}

// Cap on resident FastLRNR FP32 CTAs per SM set by lrnr_set_tuning (0 = none).
int noalloc_cta_cap(const lrnr_model *m) { return m->tune_cta[LRNR_FAST][LRNR_FP32]; }

int64_t noalloc_max_tiles(const lrnr_batch *bt, int nt) {
  return max_tiles(bt->n_int, bt->n_ic, bt->n_bc, bt->n_inst, nt);
}
}  // namespace lrnr

extern "C" {

lrnr_status lrnr_reserve(lrnr_model *m, int64_t max_points, int32_t max_inst) {
  if (!m || max_points < 0 || max_inst < 1) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  const int nt_min = 32;
  const int64_t tiles = max_points / nt_min + 3 * (int64_t)max_inst + 3;
  int Pmax = partial_len(m->L, m->RM, m->L * m->M + 1);
  const int RMm = std::max(16, m->RM);   // largest padded rank any path uses for this model
  Pmax = std::max(Pmax, partial_len(m->L, RMm, m->L * RHMAX + 1));
  // per-CTA layer-input stores (tensor-core and FastLRNR kernels): at most 4 CTAs per SM
  const size_t store = std::max(std::max(full_tc_scratch_floats(m->L, RMm, 2 * m->num_sms),
                                         fast_scratch_floats(m->L, RMm, RHMAX, 128, 4 * m->num_sms)),
                                full_fp32_scratch_floats(m->L, RMm, 64, 8 * m->num_sms));
  const size_t need = align256(sizeof(int32_t) * (size_t)(max_inst + 1)) +
                      align256((size_t)tiles * Pmax * sizeof(float)) +
                      align256(store * sizeof(float)) +
                      align256(adam_group_floats(max_inst, m->L, RMm) * sizeof(float)) +
                      align256((size_t)(tiles / kRedGroup + 1 + max_inst) * Pmax * sizeof(float));
  lrnr_status rc = ensure_tickets(m, tiles / kRedGroup + 2 + 2 * (int64_t)max_inst, nullptr);
  if (rc != LRNR_OK) return rc;
  return ensure_ws(m, need, nullptr);
}

lrnr_status lrnr_adam_update(int32_t n_inst, int32_t sum_r, const float *grad, float *s_inout,
                             float *adam_m, float *adam_v, int64_t *step, float lr, float beta1,
                             float beta2, float eps, float lambda_loc, const float *s_anchor,
                             const float *loss_in, float *loss_out, void *stream) {
  if (n_inst < 1 || sum_r < 1 || !grad || !s_inout || !adam_m || !adam_v || !step) return LRNR_EINVAL;
  if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f) || !(lambda_loc >= 0.0f))
    return LRNR_EINVAL;
  CK(launch_adam_update(n_inst, sum_r, grad, s_inout, adam_m, adam_v, step, lr, beta1, beta2, eps,
                        s_anchor ? lambda_loc : 0.0f, s_anchor, loss_in, loss_out,
                        static_cast<cudaStream_t>(stream)));
  return LRNR_OK;
}

lrnr_status lrnr_set_wait_limit(lrnr_model *m, int64_t polls) {
  if (!m) return LRNR_EINVAL;
  m->wait_limit = polls < 0 ? (1u << 20) : (uint32_t)std::min<int64_t>(polls, UINT32_MAX);
  return LRNR_OK;
}

lrnr_status lrnr_set_tuning(lrnr_model *m, lrnr_form form, lrnr_precision prec, int nt,
                            int ctas_per_sm) {
  if (!m || (form != LRNR_FULL && form != LRNR_FAST) || prec < LRNR_FP32 || prec > LRNR_BF16X3)
    return LRNR_EINVAL;
  if (nt != 0 && nt != 32 && nt != 64 && nt != 128) return LRNR_EINVAL;
  if (ctas_per_sm < 0 || ctas_per_sm > 8) return LRNR_EINVAL;
  m->tune_nt[form][prec] = nt;
  m->tune_cta[form][prec] = ctas_per_sm;
  return LRNR_OK;
}

lrnr_status lrnr_model_info(const lrnr_model *m, int *L, int *M, int *sum_r, int *sum_m,
                            int *fast_ready) {
  if (!m) return LRNR_EINVAL;
  if (L) *L = m->L;
  if (M) *M = m->M;
  if (sum_r) *sum_r = m->sum_r;
  if (sum_m) *sum_m = m->sum_m;
  if (fast_ready) {
    int ok = 1;
    for (int l = 0; l < m->L; ++l) ok &= m->rhat[l] > 0;
    *fast_ready = ok;
  }
  return LRNR_OK;
}

lrnr_status lrnr_timing(lrnr_model *m, int enable) {
  if (!m) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  m->timing = enable != 0;
  m->ev_used = 0;
  for (auto e : m->cap_start) cudaEventDestroy(e);
  for (auto e : m->cap_stop) cudaEventDestroy(e);
  m->cap_start.clear();
  m->cap_stop.clear();
  return LRNR_OK;
}

lrnr_status lrnr_timing_read(lrnr_model *m, double *ms_total, int64_t *launches) {
  if (!m) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  double tot = 0.0;
  for (size_t i = 0; i < m->ev_used; ++i) {
    CK(cudaEventSynchronize(m->ev_stop[i]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, m->ev_start[i], m->ev_stop[i]));
    tot += ms;
  }
  for (size_t i = 0; i < m->cap_start.size(); ++i) {
    CK(cudaEventSynchronize(m->cap_stop[i]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, m->cap_start[i], m->cap_stop[i]));
    tot += ms;
  }
  if (ms_total) *ms_total = tot;
  if (launches) *launches = (int64_t)(m->ev_used + m->cap_start.size());
  m->ev_used = 0;
  return LRNR_OK;
}

lrnr_status lrnr_last_device_status(lrnr_model *m) {
  if (!m) return LRNR_EINVAL;
  DeviceGuard g(m->device);
  CK(cudaDeviceSynchronize());
  int v = 0;
  CK(cudaMemcpy(&v, m->status_dev, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(m->status_dev, 0, sizeof(int)));
  switch (v) {
    case DEV_OK: return LRNR_OK;
    case DEV_NONFINITE: return LRNR_ENONFINITE;
    case DEV_TIMEOUT: return LRNR_ETIMEOUT;
    case DEV_SINGULAR: return LRNR_ESINGULAR;
    case DEV_BADBATCH: return LRNR_EINVAL;
  }
  return LRNR_ECUDA;
}

void lrnr_destroy(lrnr_model *m) {
  if (!m) return;
  DeviceGuard g(m->device);
  cudaFree(m->full_pack);
  cudaFree(m->w64);
  cudaFree(m->r_dev);
  cudaFree(m->offs_dev);
  cudaFree(m->tc_pack);
  cudaFree(m->tc16_pack);
  cudaFree(m->ftc_pack);
  cudaFree(m->tf_pack);
  cudaFree(m->ftf_pack);
  cudaFree(m->fast_pack);
  cudaFree(m->fastk_pack);
  cudaFree(m->rows_dev);
  cudaFree(m->status_dev);
  cudaFree(m->ws);
  cudaFree(m->adam_cnt);
  for (auto e : m->ev_start) cudaEventDestroy(e);
  for (auto e : m->ev_stop) cudaEventDestroy(e);
  for (auto e : m->cap_start) cudaEventDestroy(e);
  for (auto e : m->cap_stop) cudaEventDestroy(e);
  delete m;
}

}  // extern "C"
