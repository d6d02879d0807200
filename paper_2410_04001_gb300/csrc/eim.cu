// EIM row selection and FastLRNR layer reduction in FP64 (Sec. 2.2 Eq. 2.7), and
// the exact-LRNR hidden-state snapshots it is built from (Sec. 4).
//
// Greedy step j (classic EIM, incremental form) on the residual R (M x K, column-
// major, a private copy of the snapshots):
//   colmax kernel: apply step j-1's rank-one update to every column,
//       R[:,k] <- R[:,k] - xi_{j-1} * R[p_{j-1}, k]   (product, then difference:
//       __dmul_rn / __dsub_rn, never a fused multiply-add),
//     then e_k = max_i |R_ik|.
//   pivot kernel: k* = argmax_k e_k (lowest k on ties); stop when e_k* <= tol;
//     p_j = argmax_i |R_i,k*| (lowest i on ties); xi_j = R[:,k*] / R[p_j,k*].
// Every comparison is exact and every arithmetic step is one correctly rounded
// IEEE operation, so rows and Xi are bit-identical to an FP64 reference that
// performs the same operations.
#include "lrnr_internal.cuh"

namespace lrnr {
namespace {

constexpr int COLS_PER_BLOCK = 8;

struct EimState {
  int stopped;
  int used;
};

__global__ void __launch_bounds__(256) k_eim_colmax(double *R, int M, int64_t K, int j,
                                                    const int32_t *rows, const double *Xi,
                                                    const EimState *st, double *colmax,
                                                    int *status) {
  if (st->stopped) return;
  __shared__ double red[8];
  __shared__ double piv;
  const int tid = threadIdx.x;
  const int prow = j > 0 ? rows[j - 1] : 0;
  const double *xi = j > 0 ? Xi + (int64_t)(j - 1) * M : nullptr;
  for (int cc = 0; cc < COLS_PER_BLOCK; ++cc) {
    const int64_t k = (int64_t)blockIdx.x * COLS_PER_BLOCK + cc;
    if (k >= K) break;
    double *col = R + k * M;
    if (j > 0) {
      if (tid == 0) piv = col[prow];
      __syncthreads();
      const double pv = piv;
      for (int i = tid; i < M; i += 256) col[i] = __dsub_rn(col[i], __dmul_rn(xi[i], pv));
    }
    double mx = 0.0;
    bool bad = false;
    for (int i = tid; i < M; i += 256) {
      const double a = fabs(col[i]);
      if (a != a) bad = true;
      mx = a > mx ? a : mx;
    }
    if (bad) set_status(status, DEV_NONFINITE);
#pragma unroll
    for (int off = 16; off >= 1; off /= 2) {
      const double o = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = o > mx ? o : mx;
    }
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = red[0];
      for (int w = 1; w < 8; ++w) m2 = red[w] > m2 ? red[w] : m2;
      colmax[k] = m2;
    }
    __syncthreads();
  }
}

// (value, index) with "larger value, then smaller index" ordering.
__device__ __forceinline__ void better(double &v, int64_t &ix, double v2, int64_t ix2) {
  if (v2 > v || (v2 == v && ix2 < ix)) { v = v2; ix = ix2; }
}

__global__ void __launch_bounds__(1024) k_eim_pivot(double *R, int M, int64_t K, int j, double tol,
                                                    int32_t *rows, double *Xi, EimState *st,
                                                    const double *colmax) {
  if (st->stopped) return;
  __shared__ double rv[32];
  __shared__ int64_t ri[32];
  __shared__ int64_t kstar_s;
  __shared__ int prow_s;
  const int tid = threadIdx.x;
  double v = -1.0;
  int64_t ix = INT64_MAX;
  for (int64_t k = tid; k < K; k += 1024) better(v, ix, colmax[k], k);
#pragma unroll
  for (int off = 16; off >= 1; off /= 2) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
    const int64_t i2 = __shfl_xor_sync(0xffffffffu, ix, off);
    better(v, ix, v2, i2);
  }
  if ((tid & 31) == 0) { rv[tid >> 5] = v; ri[tid >> 5] = ix; }
  __syncthreads();
  if (tid == 0) {
    double bv = rv[0];
    int64_t bi = ri[0];
    for (int w = 1; w < 32; ++w) better(bv, bi, rv[w], ri[w]);
    kstar_s = bi;
    if (!(bv > tol)) {
      st->stopped = 1;
      st->used = j;
    }
  }
  __syncthreads();
  if (st->stopped) return;
  const double *col = R + kstar_s * M;
  // pivot row: argmax_i |R_i,k*|, lowest index on ties
  v = -1.0;
  ix = INT64_MAX;
  for (int i = tid; i < M; i += 1024) better(v, ix, fabs(col[i]), i);
#pragma unroll
  for (int off = 16; off >= 1; off /= 2) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
    const int64_t i2 = __shfl_xor_sync(0xffffffffu, ix, off);
    better(v, ix, v2, i2);
  }
  __syncthreads();
  if ((tid & 31) == 0) { rv[tid >> 5] = v; ri[tid >> 5] = ix; }
  __syncthreads();
  if (tid == 0) {
    double bv = rv[0];
    int64_t bi = ri[0];
    for (int w = 1; w < 32; ++w) better(bv, bi, rv[w], ri[w]);
    prow_s = (int)bi;
    rows[j] = (int)bi;
    st->used = j + 1;
  }
  __syncthreads();
  const double pv = col[prow_s];
  double *xo = Xi + (int64_t)j * M;
  for (int i = tid; i < M; i += 1024) xo[i] = __ddiv_rn(col[i], pv);
}

__global__ void k_eim_init(EimState *st) {
  st->stopped = 0;
  st->used = 0;
}

// Reduced bases of one hidden layer (Eq. 2.7): Uhat = U[P,:], bhat = b[P],
// Vhat = (P^T Xi)^{-T} Xi^T V^{l+1}.  Output (FP64, compact):
//   Uh [rh][rin], bh [rh], Vh [rh][rout].
// One block; the rh x rh solve (rh <= 32) runs on one thread by Gaussian
// elimination with partial pivoting.
__global__ void __launch_bounds__(1024) k_eim_reduce(const double *Xi, const int32_t *rows, int rh,
                                                     int M, const double *U, const double *b,
                                                     const double *Vn, int rin, int rout,
                                                     double *out, int *status) {
  __shared__ double G[RHMAX][RMAX];
  __shared__ double T[RHMAX][RHMAX];
  const int tid = threadIdx.x;
  for (int e = tid; e < rh * rout; e += blockDim.x) {
    const int a = e / rout, jj = e % rout;
    double acc = 0.0;
    const double *xc = Xi + (int64_t)a * M;
    for (int i = 0; i < M; ++i) acc += xc[i] * Vn[(int64_t)i * rout + jj];
    G[a][jj] = acc;
  }
  // T = (P^T Xi)^T:  T[a][b] = Xi[rows[b], a]
  for (int e = tid; e < rh * rh; e += blockDim.x) {
    const int a = e / rh, bb = e % rh;
    T[a][bb] = Xi[(int64_t)a * M + rows[bb]];
  }
  double *Uh = out, *bh = out + rh * rin, *Vh = bh + rh;
  for (int e = tid; e < rh * rin; e += blockDim.x) {
    const int a = e / rin, k = e % rin;
    Uh[e] = U[(int64_t)rows[a] * rin + k];
  }
  for (int a = tid; a < rh; a += blockDim.x) bh[a] = b[rows[a]];
  __syncthreads();
  if (tid == 0) {
    // solve T X = G (T = (P^T Xi)^T), X is rh x rout
    for (int c = 0; c < rh; ++c) {
      int piv = c;
      for (int rr = c + 1; rr < rh; ++rr)
        if (fabs(T[rr][c]) > fabs(T[piv][c])) piv = rr;
      if (T[piv][c] == 0.0) { set_status(status, DEV_SINGULAR); return; }
      if (piv != c) {
        for (int q = 0; q < rh; ++q) { double t = T[c][q]; T[c][q] = T[piv][q]; T[piv][q] = t; }
        for (int q = 0; q < rout; ++q) { double t = G[c][q]; G[c][q] = G[piv][q]; G[piv][q] = t; }
      }
      for (int rr = c + 1; rr < rh; ++rr) {
        const double f = T[rr][c] / T[c][c];
        if (f == 0.0) continue;
        for (int q = c; q < rh; ++q) T[rr][q] -= f * T[c][q];
        for (int q = 0; q < rout; ++q) G[rr][q] -= f * G[c][q];
      }
    }
    for (int c = rh - 1; c >= 0; --c) {
      for (int q = 0; q < rout; ++q) {
        double acc = G[c][q];
        for (int k = c + 1; k < rh; ++k) acc -= T[c][k] * G[k][q];
        G[c][q] = acc / T[c][c];
      }
    }
    for (int a = 0; a < rh; ++a)
      for (int q = 0; q < rout; ++q) Vh[a * rout + q] = G[a][q];
  }
}

// Exact LRNR hidden state of layer `layer` (value channel, FP64), one block per
// (draw, point) column; the M-wide state lives in shared memory.
__global__ void __launch_bounds__(256) k_snapshots(const double *w64, int L, int M, int4 meta,
                                                   const int *rr, const int64_t *offs,
                                                   int layer, int64_t n_pts, const double *x,
                                                   const double *t, const double *s, int sum_r,
                                                   double *out) {
  extern __shared__ double zs[];          // [M] state + [RMAX] projection
  double *pj = zs + M;
  const int64_t col = blockIdx.x;
  const int64_t draw = col / n_pts, pt = col % n_pts;
  const double *sv = s + draw * sum_r;
  const int tid = threadIdx.x;
  double z0 = x[pt], z1 = t[pt];
  int width = 2;
  if (tid == 0) { zs[0] = z0; zs[1] = z1; }
  __syncthreads();
  int soff = 0;
  for (int l = 0; l <= layer; ++l) {
    const int r = rr[l];
    const double *U = w64 + offs[3 * l + 0];
    const double *V = w64 + offs[3 * l + 1];
    const double *b = w64 + offs[3 * l + 2];
    // projection q_k = sum_i V[i][k] z_i, scaled by s
    for (int k = tid; k < r; k += blockDim.x) {
      double acc = 0.0;
      for (int i = 0; i < width; ++i) acc += V[(int64_t)i * r + k] * zs[i];
      pj[k] = acc * sv[soff + k];
    }
    __syncthreads();
    for (int i = tid; i < M; i += blockDim.x) {
      double a = b[i];
      for (int k = 0; k < r; ++k) a += U[(int64_t)i * r + k] * pj[k];
      zs[i] = tanh(a);
    }
    __syncthreads();
    width = M;
    soff += r;
  }
  for (int i = tid; i < M; i += blockDim.x) out[col * M + i] = zs[i];
  (void)meta;
  (void)L;
}

}  // namespace

cudaError_t launch_eim_greedy(double *R, int M, int64_t K, int rhat, double tol, int32_t *rows,
                              double *Xi, int *used_dev, double *colmax, int64_t * /*colarg*/,
                              int *status, cudaStream_t st) {
  EimState *est = reinterpret_cast<EimState *>(used_dev);
  k_eim_init<<<1, 1, 0, st>>>(est);
  const int nb = (int)((K + COLS_PER_BLOCK - 1) / COLS_PER_BLOCK);
  for (int j = 0; j < rhat; ++j) {
    k_eim_colmax<<<nb, 256, 0, st>>>(R, M, K, j, rows, Xi, est, colmax, status);
    k_eim_pivot<<<1, 1024, 0, st>>>(R, M, K, j, tol, rows, Xi, est, colmax);
  }
  return cudaGetLastError();
}

cudaError_t launch_eim_reduce_f64(const double *Xi, const int32_t *rows, int rh, int M,
                                  const double *U, const double *b, const double *Vn, int rin,
                                  int rout, double *out, int *status, cudaStream_t st) {
  k_eim_reduce<<<1, 1024, 0, st>>>(Xi, rows, rh, M, U, b, Vn, rin, rout, out, status);
  return cudaGetLastError();
}

cudaError_t launch_snapshots_f64(const double *w64, int L, int M, const int *r_dev,
                                 const int64_t *offs_dev, int layer, int64_t n_pts,
                                 const double *x, const double *t, int n_s, const double *s,
                                 int sum_r, double *out, cudaStream_t st) {
  const int64_t cols = n_pts * (int64_t)n_s;
  if (cols == 0) return cudaSuccess;
  const size_t smem = (size_t)(M + RMAX) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_snapshots, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_snapshots<<<(unsigned)cols, 256, smem, st>>>(w64, L, M, make_int4(0, 0, 0, 0), r_dev, offs_dev,
                                                 layer, n_pts, x, t, s, sum_r, out);
  return cudaGetLastError();
}

}  // namespace lrnr
