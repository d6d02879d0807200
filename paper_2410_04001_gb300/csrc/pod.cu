// The DEIM reading of the layer reduction (Sec. 2.2, Eq. 2.7 with Xi the leading
// left singular vectors of the snapshots and P chosen by the discrete empirical
// interpolation method), in FP64:
//
//   lrnr_pod: POD basis of a snapshot matrix S (M x K, column-major) by block
//     subspace iteration on S S^T with nb columns:
//       Q_0 = orth(S Omega)            Omega: K x nb signs from a counter hash
//       Q_t = orth(S (S^T Q_{t-1}))    t = 1..n_iter
//       Rayleigh-Ritz: Z = S^T Q, H = Z^T Z = W diag(lambda) W^T (cyclic Jacobi),
//       Xi = Q W (lambda descending), sigma = sqrt(lambda).
//     Each column of Xi is then scaled by +-1 so that its entry of largest magnitude
//     (lowest index among exact ties) is positive.
//   lrnr_deim_rows: DEIM indices of a basis.  Step j solves the j x j interpolation
//     system (P^T Xi_j) c = P^T xi_j by Gaussian elimination with partial pivoting and
//     takes the row of largest |xi_j - Xi_j c| (lowest index among exact ties).
//
// The dense products run in one tiled FP64 kernel; a long reduction dimension is
// split into partial tiles that a second kernel adds in a fixed order, so every
// result is reproducible run to run.  Orthonormalisation (classical Gram-Schmidt,
// applied twice) and the Jacobi sweeps run in one CTA each: nb <= 64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lrnr_internal.cuh"

namespace lrnr {
namespace {

constexpr int NBMAX = 64;   // subspace block columns
constexpr int GBM = 64, GBN = 64, GBK = 16;

// C(i, j) = sum_k A(i, k) B(k, j), A(i, k) = A[i sa_i + k sa_k], B(k, j) = B[k sb_k + j sb_j].
// Without a partial buffer the tile goes to C[i + j ldc]; with one, split z writes its
// sum over [z kchunk, (z + 1) kchunk) to part[(z n + j) m + i].
struct Gemm {
  const double *A;
  int64_t sa_i, sa_k;
  const double *B;
  int64_t sb_k, sb_j;
  double *C;
  int64_t ldc;
  int m, n;
  int64_t k, kchunk;
  double *part;
};

__global__ void __launch_bounds__(256) k_dgemm(Gemm g) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * GBM, j0 = blockIdx.y * GBN;
  const int64_t k0 = (int64_t)blockIdx.z * g.kchunk;
  const int64_t k1 = k0 + g.kchunk < g.k ? k0 + g.kchunk : g.k;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t kb = k0; kb < k1; kb += GBK) {
    for (int e = tid; e < GBM * GBK; e += 256) {
      // walk the unit-stride index fastest
      const int ii = g.sa_i == 1 ? e % GBM : e / GBK;
      const int kk = g.sa_i == 1 ? e / GBM : e % GBK;
      const int i = i0 + ii;
      const int64_t k = kb + kk;
      As[kk][ii] = (i < g.m && k < k1) ? g.A[(int64_t)i * g.sa_i + k * g.sa_k] : 0.0;
    }
    for (int e = tid; e < GBN * GBK; e += 256) {
      const int jj = g.sb_k == 1 ? e / GBK : e % GBN;
      const int kk = g.sb_k == 1 ? e % GBK : e / GBN;
      const int j = j0 + jj;
      const int64_t k = kb + kk;
      Bs[kk][jj] = (j < g.n && k < k1) ? g.B[k * g.sb_k + (int64_t)j * g.sb_j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty + 16 * p, j = j0 + tx + 16 * q;
      if (i >= g.m || j >= g.n) continue;
      if (g.part)
        g.part[((int64_t)blockIdx.z * g.n + j) * g.m + i] = acc[p][q];
      else
        g.C[i + (int64_t)j * g.ldc] = acc[p][q];
    }
}

// C[i + j ldc] = sum over splits z = 0, 1, ... of part[(z n + j) m + i].
__global__ void k_dgemm_sum(const double *part, int splits, int m, int n, double *C, int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * n) return;
  const int i = (int)(e % m), j = (int)(e / m);
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[((int64_t)z * n + j) * m + i];
  C[i + (int64_t)j * ldc] = s;
}

struct GemmPlan {
  int tiles_m, tiles_n, splits;
  int64_t kchunk;
};

GemmPlan plan_gemm(int m, int n, int64_t k, int sms) {
  GemmPlan p;
  p.tiles_m = (m + GBM - 1) / GBM;
  p.tiles_n = (n + GBN - 1) / GBN;
  const int64_t tiles = (int64_t)p.tiles_m * p.tiles_n;
  int64_t splits = (2 * (int64_t)sms + tiles - 1) / tiles;
  const int64_t max_splits = std::max<int64_t>(1, k / (4 * GBK));
  splits = std::max<int64_t>(1, std::min(splits, max_splits));
  int64_t chunk = (k + splits - 1) / splits;
  chunk = (chunk + GBK - 1) / GBK * GBK;
  p.kchunk = chunk;
  p.splits = (int)((k + chunk - 1) / chunk);
  return p;
}

size_t gemm_part_doubles(int m, int n, int64_t k, int sms) {
  const GemmPlan p = plan_gemm(m, n, k, sms);
  return p.splits > 1 ? (size_t)p.splits * m * n : 0;
}

cudaError_t dgemm(Gemm g, double *part, int sms, cudaStream_t st) {
  const GemmPlan p = plan_gemm(g.m, g.n, g.k, sms);
  g.kchunk = p.kchunk;
  g.part = p.splits > 1 ? part : nullptr;
  k_dgemm<<<dim3(p.tiles_m, p.tiles_n, p.splits), 256, 0, st>>>(g);
  if (p.splits > 1) {
    const int64_t tot = (int64_t)g.m * g.n;
    k_dgemm_sum<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, p.splits, g.m, g.n, g.C,
                                                                g.ldc);
  }
  return cudaGetLastError();
}

// A (r x c, column-major, leading dimension ld).
Gemm mat(const double *A, int64_t ld, bool trans) {
  Gemm g{};
  g.A = A;
  g.sa_i = trans ? ld : 1;
  g.sa_k = trans ? 1 : ld;
  return g;
}
void with_b(Gemm &g, const double *B, int64_t ld, bool trans) {
  g.B = B;
  g.sb_k = trans ? ld : 1;
  g.sb_j = trans ? 1 : ld;
}

// splitmix64 finaliser: the counter hash behind the start block and restarts.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double hash_sign(uint64_t a, uint64_t b) {
  return (mix64(a * 0x100000001B3ull + b) >> 63) ? -1.0 : 1.0;
}

__global__ void k_signs(double *Om, int64_t K, int nb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < K * nb) Om[e] = hash_sign((uint64_t)(e / K), (uint64_t)(e % K));
}

// Sum of v over the block (every thread gets the total); red holds 32 doubles.
__device__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o >= 1; o /= 2) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// Orthonormalise the nb columns of Y (M x nb, column-major) in place: classical
// Gram-Schmidt applied twice per column.  A column whose norm falls to zero (or
// below 1e-13 of its norm before the projections) is replaced by a hash sign
// vector and projected again (at most twice).
__global__ void __launch_bounds__(1024) k_orth(double *Y, int M, int nb, int *status) {
  __shared__ double d[NBMAX];
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < nb; ++j) {
    double *y = Y + (int64_t)j * M;
    double s0 = 0.0;
    for (int i = tid; i < M; i += blockDim.x) s0 += y[i] * y[i];
    double n0 = sqrt(block_sum(s0, red));
    bool done = false;
    for (int attempt = 0; attempt < 3 && !done; ++attempt) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int a = warp; a < j; a += 32) {
          const double *qa = Y + (int64_t)a * M;
          double s = 0.0;
          for (int i = lane; i < M; i += 32) s += qa[i] * y[i];
#pragma unroll
          for (int o = 16; o >= 1; o /= 2) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) d[a] = s;
        }
        __syncthreads();
        for (int i = tid; i < M; i += blockDim.x) {
          double v = y[i];
          for (int a = 0; a < j; ++a) v -= d[a] * Y[(int64_t)a * M + i];
          y[i] = v;
        }
        __syncthreads();
      }
      double s1 = 0.0;
      for (int i = tid; i < M; i += blockDim.x) s1 += y[i] * y[i];
      const double n1 = sqrt(block_sum(s1, red));
      if (n1 > 0.0 && n1 > 1e-13 * n0) {
        const double inv = 1.0 / n1;
        for (int i = tid; i < M; i += blockDim.x) y[i] *= inv;
        done = true;
      } else {
        for (int i = tid; i < M; i += blockDim.x)
          y[i] = hash_sign(0x5EED0000ull + 64 * (uint64_t)j + attempt, (uint64_t)i);
        n0 = sqrt((double)M);
      }
      __syncthreads();
    }
    if (!done) {
      if (tid == 0) set_status(status, DEV_SINGULAR);
      return;
    }
  }
}

// Symmetric eigen-decomposition of H (nb x nb, column-major) by cyclic Jacobi with a
// round-robin ordering: every step rotates nbe/2 disjoint pairs at once.  Writes the
// eigenvalues in descending order (lowest index first among ties) to lam and the
// matching eigenvectors as the columns of W (nb x nb, column-major).
constexpr int JLD = NBMAX + 1;   // leading dimension of the Jacobi tiles in shared memory
constexpr size_t kJacobiSmem = 2 * sizeof(double) * NBMAX * JLD;

__global__ void __launch_bounds__(1024) k_jacobi(const double *H, int nb, double *lam, double *W,
                                                 int *status) {
  extern __shared__ double jsm[];
  double(*A)[JLD] = reinterpret_cast<double(*)[JLD]>(jsm);
  double(*V)[JLD] = reinterpret_cast<double(*)[JLD]>(jsm + NBMAX * JLD);
  __shared__ double cs[NBMAX / 2][2];
  __shared__ int pq[NBMAX / 2][2];
  __shared__ double red[32];
  __shared__ int rot;
  const int tid = threadIdx.x;
  const int nbe = nb + (nb & 1), half = nbe / 2, m = nbe - 1;
  for (int e = tid; e < nbe * nbe; e += blockDim.x) {
    const int r = e % nbe, c = e / nbe;
    A[r][c] = (r < nb && c < nb) ? H[r + (int64_t)c * nb] : 0.0;
    V[r][c] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  double fro = 0.0;
  for (int e = tid; e < nbe * nbe; e += blockDim.x) fro += A[e % nbe][e / nbe] * A[e % nbe][e / nbe];
  // a pair is rotated while |a_pq| > 1e-16 sqrt(|a_pp a_qq|) (relative to its
  // diagonal, which keeps small eigenvalues accurate) and above 1e-30 ||H||_F
  const double floor_abs = 1e-30 * sqrt(block_sum(fro, red));
  bool conv = nbe < 2;
  for (int sweep = 0; sweep < 64 && !conv; ++sweep) {
    if (tid == 0) rot = 0;
    __syncthreads();
    for (int s = 0; s < m; ++s) {
      if (tid < half) {
        const int k = tid;
        const int p = k == 0 ? 0 : ((s + k) % m) + 1;
        const int q = ((s + m - k) % m) + 1;
        const double app = A[p][p], aqq = A[q][q], apq = A[p][q];
        double c = 1.0, sn = 0.0;
        if (fabs(apq) > floor_abs && fabs(apq) > 1e-16 * sqrt(fabs(app) * fabs(aqq))) {
          const double tau = (aqq - app) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          sn = t * c;
          rot = 1;
        }
        pq[k][0] = p;
        pq[k][1] = q;
        cs[k][0] = c;
        cs[k][1] = sn;
      }
      __syncthreads();
      // rows p, q of J^T A
      for (int e = tid; e < half * nbe; e += blockDim.x) {
        const int k = e / nbe, col = e % nbe;
        const int p = pq[k][0], q = pq[k][1];
        const double c = cs[k][0], sn = cs[k][1];
        const double hp = A[p][col], hq = A[q][col];
        A[p][col] = c * hp - sn * hq;
        A[q][col] = sn * hp + c * hq;
      }
      __syncthreads();
      // columns p, q of (J^T A) J and of V J
      for (int e = tid; e < half * nbe; e += blockDim.x) {
        const int k = e / nbe, row = e % nbe;
        const int p = pq[k][0], q = pq[k][1];
        const double c = cs[k][0], sn = cs[k][1];
        const double hp = A[row][p], hq = A[row][q];
        A[row][p] = c * hp - sn * hq;
        A[row][q] = sn * hp + c * hq;
        // the rotated pair's off-diagonal entries are zero by construction
        if (sn != 0.0 && row == p) A[p][q] = 0.0;
        if (sn != 0.0 && row == q) A[q][p] = 0.0;
        const double vp = V[row][p], vq = V[row][q];
        V[row][p] = c * vp - sn * vq;
        V[row][q] = sn * vp + c * vq;
      }
      __syncthreads();
    }
    conv = rot == 0;
    __syncthreads();
  }
  if (!conv) {
    if (tid == 0) set_status(status, DEV_TIMEOUT);
    return;
  }
  __shared__ int order[NBMAX];
  if (tid == 0) {
    // selection of the largest remaining eigenvalue, lowest index on ties; the
    // padding index (odd nb) is left out
    bool taken[NBMAX];
    for (int i = 0; i < nb; ++i) taken[i] = false;
    for (int c = 0; c < nb; ++c) {
      int best = -1;
      for (int i = 0; i < nb; ++i)
        if (!taken[i] && (best < 0 || A[i][i] > A[best][best])) best = i;
      taken[best] = true;
      order[c] = best;
    }
  }
  __syncthreads();
  for (int c = tid; c < nb; c += blockDim.x) lam[c] = A[order[c]][order[c]];
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e % nb, c = e / nb;
    W[e] = V[r][order[c]];
  }
}

// Column c of X (M x n): flip its sign unless its largest-magnitude entry (lowest
// index among ties) is positive.  One block per column.
__global__ void __launch_bounds__(256) k_canon_sign(double *X, int M) {
  __shared__ double rv[8];
  __shared__ int ri[8];
  double *x = X + (int64_t)blockIdx.x * M;
  double v = -1.0;
  int ix = INT32_MAX;
  for (int i = threadIdx.x; i < M; i += 256) {
    const double a = fabs(x[i]);
    if (a > v) { v = a; ix = i; }
  }
#pragma unroll
  for (int o = 16; o >= 1; o /= 2) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, ix, o);
    if (v2 > v || (v2 == v && i2 < ix)) { v = v2; ix = i2; }
  }
  if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = v; ri[threadIdx.x >> 5] = ix; }
  __syncthreads();
  __shared__ int flip;
  if (threadIdx.x == 0) {
    double bv = rv[0];
    int bi = ri[0];
    for (int w = 1; w < 8; ++w)
      if (rv[w] > bv || (rv[w] == bv && ri[w] < bi)) { bv = rv[w]; bi = ri[w]; }
    flip = x[bi] < 0.0;
  }
  __syncthreads();
  if (flip)
    for (int i = threadIdx.x; i < M; i += 256) x[i] = -x[i];
}

// res[c] = || R[:, c] - lam[c] X[:, c] ||_2 / lam[0]; one block per column.
__global__ void __launch_bounds__(256) k_ritz_resid(const double *R, const double *X,
                                                    const double *lam, int M, double *res) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < M; i += 256) {
    const double d = R[(int64_t)c * M + i] - lam[c] * X[(int64_t)c * M + i];
    s += d * d;
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) res[c] = lam[0] > 0.0 ? sqrt(t) / lam[0] : 0.0;
}

// Relative size of an interpolation residual (against the column's largest entry)
// at or below which DEIM treats the column as dependent on the earlier ones.
constexpr double kDeimDependent = 1e-12;

// DEIM index selection on the n columns of Xi (M x n, column-major), one CTA.
__global__ void __launch_bounds__(1024) k_deim(const double *Xi, int M, int n, int32_t *rows_out,
                                               int *status) {
  __shared__ double A[RHMAX][RHMAX + 1];
  __shared__ double c[RHMAX];
  __shared__ int rows[RHMAX];
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ double xmax[32];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double *xj = Xi + (int64_t)j * M;
    if (j > 0) {
      for (int e = tid; e < j * j; e += blockDim.x) {
        const int a = e / j, b = e % j;
        A[a][b] = Xi[rows[a] + (int64_t)b * M];
      }
      for (int a = tid; a < j; a += blockDim.x) c[a] = xj[rows[a]];
      __syncthreads();
      if (tid == 0) {
        // Gaussian elimination with partial pivoting (first largest pivot), then
        // back substitution: c <- A^{-1} c
        for (int col = 0; col < j && !bad; ++col) {
          int piv = col;
          for (int r = col + 1; r < j; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
          if (!(fabs(A[piv][col]) > 0.0)) { bad = 1; break; }
          if (piv != col) {
            for (int q = 0; q < j; ++q) { const double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
            const double t = c[col]; c[col] = c[piv]; c[piv] = t;
          }
          for (int r = col + 1; r < j; ++r) {
            const double f = A[r][col] / A[col][col];
            for (int q = col; q < j; ++q) A[r][q] -= f * A[col][q];
            c[r] -= f * c[col];
          }
        }
        for (int r = j - 1; r >= 0 && !bad; --r) {
          double acc = c[r];
          for (int q = r + 1; q < j; ++q) acc -= A[r][q] * c[q];
          c[r] = acc / A[r][r];
        }
      }
      __syncthreads();
      if (bad) break;
    }
    double v = -1.0, xm = 0.0;
    int ix = INT32_MAX;
    bool nan = false;
    for (int i = tid; i < M; i += blockDim.x) {
      double r = xj[i];
      xm = fmax(xm, fabs(r));
      for (int b = 0; b < j; ++b) r -= Xi[i + (int64_t)b * M] * c[b];
      r = fabs(r);
      if (r != r) nan = true;
      if (r > v) { v = r; ix = i; }
    }
    if (nan) bad = 2;
#pragma unroll
    for (int o = 16; o >= 1; o /= 2) {
      const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, ix, o);
      if (v2 > v || (v2 == v && i2 < ix)) { v = v2; ix = i2; }
      xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    }
    if ((tid & 31) == 0) { rv[tid >> 5] = v; ri[tid >> 5] = ix; xmax[tid >> 5] = xm; }
    __syncthreads();
    if (tid == 0 && !bad) {
      double bv = rv[0], bx = xmax[0];
      int bi = ri[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        if (rv[w] > bv || (rv[w] == bv && ri[w] < bi)) { bv = rv[w]; bi = ri[w]; }
        bx = fmax(bx, xmax[w]);
      }
      bool dup = false;
      for (int a = 0; a < j; ++a) dup = dup || rows[a] == bi;
      // a residual at the rounding level of the column means the column lies in
      // the span of the earlier ones
      if (!(bv > kDeimDependent * bx) || dup) bad = 1;
      else {
        rows[j] = bi;
        rows_out[j] = bi;
      }
    }
    __syncthreads();
    if (bad) break;
  }
  if (tid == 0 && bad) set_status(status, bad == 2 ? DEV_NONFINITE : DEV_SINGULAR);
}

lrnr_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return LRNR_OK;
  if (e == cudaErrorMemoryAllocation) return LRNR_ENOMEM;
  return LRNR_ECUDA;
}

lrnr_status from_dev(int code) {
  switch (code) {
    case DEV_OK: return LRNR_OK;
    case DEV_NONFINITE: return LRNR_ENONFINITE;
    case DEV_TIMEOUT: return LRNR_ETIMEOUT;
    default: return LRNR_ESINGULAR;
  }
}

}  // namespace
}  // namespace lrnr

using namespace lrnr;

extern "C" {

lrnr_status lrnr_pod(const double *snapshots, int M, int64_t K, int n_modes, int n_iter,
                     double tol, double *basis_out, double *sigma_out, double *resid_out,
                     int *n_used, void *stream) {
  if (!snapshots || !basis_out || M < 1 || K < 1 || n_modes < 1 || n_modes > RHMAX ||
      n_iter < 0 || n_iter > 1000 || !(tol >= 0.0) || tol >= 1.0)
    return LRNR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LRNR_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LRNR_ECUDA;
  const int mk = (int)std::min<int64_t>(M, K);
  const int n = std::min(n_modes, mk);
  const int nb = std::min(std::min(mk, NBMAX), std::max(n + 8, 2 * n));
  // scratch: Q (M nb), Z (K nb, also the start signs), H, W (nb nb), lam (nb),
  // X (M n), T (K n), R (M n), split partials, status
  size_t part = 0;
  part = std::max(part, gemm_part_doubles(M, nb, K, sms));          // Y = S Z, and S Omega
  part = std::max(part, gemm_part_doubles((int)K, nb, M, sms));     // Z = S^T Q
  part = std::max(part, gemm_part_doubles(nb, nb, K, sms));         // H = Z^T Z
  part = std::max(part, gemm_part_doubles(M, n, nb, sms));          // X = Q W
  part = std::max(part, gemm_part_doubles((int)K, n, M, sms));      // T = S^T X
  part = std::max(part, gemm_part_doubles(M, n, K, sms));           // R = S T
  const size_t nQ = (size_t)M * nb, nZ = (size_t)K * nb, nH = (size_t)nb * nb;
  const size_t nX = (size_t)M * n, nT = (size_t)K * n;
  const size_t total = nQ + nZ + 2 * nH + nb + 2 * nX + nT + part + 1;
  double *ws = nullptr;
  cudaError_t e = cudaMalloc(&ws, total * sizeof(double));
  if (e != cudaSuccess) return to_status(e);
  double *Q = ws, *Z = Q + nQ, *H = Z + nZ, *W = H + nH, *lam = W + nH, *X = lam + nb;
  double *T = X + nX, *R = T + nT, *P = R + nX;
  int *status = reinterpret_cast<int *>(P + part);
  lrnr_status rc = LRNR_OK;
  auto fail = [&](cudaError_t err) {
    cudaFree(ws);
    return to_status(err);
  };
#define CKP(call)                             \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return fail(e_);   \
  } while (0)
  CKP(cudaMemsetAsync(status, 0, sizeof(int), st));
  // Q_0 = orth(S Omega)
  k_signs<<<(unsigned)((nZ + 255) / 256), 256, 0, st>>>(Z, K, nb);
  CKP(cudaGetLastError());
  {
    Gemm g = mat(snapshots, M, false);     // S (M x K)
    with_b(g, Z, K, false);                // Omega (K x nb)
    g.C = Q; g.ldc = M; g.m = M; g.n = nb; g.k = K;
    CKP(dgemm(g, P, sms, st));
  }
  k_orth<<<1, 1024, 0, st>>>(Q, M, nb, status);
  CKP(cudaGetLastError());
  for (int it = 0; it <= n_iter; ++it) {
    {
      Gemm g = mat(snapshots, M, true);    // S^T (K x M)
      with_b(g, Q, M, false);              // Q (M x nb)
      g.C = Z; g.ldc = K; g.m = (int)K; g.n = nb; g.k = M;
      CKP(dgemm(g, P, sms, st));
    }
    if (it == n_iter) break;
    {
      Gemm g = mat(snapshots, M, false);   // S
      with_b(g, Z, K, false);              // Z (K x nb)
      g.C = Q; g.ldc = M; g.m = M; g.n = nb; g.k = K;
      CKP(dgemm(g, P, sms, st));
    }
    k_orth<<<1, 1024, 0, st>>>(Q, M, nb, status);
    CKP(cudaGetLastError());
  }
  // Rayleigh-Ritz: H = Z^T Z, H = W diag(lam) W^T, X = Q W[:, :n]
  {
    Gemm g = mat(Z, K, true);
    with_b(g, Z, K, false);
    g.C = H; g.ldc = nb; g.m = nb; g.n = nb; g.k = K;
    CKP(dgemm(g, P, sms, st));
  }
  CKP(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kJacobiSmem));
  k_jacobi<<<1, 1024, kJacobiSmem, st>>>(H, nb, lam, W, status);
  CKP(cudaGetLastError());
  {
    Gemm g = mat(Q, M, false);
    with_b(g, W, nb, false);
    g.C = X; g.ldc = M; g.m = M; g.n = n; g.k = nb;
    CKP(dgemm(g, P, sms, st));
  }
  k_canon_sign<<<n, 256, 0, st>>>(X, M);
  CKP(cudaGetLastError());
  if (resid_out) {
    // R = S (S^T X); resid_c = ||R_c - lam_c X_c|| / lam_0
    {
      Gemm g = mat(snapshots, M, true);
      with_b(g, X, M, false);
      g.C = T; g.ldc = K; g.m = (int)K; g.n = n; g.k = M;
      CKP(dgemm(g, P, sms, st));
    }
    {
      Gemm g = mat(snapshots, M, false);
      with_b(g, T, K, false);
      g.C = R; g.ldc = M; g.m = M; g.n = n; g.k = K;
      CKP(dgemm(g, P, sms, st));
    }
    k_ritz_resid<<<n, 256, 0, st>>>(R, X, lam, M, resid_out);
    CKP(cudaGetLastError());
  }
  std::vector<double> hl(nb);
  int hst = 0;
  CKP(cudaMemcpyAsync(hl.data(), lam, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  CKP(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKP(cudaStreamSynchronize(st));
  if (hst != DEV_OK) {
    cudaFree(ws);
    return from_dev(hst);
  }
  // keep the leading modes with sigma_j > tol * sigma_1
  std::vector<double> sig(n);
  int used = 0;
  for (int j = 0; j < n; ++j) sig[j] = std::sqrt(std::max(hl[j], 0.0));
  while (used < n && sig[used] > 0.0 && sig[used] > tol * sig[0]) ++used;
  if (used > 0) {
    CKP(cudaMemcpyAsync(basis_out, X, sizeof(double) * (size_t)M * used, cudaMemcpyDeviceToDevice,
                        st));
    if (sigma_out)
      CKP(cudaMemcpyAsync(sigma_out, sig.data(), sizeof(double) * used, cudaMemcpyHostToDevice, st));
  }
  CKP(cudaStreamSynchronize(st));
  cudaFree(ws);
  if (n_used) *n_used = used;
#undef CKP
  return rc;
}

lrnr_status lrnr_deim_rows(const double *basis, int M, int n, int32_t *rows_out, void *stream) {
  if (!basis || !rows_out || M < 1 || n < 1 || n > RHMAX || n > M) return LRNR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *status = nullptr;
  cudaError_t e = cudaMalloc(&status, sizeof(int));
  if (e != cudaSuccess) return to_status(e);
  int hst = 0;
  e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_deim<<<1, 1024, 0, st>>>(basis, M, n, rows_out, status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(status);
  if (e != cudaSuccess) return to_status(e);
  return from_dev(hst);
}

}  // extern "C"
