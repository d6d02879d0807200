/*
 * lrnr.h -- C ABI of the GB300 (sm_103a) FastLRNR / sparse physics-informed
 * backpropagation library (liblrnr.so).
 *
 * The library evaluates a low rank neural representation (LRNR) and its
 * EIM-reduced form (FastLRNR) at many collocation points, carries the input
 * derivatives u, u_t, u_x, u_xx forward with it, forms the convection-diffusion-
 * reaction residual and physics-informed loss, and returns the exact gradient of
 * that loss with respect to the coefficients s and the biases b.
 *
 * Notation (paper: "FastLRNR and Sparse Physics Informed Backpropagation").
 *   L      number of activated (hidden) layers; the network has L+1 weight layers
 *          l = 0..L (the paper's 1..L+1, Sec. 2.1 Eq. 2.1).
 *   M      hidden width; input width 2 (x, t), output width 1 (u) (Sec. 2.1).
 *   r[l]   rank of weight layer l, W^l = U^l diag(s^l) V^l^T (Sec. 2.1 Eq. 2.2).
 *          U^l is M_l x r[l], V^l is M_{l-1} x r[l] (V has as many rows as the
 *          layer's input; the printed M_l rows cannot multiply z^{l-1}).
 *          Constraints: 1 <= r[0] <= 2, 1 <= r[l] <= 64 for 0 < l < L, r[L] == 1.
 *          Ranks are padded to 8, 16, 32 or 64.  Full-width FP32 takes every padded
 *          rank (at 32 and 64 a point is spread over rank / 16 threads); FastLRNR
 *          FP32 takes any padded rank with rhat <= 16 (ranks 32 and 64 through
 *          reduced coordinates, Eq. 2.8 regrouped per layer); on the tensor cores
 *          the full-width network at rank 64 runs in LRNR_BF16 only; other
 *          combinations, and shapes whose per-CTA shared memory would not fit,
 *          return LRNR_ENOTSUP.
 *   s      coefficients, per PDE instance a vector of sum(r) floats, layer-major.
 *   b      biases, b^l of length M_l; sum over layers = L*M + 1 ("sum_m").
 *   mu     (beta, nu, rho): N[u] = u_t + beta u_x - nu u_xx - rho u (1-u)
 *          on (0, 2pi) x (0, 1), u(x,0) = sin x, u(0,t) = u(2pi,t) (Sec. 4 Eq. 4.1).
 *
 * Conventions.
 *   Memory: every pointer documented "device" is caller-owned CUDA device memory
 *     on the model's device; "host" pointers are ordinary host memory.  The
 *     library owns only the model handle, its packed copies of the bases and a
 *     workspace for per-tile partial sums (grown by lrnr_reserve or on first use).
 *   Streams: every launch goes on the given cudaStream_t (passed as void*; NULL
 *     = legacy default stream).  lrnr_residual, lrnr_residual_grad and
 *     spinprop_step do no host synchronisation and can be captured in a CUDA graph
 *     once the workspace is large enough (otherwise they return LRNR_ENOTREADY
 *     while the stream is capturing).  fastlrnr_select_rows synchronises.
 *   Errors: functions return a status and never abort.  Launch failures return
 *     LRNR_ECUDA; errors found by kernels (non-finite inputs, iteration caps) are
 *     recorded in a device status word read by lrnr_last_device_status.
 *   Concurrency: calls on one model share its workspace and must be ordered
 *     (one stream, or explicit events).
 */
#ifndef LRNR_H
#define LRNR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRNR_OK = 0,
  LRNR_EINVAL = 1,      /* bad argument: null pointer, size or rank out of range */
  LRNR_ENOMEM = 2,      /* device allocation failed */
  LRNR_ECUDA = 3,       /* a CUDA call or kernel launch failed */
  LRNR_ESINGULAR = 4,   /* EIM: the interpolation block P^T Xi is singular */
  LRNR_EEARLYSTOP = 5,  /* reserved: EIM stop is reported through rhat_used */
  LRNR_ETIMEOUT = 6,    /* a device wait reached its iteration cap */
  LRNR_ENOTREADY = 7,   /* FastLRNR layers not selected, or workspace too small while capturing */
  LRNR_ENONFINITE = 8,  /* a kernel met a NaN or infinity in its input */
  LRNR_ENOTSUP = 9,     /* the (form, precision) pair is not implemented */
  LRNR_ETOOBIG = 10     /* batch larger than the fixed scratch of lrnr_residual_grad_noalloc */
} lrnr_status;

typedef enum {
  LRNR_FP32 = 0,        /* FP32 SIMT everywhere (reference precision of the GPU path) */
  LRNR_TF32 = 1,        /* tcgen05 kind::tf32: operands rounded to TF32 (10-bit mantissa,
                           nearest), FP32 accumulation in TMEM (both forms; padded
                           ranks up to 32) */
  LRNR_BF16 = 2,        /* tcgen05 BF16 operands, FP32 accumulation in TMEM (both forms;
                           the reduced network is an LRNR of width rhat, Sec. 2.2 Eq. 2.8) */
  LRNR_BF16X3 = 3       /* split-BF16 (bf16 x 3): every operand as three BF16 pieces
                           hi + mid + lo, the six products with piece orders adding up to
                           at most two (hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid),
                           FP32 accumulation in TMEM; full width: padded ranks 16 and 32 */
} lrnr_precision;

typedef enum { LRNR_FULL = 0, LRNR_FAST = 1 } lrnr_form;
typedef enum { LRNR_LOSS_MSE = 0, LRNR_LOSS_L1 = 1 } lrnr_loss;

typedef struct lrnr_model lrnr_model;

/*
 * A batch of PDE instances and their collocation points (Sec. 3.2 Eq. 3.5-3.6,
 * Sec. 4 Eq. 4.1).  All arrays are device memory; instance i owns the points
 * [off[i], off[i+1]) of each class.  Totals are host values and must equal
 * int_off[n_inst], ic_off[n_inst], bc_off[n_inst].  The kernels check the offsets
 * on the device: offsets that decrease, start below zero or end past the totals
 * make the call process no point (lrnr_residual writes no output; loss and
 * gradients are zero; spinprop_step applies its Adam update with a zero loss
 * gradient) and record LRNR_EINVAL for lrnr_last_device_status.
 *
 * norm (optional, device int64 [n_inst][3]): the denominators of the three MSE
 * means of Eq. 3.5 per instance (interior, initial, periodic), used in place of
 * the instance's own counts in this batch.  The gradient is a sum over collocation
 * points (Sec. 2.3), so when one instance's points are split across several calls
 * (ranks of a data-parallel run), each call given the whole instance's counts
 * returns partial losses and gradients that add up to the instance's; NULL = the
 * counts in this batch.  A count must be >= 1 where the batch has points of that
 * class.  L1 losses (plain sums) ignore it.
 */
typedef struct {
  int32_t n_inst;                 /* number of instances (mu, s pairs), >= 1 */
  int64_t n_int, n_ic, n_bc;      /* host: total interior points, initial points, periodic pairs */
  const float *beta, *nu, *rho;   /* device [n_inst]: mu = (beta, nu, rho) */
  const float *s;                 /* device [n_inst][sum_r]: coefficients (ignored by spinprop_step) */
  const int64_t *int_off;         /* device [n_inst+1] CSR offsets into x_int/t_int */
  const int64_t *ic_off;          /* device [n_inst+1] offsets into x_ic */
  const int64_t *bc_off;          /* device [n_inst+1] offsets into t_bc */
  const float *x_int, *t_int;     /* device [n_int]: interior points (x, t) */
  const float *x_ic;              /* device [n_ic]: initial points (x, 0), target sin x */
  const float *t_bc;              /* device [n_bc]: periodic pairs (0, t) and (2pi, t) */
  const int64_t *norm;            /* device [n_inst][3] MSE denominators, or NULL (see above) */
} lrnr_batch;

/*
 * lrnr_build -- create a model from frozen bases (U*, V*, b*) (Sec. 2.1 Eq. 2.4).
 *   L, M : hidden layers (1..16) and width (1..4096).
 *   r    : host [L+1] ranks (constraints above).
 *   U, V, b : host arrays of L+1 pointers to row-major FP64 matrices
 *          U[l]: M_l x r[l], V[l]: M_{l-1} x r[l], b[l]: M_l, with M_{-1} = 2,
 *          M_l = M for l < L and M_L = 1.  Copied; the caller keeps ownership.
 *   out  : receives the handle (on the current CUDA device).
 * Returns LRNR_EINVAL for bad sizes or null pointers, LRNR_ENOMEM / LRNR_ECUDA.
 */
lrnr_status lrnr_build(int L, int M, const int *r, const double *const *U,
                       const double *const *V, const double *const *b, lrnr_model **out);

/*
 * lrnr_snapshots -- FP64 hidden states z^layer = tanh(U s V^T z + b) of the exact
 * LRNR (the EIM snapshots of Sec. 4) at n_pts points for n_s coefficient draws.
 *   layer : hidden layer 0..L-1.
 *   x, t  : device FP64 [n_pts].  s: device FP64 [n_s][sum_r].
 *   out   : device FP64, M x (n_s*n_pts), column-major; column j*n_pts + p holds
 *           the state for draw j at point p.
 */
lrnr_status lrnr_snapshots(lrnr_model *m, int layer, int64_t n_pts, const double *x,
                           const double *t, int n_s, const double *s, double *out,
                           void *stream);

/*
 * fastlrnr_select_rows -- EIM row selection for hidden layer `layer` and
 * installation of its reduced bases (Sec. 2.2 Eq. 2.7-2.8):
 *   Uhat = P^T U^l, bhat = P^T b^l, Vhat = (P^T Xi)^{-T} Xi^T V^{l+1}.
 * Greedy (rows_in == NULL): classic EIM on `snapshots` (device FP64, M x K,
 *   column-major, not modified), at most `rhat` (1..32) steps; picks the column
 *   with the largest max-abs residual and, in it, the row of largest |value|
 *   (lowest index on exact ties); stops early when that max-abs <= tol (absolute).
 *   FP64 throughout, no fused multiply-add in the residual update, so the rows
 *   match an IEEE FP64 reference bit for bit.
 * Given (rows_in != NULL): device int32 [rhat] distinct rows and Xi_in, device
 *   FP64 M x rhat column-major; P^T Xi must be invertible (LRNR_ESINGULAR).
 * Outputs: rows_out (device int32 [rhat], may be NULL), Xi_out (device FP64
 *   M x rhat column-major, may be NULL), *rhat_used (host) = rows kept.
 * Synchronises `stream`.  After every layer 0..L-1 has been selected, LRNR_FAST
 * calls are allowed.
 */
lrnr_status fastlrnr_select_rows(lrnr_model *m, int layer, const double *snapshots, int64_t K,
                                 int rhat, double tol, const int32_t *rows_in,
                                 const double *Xi_in, int32_t *rows_out, double *Xi_out,
                                 int *rhat_used, void *stream);

/*
 * lrnr_pod -- POD basis of a snapshot matrix: the leading left singular vectors
 * Xi of S, the basis of the DEIM reading of Sec. 2.2 Eq. 2.7.  FP64 throughout.
 *   snapshots: device FP64 M x K, column-major, not modified.  n_modes: 1..32
 *   (at most min(M, K) are returned).  Method: block subspace iteration on S S^T
 *   with nb = min(M, K, 64, max(n_modes + 8, 2 n_modes)) columns, started from
 *   S times a K x nb sign matrix (a fixed counter hash), n_iter (0..1000)
 *   iterations Q <- orth(S (S^T Q)), then Rayleigh-Ritz on (S^T Q)^T (S^T Q) by
 *   cyclic Jacobi.  Accuracy of mode j grows like (sigma_{nb+1} / sigma_j)^(2 n_iter).
 *   Each returned column is scaled by +-1 so that its entry of largest magnitude
 *   (lowest index among exact ties) is positive.  Modes with sigma_j <= tol * sigma_1
 *   (0 <= tol < 1) are dropped.
 *   Outputs: basis_out device FP64 M x n_modes column-major (the first *n_used
 *   columns are written); sigma_out device FP64 [n_modes] or NULL; resid_out
 *   device FP64 [n_modes] or NULL: ||S S^T xi_j - sigma_j^2 xi_j||_2 / sigma_1^2 of
 *   each returned mode; *n_used (host, may be NULL).
 *   Allocates scratch ((M + K) * nb doubles and split partials), synchronises
 *   `stream`, runs on the current device.  LRNR_ETIMEOUT if the Jacobi sweeps do
 *   not converge (cap 64 sweeps), LRNR_ESINGULAR if orthonormalisation fails.
 */
lrnr_status lrnr_pod(const double *snapshots, int M, int64_t K, int n_modes, int n_iter,
                     double tol, double *basis_out, double *sigma_out, double *resid_out,
                     int *n_used, void *stream);

/*
 * lrnr_deim_rows -- DEIM index selection (the sampling matrix P of Sec. 2.2
 * Eq. 2.7 for a given basis): p_1 = argmax_i |xi_1(i)|; step j solves
 * (P^T Xi_{j-1}) c = P^T xi_j (Gaussian elimination, partial pivoting, FP64) and
 * takes p_j = argmax_i |xi_j(i) - (Xi_{j-1} c)(i)|, lowest index among exact ties.
 *   basis: device FP64 M x n column-major (n 1..32, n <= M); rows_out: device
 *   int32 [n].  LRNR_ESINGULAR when the columns are dependent (a zero residual or
 *   pivot), LRNR_ENONFINITE on NaN.  Synchronises `stream`.  The rows and basis are
 *   what fastlrnr_select_rows takes as rows_in / Xi_in.
 */
lrnr_status lrnr_deim_rows(const double *basis, int M, int n, int32_t *rows_out, void *stream);

/*
 * lrnr_residual -- forward only (Sec. 2.1 Eq. 2.1 / Sec. 2.2 Eq. 2.8 and Eq. 4.1).
 * Writes, for interior points, u, u_t, u_x, u_xx and the residual N[u] (device
 * FP32 [n_int] each), the initial residual u(x,0) - sin x (device [n_ic]) and the
 * periodic residual u(0,t) - u(2pi,t) (device [n_bc]).  Any output may be NULL.
 */
lrnr_status lrnr_residual(lrnr_model *m, lrnr_form form, lrnr_precision prec,
                          const lrnr_batch *bt, float *u, float *u_t, float *u_x, float *u_xx,
                          float *res, float *res_ic, float *res_bc, void *stream);

/*
 * lrnr_residual_grad -- loss and exact gradient per instance (Sec. 2.3, Eq. 3.5 /
 * Eq. 3.6).  MSE: w0 mean R^2 + w1 mean B_ic^2 + w2 mean B_bc^2 (a term with no
 * points is absent); L1: w0 sum|R| + w1 sum|B_ic| + w2 sum|B_bc| (sign(0) = 0).
 *   w        : host float[3] or NULL (= 1, 1, 1).
 *   loss_out : device [n_inst].  dL_ds: device [n_inst][sum_r].
 *   dL_db    : device [n_inst][sum_m] or NULL; FastLRNR puts the gradient of the
 *              kept rows at their positions and zero elsewhere.
 * Results are deterministic: partial sums are reduced in a fixed order.
 */
lrnr_status lrnr_residual_grad(lrnr_model *m, lrnr_form form, lrnr_precision prec,
                               const lrnr_batch *bt, lrnr_loss loss, const float *w,
                               float *loss_out, float *dL_ds, float *dL_db, void *stream);

/*
 * spinprop_step -- n_steps Adam steps on s (Sec. 3.2 Eq. 3.6-3.7, Sec. 4), each a
 * fused residual + gradient pass followed by the update
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   s -= lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps),   k = ++(*step),
 * with g = dL/ds + lambda_loc sign(s - s_anchor) when s_anchor != NULL.
 *   s_inout, adam_m, adam_v : device [n_inst][sum_r] (bt->s is ignored).
 *   step     : device int64 [1], Adam step count, incremented on the device.
 *   loss_out : device [n_inst] or NULL: loss (with the locality term) of the last step.
 */
lrnr_status spinprop_step(lrnr_model *m, lrnr_form form, lrnr_precision prec,
                          const lrnr_batch *bt, lrnr_loss loss, const float *w,
                          float *s_inout, float *adam_m, float *adam_v, int64_t *step,
                          int n_steps, float lr, float beta1, float beta2, float eps,
                          float lambda_loc, const float *s_anchor, float *loss_out,
                          void *stream);

/*
 * lrnr_residual_grad_noalloc -- the FastLRNR FP32 loss and gradient of
 * lrnr_residual_grad (form LRNR_FAST, precision LRNR_FP32, same arguments and
 * results), for callers that cannot allocate device memory: applications whose
 * device memory belongs to another allocator or is held to a fixed budget, and
 * latency-critical loops that cannot afford the device-wide synchronisation of
 * cudaMalloc / cudaFree.  It allocates nothing: its scratch (tile offsets,
 * per-tile partial sums and the kernel's per-CTA layer store) is a fixed 32 MiB
 * array in the library's device image, held by every GPU that loads the library
 * until the process exits.  The paper has no counterpart; this is an interface
 * option.
 *   Capacity: 4*(n_inst+1) bytes (rounded up to 256), plus one partial row of
 *     4*(1 + (L+1)*RM + L*RH + 1) bytes per tile of nt points (nt = 128 unless
 *     lrnr_set_tuning chose 32 or 64; a periodic tile holds nt/2 pairs), plus the
 *     layer store of at least one CTA, 4*(4*(L-1)*RM + 4*L*RH)*nt bytes, must fit
 *     in 32 MiB (RM, RH: rank and EIM rows rounded up to 8 or 16); larger batches
 *     return LRNR_ETOOBIG before any GPU work.  The grid is capped at the CTAs
 *     whose stores fit in what the partial rows leave of the 32 MiB, so large
 *     batches run on fewer SMs (at L = 5, r = rhat = 16, nt = 128 a store is
 *     288 KiB: at most 113 CTAs fit beside no partial rows); results do not depend
 *     on the grid.  At L = 5, r = rhat = 16 the batch limit is about 5.9 million
 *     points (one CTA's store left).
 *   Set-up: the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   Sharing: every call uses the same array and leaves its contents behind (all
 *     of it is rewritten before it is read, nothing relies on zeros); calls whose
 *     kernels overlap on the GPU (different streams, or several host threads)
 *     race on it and must be serialised by the caller.
 *   Requires every hidden layer selected (fastlrnr_select_rows), else
 *     LRNR_ENOTREADY; the model's own workspace is not used or grown.  The tile
 *     size, CTA cap (lrnr_set_tuning) and wait cap (lrnr_set_wait_limit) of the
 *     model apply as in lrnr_residual_grad.
 *   Ranks: padded ranks 8 and 16 (the rank-r FastLRNR kernel); the
 *     reduced-coordinate kernel for padded ranks 32 and 64 runs only through
 *     lrnr_residual_grad and spinprop_step, and here returns LRNR_ENOTSUP.
 */
lrnr_status lrnr_residual_grad_noalloc(lrnr_model *m, const lrnr_batch *bt, lrnr_loss loss,
                                       const float *w, float *loss_out, float *dL_ds,
                                       float *dL_db, void *stream);

/*
 * lrnr_adam_update -- one Adam step on s from a given gradient: the update of
 * spinprop_step (Sec. 4; l1 locality subgradient of Eq. 3.7 when s_anchor != NULL)
 * applied to dL/ds computed elsewhere, e.g. the sum over ranks of the partial
 * gradients of one instance whose collocation points are split across GPUs
 * (lrnr_residual_grad with lrnr_batch.norm, then an all-reduce).
 *   grad     : device [n_inst][sum_r] dL/ds.
 *   s_inout, adam_m, adam_v : device [n_inst][sum_r], updated in place.
 *   step     : device int64 [1]; the update uses k = *step + 1 and then advances it.
 *   loss_in  : device [n_inst] or NULL; loss_out (device [n_inst] or NULL) receives
 *              loss_in + lambda_loc * sum |s - s_anchor| at the s before the update.
 * Two kernel launches on `stream`, no allocation, no host synchronisation.
 * Errors: LRNR_EINVAL for null arrays, n_inst or sum_r < 1, or hyper-parameters out
 * of range (as spinprop_step); LRNR_ECUDA if a launch fails.
 */
lrnr_status lrnr_adam_update(int32_t n_inst, int32_t sum_r, const float *grad, float *s_inout,
                             float *adam_m, float *adam_v, int64_t *step, float lr, float beta1,
                             float beta2, float eps, float lambda_loc, const float *s_anchor,
                             const float *loss_in, float *loss_out, void *stream);

/*
 * lrnr_copy_pinned -- copy `bytes` bytes from `src` to `dst` with a kernel on `stream`
 * that reads and writes through the unified address space (not an operation of the
 * paper: it carries a step's batch and s in from the host and s and the loss back out,
 * in less time than a copy-engine transfer at these sizes, and is captured into a CUDA
 * graph like any launch).
 *   dst, src : each either device memory of the current device (or managed memory) or
 *              page-locked host memory (cudaHostAlloc / cudaMallocHost /
 *              cudaHostRegister, e.g. a pinned torch tensor); any byte alignment
 *              (16-byte loads where both addresses agree modulo 16).  Host bytes are
 *              read uncached, so host writes made before the launch are seen.
 *   The ranges must not overlap.  The caller owns both buffers and keeps them alive
 *   until the copy has run; host results are complete once `stream` has been
 *   synchronised.  bytes = 0 does nothing.
 * Errors: LRNR_EINVAL for a null pointer with bytes > 0, pageable host memory, memory
 * of another device, or overlapping ranges; LRNR_ECUDA if the launch fails.
 */
lrnr_status lrnr_copy_pinned(void *dst, const void *src, size_t bytes, void *stream);

/* lrnr_reserve -- size the workspace for batches of up to max_points collocation
 * points (interior + initial + 2 x pairs) in up to max_inst instances.  Call it
 * before capturing a CUDA graph. */
lrnr_status lrnr_reserve(lrnr_model *m, int64_t max_points, int32_t max_inst);

/* lrnr_set_tuning -- override the launch shape used for (form, prec): points per
 * tile `nt` (32, 64 or 128; 0 = automatic) and a cap on resident CTAs per SM
 * `ctas_per_sm` (1..8; 0 = automatic).  Shapes that do not fit the kernel's
 * shared memory fall back to the automatic choice.  Results change only by
 * rounding (tiles regroup the partial sums).  Set by the autotuner
 * (paper_2410_04001_gb300/autotune.py), which times the candidates on the
 * caller's batch.  The tensor-core form has a fixed shape (128 points, 1 CTA). */
lrnr_status lrnr_set_tuning(lrnr_model *m, lrnr_form form, lrnr_precision prec, int nt,
                            int ctas_per_sm);

/* lrnr_set_wait_limit -- iteration cap of the tensor-core kernel's mbarrier waits
 * (tensor-core MMA completion and bulk-copy arrival; the paper has no counterpart):
 * `polls` >= 0 polls per wait (each poll may block briefly in the barrier), < 0 =
 * the default (2^20).  A wait that reaches the cap records LRNR_ETIMEOUT in the
 * device status (lrnr_last_device_status) and the kernel returns after waiting,
 * with a fixed bound of its own, for the MMAs and copies it still has outstanding;
 * no other state is changed.  A cap of 0 makes every call time out: it exists to
 * exercise that path. */
lrnr_status lrnr_set_wait_limit(lrnr_model *m, int64_t polls);

/* lrnr_model_info -- host outputs (any may be NULL): L, M, sum_r, sum_m and
 * whether every hidden layer has reduced bases (fast_ready). */
lrnr_status lrnr_model_info(const lrnr_model *m, int *L, int *M, int *sum_r, int *sum_m,
                            int *fast_ready);

/* lrnr_timing -- when enable != 0, record a CUDA event pair on the launch stream
 * around every tile kernel (the fused residual / adjoint kernel) of later calls.
 * Recording is captured by CUDA graphs like any stream work. */
lrnr_status lrnr_timing(lrnr_model *m, int enable);

/* lrnr_timing_read -- wait for the recorded events, return the summed kernel time
 * (host, milliseconds) and the number of timed launches since the last read (or
 * since lrnr_timing), and start a new count.  Pairs recorded while the stream was
 * being captured into a CUDA graph belong to the graph: every replay re-records
 * them and every read reports them again, so replay the graph once before each
 * read.  lrnr_timing releases them. */
lrnr_status lrnr_timing_read(lrnr_model *m, double *ms_total, int64_t *launches);

/* lrnr_measure_peaks -- compute-throughput microbenchmarks of the current device
 * (the roofline denominators of the FP32 SIMT kernels; the paper has no counterpart):
 * FP32 fused multiply-add, scalar and packed two-lane (TFLOP/s, 2 flops per lane
 * FMA), tanh.approx.f32 and tanhf (10^9 results/s), FP64 FMA (TFLOP/s), and the SM
 * clock while they ran (MHz, from clock64 over CUDA-event time).  Runs on `stream`
 * (a few tens of ms), allocates and frees a few KB of device memory, synchronises.
 * Errors: LRNR_EINVAL (out NULL), LRNR_ENOMEM, LRNR_ECUDA. */
typedef struct {
  double fp32_fma_tflops, fp32_fma2_tflops, tanh_approx_gops, tanhf_gops, fp64_fma_tflops;
  double sm_mhz;
  int sms;
} lrnr_peaks;
lrnr_status lrnr_measure_peaks(lrnr_peaks *out, void *stream);

/* lrnr_last_device_status -- synchronises the device, returns and clears the
 * status word written by kernels (LRNR_OK if none): LRNR_ENONFINITE, LRNR_ETIMEOUT,
 * LRNR_ESINGULAR, or LRNR_EINVAL for batch offsets that failed the device check. */
lrnr_status lrnr_last_device_status(lrnr_model *m);

const char *lrnr_status_string(lrnr_status s);

void lrnr_destroy(lrnr_model *m);

#ifdef __cplusplus
}
#endif

#endif /* LRNR_H */
