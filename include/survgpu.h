/*
 * survgpu.h - C ABI of libsurvgpu.so: penalised Cox (Breslow ties) and
 * Fine-Gray regression by cyclic coordinate descent (CCD) on one GB300 GPU.
 *
 * The library computes, for one coordinate j at a time, the gradient and
 * Hessian of the log partial likelihood (Cox, Eq. cox_l, Section 2.1) or of
 * the log pseudo-likelihood (Fine-Gray, Eq. fg_l, Section 2.2) through risk-set
 * prefix sums over subjects arranged by decreasing time (Section 2.7, Eqs.
 * cox_g, cox_h, fg_g, fg_h), takes a trust-region Newton step on the L1/L2
 * penalised objective (Sections 2.3, 2.4) and updates eta = X beta.  All of
 * that runs in CUDA kernels; the host only validates sizes, stages buffers and
 * reads the result.
 *
 * Memory: every array pointer may point to host memory or to device memory of
 * the current device; the library asks the CUDA runtime which one it is.
 * Host arrays are copied to device workspace inside the call (and results
 * copied back), so a host-buffer call includes those transfers.  The caller
 * owns every buffer it passes; the library never frees caller memory and keeps
 * no pointer to it after the call returns.
 *
 * Threading: calls on different workspaces may run concurrently on different
 * streams.  A workspace must not be used by two calls at the same time.
 *
 * Errors: every entry point returns SURV_OK (0) on success, a positive warning
 * or a negative error code.  surv_strerror() names a code and
 * surv_last_error() returns a message with details for the calling thread.
 * On error no output array is written, except that beta_inout may hold the
 * last iterate for SURV_W_NOT_CONVERGED and SURV_E_DEVICE_TIMEOUT.
 */
#ifndef SURVGPU_H
#define SURVGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define SURV_OK 0
#define SURV_W_NOT_CONVERGED 1    /* max_sweeps reached; beta holds the last iterate */
#define SURV_E_INVALID (-1)       /* null pointer, negative size, bad enum, bad j   */
#define SURV_E_UNSORTED (-2)      /* time is not non-increasing                     */
#define SURV_E_STATUS (-3)        /* status code outside {0,1} (Cox) / {0,1,2} (FG)  */
#define SURV_E_NONFINITE (-4)     /* NaN or Inf in X, beta or penalty factors        */
#define SURV_E_NO_EVENTS (-5)     /* no event (Cox) / no primary event (FG)          */
#define SURV_E_CUDA (-6)          /* a CUDA runtime call failed                      */
#define SURV_E_DEVICE_TIMEOUT (-7)/* a device-side wait gave up (bounded spin)       */
#define SURV_E_NOMEM (-8)         /* device allocation failed                        */
#define SURV_E_INDEX (-9)         /* CSC col_ptr/row_idx malformed or out of range   */

/* ---- enumerations ------------------------------------------------------ */
#define SURV_CSC 0            /* column-compressed: col_ptr, row_idx, values   */
#define SURV_DENSE 1          /* dense column-major, leading dimension n        */

#define SURV_F32 0
#define SURV_F64 1
#define SURV_BF16 2      /* dense X only: bfloat16 values, widened on the device
                            to the working precision (exactly: every bfloat16 is
                            an FP32 value), so the fit is that of the rounded X */

#define SURV_COX 0
#define SURV_FG 1

#define SURV_PEN_NONE 0
#define SURV_PEN_L1 1         /* pi = -sum_j lambda pf_j |beta_j|       (Section 2.3) */
#define SURV_PEN_L2 2         /* pi = -sum_j lambda pf_j beta_j^2 / 2  (1/tau = lambda pf) */

#define SURV_PREC_F32C 0      /* FP32 exp/scans with float-float (compensated) carries,
                                 FP64 Newton step, logs and final scalars            */
#define SURV_PREC_F64 1       /* FP64 throughout                                     */

/* ---- data -------------------------------------------------------------- */
/* Survival data in decreasing-time order (Section 2.7).
 *   time    [n]  int32, non-increasing (validated: SURV_E_UNSORTED).  Use
 *                surv_sort_desc() to obtain the order of unsorted data.
 *   status  [n]  int8: 0 censored, 1 event (Cox) / primary event (FG),
 *                2 competing event (FG only).
 *   layout = SURV_CSC:
 *     col_ptr [p+1] int64, col_ptr[0] = 0, non-decreasing; nnz = col_ptr[p].
 *     row_idx [nnz] int32, strictly increasing inside each column, in [0,n).
 *     values  [nnz] of dtype (SURV_F32 or SURV_F64), or NULL for an
 *             all-ones (indicator) matrix.
 *   layout = SURV_DENSE:
 *     values  [n*p] of dtype (SURV_F32, SURV_F64 or SURV_BF16),
 *             column-major (element (i,j) at j*n+i);
 *     col_ptr and row_idx are ignored.
 */
typedef struct surv_data {
  int64_t n;
  int64_t p;
  const int32_t *time;
  const int8_t *status;
  int32_t layout;
  int32_t dtype;
  const int64_t *col_ptr;
  const int32_t *row_idx;
  const void *values;
} surv_data;

typedef struct surv_workspace surv_workspace;   /* opaque device workspace */

/* ---- options ----------------------------------------------------------- */
typedef struct surv_opts {
  int32_t penalty;               /* SURV_PEN_*                                      */
  int32_t precision;             /* SURV_PREC_*                                     */
  double lambda;                 /* L1: gamma; L2: 1/tau (Section 2.3)              */
  const double *penalty_factor;  /* [p] multiplier per coordinate (0 = unpenalised),
                                    host or device, or NULL for all ones            */
  double tol;                    /* stop when |f_k - f_{k-1}| / |f_k| < tol after a
                                    sweep, f = loglik + penalty                     */
  int32_t max_sweeps;            /* cap on full sweeps (>= 0)                       */
  int32_t flags;                 /* SURV_FLAG_* bits, normally 0                    */
  double wait_limit_s;           /* bound on every device-side wait of the grid-wide
                                    exchange; <= 0 selects 2 seconds                */
  void *stream;                  /* cudaStream_t, or NULL for the default stream    */
  surv_workspace *workspace;     /* reusable workspace, or NULL (allocate per call) */
} surv_opts;

/* Test only: one CTA of the CCD kernel never announces its first exchange,
 * so every other CTA's bounded wait expires; the call must then return
 * SURV_E_DEVICE_TIMEOUT and leave the device usable. */
#define SURV_FLAG_TEST_STALL 1
/* Run a fit as one persistent cooperative launch (grid-wide exchanges in
 * device memory, bounded waits) instead of the default schedule of two
 * kernels per coordinate replayed as a CUDA graph, one replay per sweep.
 * Both schedules compute the same quantities in the same order of
 * coordinates; this flag exists to compare them.  loglik_grad_hess always
 * uses the persistent kernel. */
#define SURV_FLAG_PERSISTENT 2
/* cox_cv_path only, with ctas_per_fit = 0: time one sweep of the batched
 * schedule for each of a few CTA-per-fit counts around the default and, for
 * CSC data, each of the two forms of the row pass (one warp reduction per
 * tie-group end, or lane scans per tile for warps that hold many ends) and,
 * in the FP32 mode, three tile shapes (see surv_cv_info.tile_form), every
 * candidate from the same cold start; run the path with the fastest, and
 * keep the choice in the workspace for later calls with the same shape
 * (n, p, number of fits, layout, precision). */
#define SURV_FLAG_CV_TUNE 4
/* cox_fit only (CSC data, SURV_PREC_F32C): the sparse-numerator form, not
 * in the paper.  The same CCD with the same l'_j and l''_j, computed from
 * the nonzeros of column j alone:
 *   sum_k d_k N1_k/Den_k = sum_t x_t e_t Lambda(g_t),
 *   sum_k d_k N2_k/Den_k = sum_t x_t^2 e_t Lambda(g_t),
 *   sum_k d_k (N1_k/Den_k)^2 = sum_t C_t^2 [W(g_{t+1}) - W(g_t)],
 * with Lambda(g) = sum_{k >= g} d_k/Den_k, W(g) = sum_{k < g} d_k/Den_k^2,
 * C_t the running sum of x e over the column's nonzeros (rows increasing)
 * and g_t the tie group of row t.  The risk-set sums Den_k, Lambda and W
 * are rebuilt with a pass over all subjects only after a nonzero step, so a
 * coordinate whose step is zero costs O(nnz_j).  Its speed is reported
 * separately from the paper's method. */
#define SURV_FLAG_SPARSE_NUMERATOR 8
/* Cox fits of CSC data in the FP32 mode run speculative coordinate batches
 * by default: one row pass evaluates the derivatives of 4 consecutive
 * coordinates at the same e; their steps are taken in order up to and
 * including the first nonzero one (e is unchanged before it, so each step is
 * the one cyclic CCD takes, from the same sums) and the next pass starts
 * after it.  (Fits whose tie groups outnumber twice the warps of the grid
 * take one coordinate per pass.)  This flag turns the batches off: one
 * coordinate per row pass, as the paper's schedule. */
#define SURV_FLAG_ONE_COORDINATE 16
/* Speculative batches of 8 coordinates per row pass instead of 4 (for
 * comparison; 4 is the faster at the measured sizes). */
#define SURV_FLAG_SPEC_B8 32
/* Capture the per-coordinate and batch graphs without programmatic dependent
 * launch (each kernel starts after the previous one has finished), for
 * comparison with the default. */
#define SURV_FLAG_NO_PDL 64
/* cox_cv_path only, CSC data in the FP32 mode: run the batched row pass with
 * tile shape 1 (two 16-byte loads of e per lane a tile) or 2 (two rounds of
 * 32 nonzeros a load) instead of the tuned or default shape, for comparison
 * and testing (surv_cv_info.tile_form reports the shape that ran). */
#define SURV_FLAG_CV_TILE1 256
#define SURV_FLAG_CV_TILE2 512

/* Fill *opts with defaults: no penalty, FP32-compensated precision,
 * tol 1e-8, max_sweeps 1000, default stream, no workspace. */
void surv_opts_default(surv_opts *opts);

typedef struct surv_fit_info {
  int32_t sweeps;                /* full sweeps performed                         */
  int32_t converged;             /* 1 if the tolerance test passed                */
  int32_t nnz_beta;              /* nonzero coefficients at exit                  */
  int32_t device_error;          /* device error word (0 = none)                  */
  double loglik;                 /* log (pseudo-)likelihood at the returned beta  */
  double objective;              /* loglik + penalty at the returned beta         */
  double objective_prev;         /* the same after the previous sweep             */
  int64_t n_groups;              /* number of tie groups K                        */
  int64_t coordinate_passes;     /* risk-set passes run (sweeps * p + 1)          */
  int64_t eta_updates;           /* coordinates whose step was nonzero            */
  int64_t kernel_launches;       /* CUDA kernels launched by this call            */
  double ccd_kernel_ms;          /* device time of the CCD kernel (CUDA events on
                                    the call's stream)                            */
  double phase_ms[16];           /* diagnostics summed over the fit (CTA 0):
                                    [0] row pass, [1..3] exchange 1 (arrive,
                                    wait, after), [4] group-end transform,
                                    [5..7] exchange 2 (arrive, wait, Newton),
                                    [8] eta update; row-pass totals over CTAs:
                                    [9] max, [10] min, [11] mean; largest
                                    dense [12] and sparse [13] part of the
                                    pass; CTA 0 exchange-1 warp sums [14] and
                                    payload stores [15] (inside [1])        */
  int64_t row_passes;            /* passes over the subjects run: one per
                                    coordinate, fewer with speculative batches */
} surv_fit_info;

/* ---- entry points ------------------------------------------------------ */

/* Workspace that caches device buffers between calls on the same device.
 * surv_workspace_create: *ws receives a new handle (SURV_E_INVALID if ws is
 * NULL).  surv_workspace_destroy frees its device memory (NULL is a no-op). */
int surv_workspace_create(surv_workspace **ws);
int surv_workspace_destroy(surv_workspace *ws);

/* Stable order of decreasing time (Section 2.7 arranges subjects by
 * decreasing observed time; ties keep input order, so the result is unique).
 *   time [n] int32 (host or device), perm [n] int32 output (host or device):
 *   perm[r] = input index of the subject at rank r.
 * Device LSD radix sort; the stream is used for all work.  n = 0 is a no-op. */
int surv_sort_desc(const int32_t *time, int64_t n, int32_t *perm, void *stream);

/* Penalised Cox fit by CCD (Sections 2.1, 2.3, 2.4, 2.7).
 *   beta_inout [p] double (host or device): warm start on entry, estimate on
 *   return.  info (host, may be NULL) receives the fit summary.
 * Returns SURV_OK, SURV_W_NOT_CONVERGED or an error code. */
int cox_fit(const surv_data *data, const surv_opts *opts, double *beta_inout,
            surv_fit_info *info);

/* Penalised Fine-Gray fit by CCD (Sections 2.2-2.4, 2.7); status 2 marks the
 * competing event and the censoring weights use the Kaplan-Meier estimate of
 * the censoring distribution computed on the device.  Same contract as
 * cox_fit. */
int fg_fit(const surv_data *data, const surv_opts *opts, double *beta_inout,
           surv_fit_info *info);

/* One risk-set pass (Section 2.7, steps 1-4) at beta for coordinate j:
 *   *loglik = l(beta) (Eq. cox_l or fg_l), *grad = dl/dbeta_j,
 *   *hess = d2l/dbeta_j^2 (Eqs. cox_g/cox_h or fg_g/fg_h), unpenalised.
 *   model = SURV_COX or SURV_FG; beta [p] double host or device;
 *   loglik/grad/hess: host doubles (any may be NULL).  opts may be NULL
 *   (precision F32C, default stream, no workspace).  j in [0, p). */
int loglik_grad_hess(const surv_data *data, int32_t model, const double *beta,
                     int32_t j, double *loglik, double *grad, double *hess,
                     const surv_opts *opts);

/* Breslow tie-group table of data already in decreasing-time order
 * (Section 2.7; the Fine-Gray weights of Section 2.2).
 *   time [n] int32 non-increasing, status [n] int8 (host or device).
 *   *K receives the number of groups (maximal runs of equal time).  If the
 *   output arrays are non-NULL they must hold max_groups entries (host or
 *   device) and receive: gend[k] = position of the last subject of group k,
 *   dk[k] = subjects with status 1 in group k, Gk[k] = Kaplan-Meier estimate
 *   of the censoring survival G(t_k) = prod_{t_k' <= t_k} (1 - c_k'/n_k')
 *   with c = censored count and n = #{y >= t_k'}.
 *   Returns SURV_E_INVALID if K > max_groups and an output is requested;
 *   SURV_E_UNSORTED / SURV_E_STATUS on invalid input (status codes 0..2). */
int surv_groups(const int32_t *time, const int8_t *status, int64_t n, int64_t max_groups, int64_t *K,
                int32_t *gend, int32_t *dk, double *Gk, void *stream);

/* Allocation-free variant of loglik_grad_hess.  The paper has no counterpart;
 * this entry point is for callers that cannot allocate device memory while
 * they run, for example a host program whose device memory is entirely owned
 * by another allocator (a framework's caching pool, or a fixed budget taken
 * at start-up), or a latency-sensitive loop that cannot afford cudaMalloc and
 * cudaFree, which may synchronise the whole device.  It returns the same
 * (l, l', l'') as loglik_grad_hess for coordinate j and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Scratch: one fixed 16 MiB array in device memory, reserved by every GPU
 * that loads this library until the process exits.  A problem needs about
 * 12 bytes per subject (Cox, FP32; 16-24 for Fine-Gray or FP64), 52-76 bytes
 * per tie group and, for CSC, 19.5 KB per covariate; for example one million
 * subjects with 3650 distinct times and p = 100 fit.  A problem whose
 * subject or covariate count needs more is rejected with SURV_E_INVALID
 * before any work is queued; one whose tie groups need more is rejected
 * after the validation and tie-group count kernels, which write only into
 * the array.  p <= 4096.  col_ptr is copied to the host and checked
 * (col_ptr[0] = 0, non-decreasing: SURV_E_INDEX otherwise) before any
 * kernel reads row_idx through it.
 * The first call on a device looks up the array's device address and caches
 * it; make that first call before any stream capture.  All calls on a device
 * share the array, which keeps the last call's contents (the call zeroes
 * what must start at zero itself); calls that overlap on the GPU, from other
 * host threads or streams, race on it and must be serialised by the caller.
 *   data: time, status and X must be arrays on the current device (or
 *   managed memory; there is no staging buffer); X values in the dtype that `precision` uses (SURV_PREC_F32C:
 *   float32, SURV_PREC_F64: float64; CSC values may be NULL); dense X with a
 *   16-byte aligned base and n divisible by 4.  beta [p] host or device.
 *   loglik, grad, hess: host doubles (any may be NULL).  stream:
 *   cudaStream_t or NULL.  Errors as loglik_grad_hess, plus SURV_E_INVALID
 *   for the limits above. */
int loglik_grad_hess_noalloc(const surv_data *data, int32_t model, const double *beta, int32_t j,
                             double *loglik, double *grad, double *hess, int32_t precision, void *stream);

/* ---- differentiable form ------------------------------------------------
 * The Cox negative log partial likelihood (Breslow ties, Section 2.9 with
 * the risk-set sums of Section 2.7) of C linear predictors at once,
 * eta = X B:
 *   NLL_b = - sum_i delta_i eta_ib + sum_k d_k log sum_{r <= e_k} exp(eta_rb),
 * delta_i = (status_i == 1), subjects in non-increasing time, and its
 * gradient dNLL/dB = X^T (exp(eta) * Lambda - delta), Lambda_b(i) the sum of
 * d_k / den_kb over the tie groups whose risk set holds i.
 *
 * X is bfloat16, row-major n x p; B float32 row-major p x C.  X B and
 * X^T G run on the tensor cores in the library's own kernels (TMA tile
 * loads, tcgen05.mma, bf16 inputs, FP32 accumulation in tensor memory) with
 * B and G split into a bf16 high and low part, so eta carries about 16
 * significant bits of B; the partial sums of X^T G over row ranges are added
 * in FP64; the risk-set scans use FP32 values with float-float running sums
 * and the logs are FP64.  All arrays are device memory; C <= 64; B is held
 * in shared memory during X B, which bounds p (p <= 512 for C = 64, about
 * 1500 for C <= 16; SURV_E_INVALID beyond). */
typedef struct surv_nll_data {
  int64_t n;                     /* subjects                                       */
  int32_t p;                     /* covariates (columns of X)                      */
  int32_t ncols;                 /* C: linear predictors (columns of B), 1..64     */
  const int32_t *time;           /* [n] non-increasing                              */
  const int8_t *status;          /* [n] 0 censored, 1 event (2 counts as censored)   */
  const void *X;                 /* [n][p] bfloat16, row-major                       */
} surv_nll_data;

/* nll[C] (device doubles) at B [p][C] (device floats).  Keeps eta and the
 * risk-set sums in the workspace `ws` (required) for cox_nll_backward.
 * Errors: SURV_E_INVALID (null, sizes, host pointers), SURV_E_UNSORTED,
 * SURV_E_STATUS, SURV_E_NOMEM, SURV_E_CUDA; SURV_E_DEVICE_TIMEOUT when a
 * bounded wait inside the tensor-core kernels of an earlier forward or
 * backward call on this workspace expired (those results were invalid; the
 * calls do not synchronise, so the next forward reports it). */
int cox_nll_forward(const surv_nll_data *data, const float *B, double *nll, void *stream, surv_workspace *ws);

/* grad_B [p][C] (device floats) = sum_b grad_nll[b] dNLL_b/dB at the B of
 * the last cox_nll_forward on the same workspace and data (SURV_E_INVALID
 * otherwise).  grad_nll [C] device doubles (the incoming gradient). */
int cox_nll_backward(const surv_nll_data *data, const double *grad_nll, float *grad_B, void *stream,
                     surv_workspace *ws);

/* ---- cross-validated penalty path (Section 2.8) ------------------------ */

/* Largest useful L1 strength for Cox: the smallest gamma whose penalised
 * optimum is beta = 0, i.e. max over penalised j of |l'_j(0)| / pf_j (the
 * Karush-Kuhn-Tucker condition of Section 2.3 at 0).  At beta = 0 every e_i
 * is 1, so l'_j(0) = sum_i x_ij (delta_i - Lambda(i)) with Lambda(i) the sum
 * of d_k / |R_k| over the tie groups whose risk set holds i; the sums run in
 * FP64 on the device.
 *   data: as for cox_fit (either layout and dtype).  penalty_factor [p]
 *   (host or device) or NULL for all ones.  *lambda_max: host double.
 *   stream: cudaStream_t or NULL.  Errors as cox_fit. */
int cox_lambda_max(const surv_data *data, const double *penalty_factor, double *lambda_max, void *stream);

typedef struct surv_cv_info {
  int32_t nfits;                 /* nlambda * nfolds                                 */
  int32_t best_lambda;           /* index of the largest mean held-out score         */
  int32_t max_sweeps_used;       /* most sweeps of any fit                           */
  int32_t fits_converged;        /* fits that met the tolerance                      */
  int32_t graph_replays;         /* replays of the batched sweep graph               */
  int32_t ctas_per_fit;          /* CTAs each fit runs on in the batched kernels     */
  int32_t row_pass_form;         /* CSC row pass: 1 one warp reduction per group end, */
                                 /* 2 lane scans per tile (many ends per warp);      */
                                 /* 0 for dense X                                    */
  int32_t tile_form;             /* CSC FP32 row pass: 0 four 16-byte loads of e per */
                                 /* lane a tile and 4 rounds of 32 nonzeros a load,  */
                                 /* 1 two loads, 2 two rounds                        */
  int64_t kernel_launches;       /* CUDA kernels launched (graph nodes counted)      */
  int64_t n_groups;              /* tie groups K of the whole data                   */
  int64_t coordinate_passes;     /* risk-set passes summed over fits                 */
  int64_t eta_updates;           /* nonzero steps summed over fits                   */
  double ccd_kernel_ms;          /* batched CCD: first replay to the last stop       */
  double heldout_ms;             /* held-out scores and the choice of lambda         */
} surv_cv_info;

/* K-fold cross-validation over a penalty path for Cox (Section 2.8): one
 * penalised fit per (lambda, fold) pair, F = nlambda * nfolds fits in all,
 * each on the subjects outside its fold, all run together: every kernel of
 * the per-coordinate schedule carries every fit (one fit per grid row), the
 * sweep is captured once as a CUDA graph and replayed until every fit has
 * stopped by its own rule.  A held-out subject keeps e = 0 in its fit, so
 * it is in no risk set, and each fold has its own event counts d_k and
 * delta^T X_j; X and the tie groups are shared.  Every fit starts from
 * beta = 0 (cold start).
 *
 * Afterwards each fit's held-out score is the log partial likelihood of the
 * subjects of its fold alone, on their own risk sets, at the fit's beta
 * (Breslow ties as in Eq. cox_l); the path's score at lambda l is the mean
 * over folds, and best_lambda is the first index with the largest score.
 *   data: as for cox_fit.  fold_id [n] int8 (host or device), the fold
 *   0..nfolds-1 of each subject in data order; every fold's training part
 *   needs an event (SURV_E_NO_EVENTS otherwise).  lambdas [nlambda] host
 *   doubles >= 0.  opts: penalty (L1 or L2), precision, tol, max_sweeps,
 *   penalty_factor, stream and workspace as for cox_fit (lambda is
 *   ignored; flags may hold SURV_FLAG_CV_TUNE).  ctas_per_fit: CTAs per fit
 *   in the batched kernels, or 0 for the value tuned earlier on this
 *   workspace for the same shape, else a default from the device's SM
 *   count and the number of fits.
 * Outputs (host or device, any may be NULL except beta_out):
 *   beta_out [nlambda][nfolds][p] doubles (fit f = l * nfolds + k),
 *   heldout [nlambda][nfolds], cv_mean [nlambda] doubles,
 *   sweeps [nlambda][nfolds] int32, info (host).
 * Returns SURV_OK when every fit converged, SURV_W_NOT_CONVERGED when some
 * stopped at max_sweeps (all outputs are written), or an error code.
 * 1 <= nfolds <= 127, 1 <= nlambda, F <= 65535. */
int cox_cv_path(const surv_data *data, const int8_t *fold_id, int32_t nfolds, const double *lambdas,
                int32_t nlambda, const surv_opts *opts, int32_t ctas_per_fit, double *beta_out,
                double *heldout, double *cv_mean, int32_t *sweeps, surv_cv_info *info);

/* Short name of a return code (static string). */
const char *surv_strerror(int code);

/* Details of the last error on the calling thread (static per thread). */
const char *surv_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int surv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SURVGPU_H */
