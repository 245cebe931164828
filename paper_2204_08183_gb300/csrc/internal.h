// Internal declarations shared by the survgpu translation units (not part of
// the public C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace survgpu {

constexpr int kMaxWarpsPerCta = 32;            // persistent CCD kernel: up to 1024 threads
constexpr int kSlotWords = 32;                 // one 128-byte exchange slot per CTA

// Prep error bits (host maps them to SURV_E_* codes).
enum : unsigned {
  PREP_UNSORTED = 1u,
  PREP_STATUS = 2u,
  PREP_NONFINITE = 4u,
  PREP_INDEX = 8u,
  PREP_FOLD = 16u,
  PREP_VALUES_NOT_ONE = 32u,  // not an error: some CSC value differs from 1
};

// Parameters of the persistent CCD kernel (passed as a __grid_constant__).
struct CcdParams {
  int64_t n;          // subjects
  int64_t ld;         // leading dimension of dense X (>= n, multiple of 4)
  int32_t p;          // covariates
  int32_t K;          // tie groups
  int32_t G;          // CTAs (co-resident)
  int32_t wpc;        // warps per CTA (blockDim.x = 32 * wpc)
  int32_t wpw;        // 32-row words per warp
  int32_t nwarps;     // G * wpc

  const int32_t* gend;   // [K] group end positions
  const int32_t* dk;     // [K] events per group (Cox) / primary events (FG)
  const double* Gk;      // [K] Kaplan-Meier censoring survival at t_k (FG)
  const float2* Gkff;    // [K] the same as float-float (hi, lo)
  const int32_t* wk0;    // [nwarps+1] first group index whose end is in warp w

  const int64_t* col_ptr;  // CSC
  const int32_t* row_idx;
  const void* values;      // CSC values (T) or null for indicators
  const int32_t* woff;     // [p][nwarps+1] entry offset of warp boundaries
  const void* X;           // dense column-major (T), leading dimension ld

  void* e;               // [n] exp(eta) (T)
  void* eta;             // [n] eta: float2 (float-float) or double
  const void* w2;        // [n] I(status=2)/G(y_i) (T), FG only
  const double* dTx;     // [p] delta^T X_j
  double* beta;          // [p] coefficients (written by CTA 0)
  double* width;         // [p] trust-region half-widths (written by CTA 0)
  const double* pen;     // [p] lambda * penalty_factor_j
  void* rec;             // [K][M] accumulators: prefix at group ends, warp-relative

  unsigned* slot_agg;    // [2][G][kSlotWords] CTA aggregates, by epoch parity
  unsigned* slot_part;   // [2][G][kSlotWords] CTA partial sums, by epoch parity
  unsigned* counters;    // [2] arrival counters of the two exchanges (zeroed per launch)
  unsigned* err;         // device error word
  double* out;           // results, see OutIndex
  unsigned long long* timing;  // [8] phase times (ns): see PhaseIndex

  int32_t penalty;
  int32_t max_sweeps;
  double tol;
  int32_t single_j;      // >= 0: evaluate coordinate single_j once and stop
  int32_t withhold_cta;  // test knob: this CTA never publishes (-1 = off)
  int32_t no_pdl;        // graph schedules: capture without programmatic dependent launch
  int32_t pass_form;     // Cox CSC row pass: 0 by the ends per warp, 1 one reduction per end,
                         //   2 the many-ends form (lane scans per tile)
  int32_t tile_form;     // batched Cox CSC FP32 row pass: 0 four 16-byte loads of e per lane a
                         //   tile and 4 rounds of nonzeros a load, 1 two loads, 2 two rounds
  uint64_t timeout_ns;   // bound on every grid-exchange wait

  // per-coordinate kernel pair only (null for the persistent kernel)
  uint64_t* wt;          // [M][nwarps] warp totals of the last pass (8-byte payload words)
  uint64_t* agg;         // [kRep][M][G] CTA aggregates of the last pass, replicated
  struct GraphCtl* gctl; // fit state carried between kernels
  unsigned* done_count;  // fits that have stopped (the host polls it)

  // Batched fits (cross-validation path): fit f = blockIdx.y of every kernel
  // takes its parameters from fits[f], a complete copy of this struct whose
  // pointers lead to the fit's own e, eta, beta, width, pen, outputs,
  // records and control lines, and to its fold's event counts dk and
  // delta^T X.  Subjects of the fit's fold are held out: their e stays 0.
  // nfit = 0 and fits = null for one fit.
  int32_t nfit;
  int32_t fold;               // the fit's held-out fold (fold_id null: unused)
  const int8_t* fold_id;      // [n] fold of each subject, or null
  const struct CcdParams* fits;  // [nfit] per-fit parameters (device memory)
};

// Fit state of the per-coordinate kernel pair.  The last transform CTA of
// each coordinate j (found with an atomic ticket) owns the scalar state: it
// takes the Newton step, stores beta_j and its width, decides convergence on
// j = 0, and publishes in kRep identical 128-byte lines everything the next
// two kernels need (the step, and the scalars of coordinate j + 1).  CTA c of
// a kernel reads line c % kRep once, so no line has more than a handful of
// readers.
constexpr int kRep = 32;
struct alignas(128) CtlLine {
  int32_t stop;          // the fit has stopped: every later kernel returns
  int32_t nevals;        // objective evaluations so far (one per sweep)
  double applied;        // step applied to the coordinate just finished
  float delta_hi;        // the same step as float-float
  float delta_lo;
  double beta;           // beta, trust-region width, lambda * penalty factor
  double width;          //   and delta^T X of the next coordinate
  double pen;
  double dtx;
  double f_prev;         // objective at the latest evaluation
  long long passes;      // coordinate passes so far
  long long eta_updates; // nonzero steps so far
  int32_t dirty;         // the stored risk-set sums of e are stale (set at the start of a fit; sparse-
                         //   numerator form and speculative batches)
  int32_t j0;            // speculative batches: first coordinate of the next batch
  int32_t q;             //   and the coordinate whose step is still to be applied (-1: none)
  long long batches;     //   and the row passes so far
  char pad[128 - 112];
};
struct GraphCtl {
  CtlLine line[kRep];
  int32_t done;          // host-visible copy of stop
  uint32_t ticket;       // transform CTAs finished in the current kernel
};

// Phase times accumulated by thread 0 of CTA 0 (ns), plus statistics of the
// per-CTA total pass time.
enum PhaseIndex : int {
  PH_PASS = 0,        // warp pass (step 2) of CTA 0
  PH_EX1_PRE = 1,     // CTA combine, payload, arrival at exchange #1
  PH_EX1_WAIT = 2,    // waiting for the other CTAs (exchange #1)
  PH_EX1_POST = 3,    // prefix / totals after exchange #1
  PH_TRANSFORM = 4,   // group-end transform and CTA reduction (steps 3-4)
  PH_EX2_PRE = 5,     // payload and arrival at exchange #2
  PH_EX2_WAIT = 6,    // waiting for the other CTAs (exchange #2)
  PH_EX2_POST = 7,    // final sums and the Newton step
  PH_UPDATE = 8,      // eta / e update
  PH_PASS_MAX = 9,    // largest total pass time of any CTA
  PH_PASS_MIN = 10,   // smallest total pass time of any CTA
  PH_PASS_SUM = 11,   // sum over CTAs of the total pass time
  PH_DENSE_MAX = 12,  // largest total time of the dense part of the pass (any CTA)
  PH_SPARSE_MAX = 13, // largest total time of the sparse part (any CTA)
  PH_EX1_SUMS = 14,   // CTA 0: warp sums before the exchange #1 payload
  PH_EX1_STORE = 15,  // CTA 0: payload stores before the arrival
  PH_COUNT = 16,
};

enum OutIndex : int {
  OUT_LOGLIK = 0,
  OUT_OBJECTIVE = 1,
  OUT_OBJECTIVE_PREV = 2,
  OUT_SWEEPS = 3,
  OUT_CONVERGED = 4,
  OUT_ETA_UPDATES = 5,
  OUT_GRAD = 6,
  OUT_HESS = 7,
  OUT_PASSES = 8,
  OUT_EPOCH_END = 9,
  OUT_BATCHES = 10,     // row passes of the speculative-batch schedule
  OUT_COUNT = 16,
};

// Launch the persistent CCD kernel (cooperative launch).  model 0 Cox / 1 FG,
// layout 0 CSC / 1 dense, prec 0 float-float / 1 double.
cudaError_t launch_ccd(int model, int layout, int prec, const CcdParams& P, cudaStream_t s);
// Co-resident CTAs and warps per CTA of the CCD kernel for this configuration.
cudaError_t ccd_grid_size(int model, int layout, int prec, int* G, int* wpc);

// Per-coordinate schedule (ccd_graph.cu): grid of the pass / transform
// kernels, and a fit that replays one captured sweep (2p kernels) until the
// device reports that the fit has stopped.  P.gctl and P.wt must be set and
// *P.gctl zeroed; at most max_sweeps + 2 sweeps are replayed.
// The instantiated sweep graph is kept in a GraphCache (one per workspace)
// and reused while the parameters are byte-identical; t0 (optional) is
// recorded on s right before the first replay.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  CcdParams key;
  unsigned char key2[256] = {};  // further launch parameters (sparse-numerator form)
  int mlp = -1;
  cudaStream_t cs = nullptr;     // capture stream
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int* flag = nullptr;           // pinned [2]: stop flag of the last two replays
};
cudaError_t graph_grid_size(int model, int layout, int prec, int* G, int* wpc);
// Fill the control lines for the first coordinate of a fit (P.gctl zeroed).
cudaError_t graph_init(const CcdParams& P, cudaStream_t s);
cudaError_t run_ccd_graph(int model, int layout, int prec, const CcdParams& P, cudaStream_t s, GraphCache* gc,
                          cudaEvent_t t0, int* replays, int* launches);
void graph_cache_free(GraphCache* gc);
// Stream, events and pinned flags of a graph cache (idempotent).
cudaError_t graph_cache_prepare(GraphCache* gc);
// Replay gc->exec on s until the device reports the fit(s) stopped (at most
// P.max_sweeps + 2 replays); t0 (optional) is recorded before the first.
cudaError_t replay_until_stop(const CcdParams& P, cudaStream_t s, GraphCache* gc, cudaEvent_t t0,
                              int launches_per_replay, int* replays, int* launches, int max_replays = 0);

// ---- speculative coordinate batches (spec.cu) ----------------------------
// Cox, CSC, FP32 mode: each row pass evaluates the derivatives of B
// consecutive coordinates at the same e; the steps are taken in order up to
// the first nonzero one (e is unchanged before it, so every committed step
// is the one cyclic CCD takes).  graph_init(P) first.
cudaError_t run_spec_graph(const CcdParams& P, int B, cudaStream_t s, GraphCache* gc, cudaEvent_t t0, int* replays,
                           int* launches);
// Batches per graph replay.
int spec_slots(int p, int B);

// ---- sparse-numerator form (sn.cu; not in the paper) --------------------
// Cox, CSC, FP32 mode.  Per coordinate, after a nonzero step only, the risk
// sets are rebuilt (Den_k, Lambda, W); every coordinate's derivatives then
// come from its nonzeros alone (O(nnz_j)).
struct SnParams {
  const int32_t* grp;    // [n] tie group of each subject
  double* den;           // [K] Den_k
  double* v1;            // [K] d_k / Den_k
  double* v2;            // [K] d_k / Den_k^2
  float2* lam;           // [K] Lambda(k) = sum_{k' >= k} d_k' / Den_k' (float-float)
  float2* W;             // [K + 1] W(k) = sum_{k' < k} d_k' / Den_k'^2 (float-float)
  double* part_den;      // [3][G] per-CTA sums of v1, v2 and d_k log Den_k
  double* ll_den;        // [1] sum_k d_k log Den_k at the current e
  uint64_t* part_col;    // [4][G2] per-CTA chunk totals of a = x e, S1, S2 and Q
  int32_t G2;            // CTAs of the column kernels
  int32_t multi;         // row pass for many group ends per warp
};
// Group of each subject from the group ends (prep).
cudaError_t sn_groups(const int32_t* gend, int32_t K, int64_t n, int32_t* grp, cudaStream_t s);
// Fit with the sparse-numerator kernels: graph_init(P) first, then replays
// as run_ccd_graph.
cudaError_t run_sn_graph(const CcdParams& P, const SnParams& S, cudaStream_t s, GraphCache* gc, cudaEvent_t t0,
                         int* replays, int* launches);
// One replay of the sweep graph of P (captured and destroyed here), timed
// with events on s: *ms.  P's state must be initialised (graph_init).
cudaError_t time_one_sweep(int model, int layout, int prec, const CcdParams& P, cudaStream_t s, float* ms);

// ---- prep kernels (prep.cu) --------------------------------------------
cudaError_t prep_check_times(const int32_t* time, const int8_t* status, int64_t n, int model,
                             unsigned* perr, cudaStream_t s);
cudaError_t prep_check_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* values, int prec,
                           int64_t p, int64_t n, unsigned* perr, cudaStream_t s);
cudaError_t prep_check_dense(const void* X, int prec, int64_t ld, int64_t n, int64_t p, unsigned* perr,
                             cudaStream_t s);
cudaError_t prep_check_finite_f64(const double* v, int64_t count, unsigned* perr, cudaStream_t s);
// Count tie groups: writes per-block counts into blockcnt [nblocks] and K into *K_dev.
int64_t prep_end_blocks(int64_t n);
cudaError_t prep_count_ends(const int32_t* time, int64_t n, int32_t* blockcnt, int32_t* K_dev, cudaStream_t s);
cudaError_t prep_write_ends(const int32_t* time, int64_t n, const int32_t* blockoff, int32_t* gend, cudaStream_t s);
// dk, ck [K] (zeroed here): events and censored subjects per group, n subjects;
// *total_events (zeroed by the caller) += all events
cudaError_t prep_group_stats(const int32_t* gend, int32_t K, const int8_t* status, int64_t n, int32_t* dk,
                             int32_t* ck, int32_t* total_events, cudaStream_t s);
cudaError_t prep_km(const int32_t* gend, const int32_t* ck, int32_t K, double* Gk, float2* Gkff, cudaStream_t s);
cudaError_t prep_w2(const int32_t* gend, int32_t K, const int8_t* status, const double* Gk, void* w2, int prec,
                    cudaStream_t s);
cudaError_t prep_dtx_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* values, int prec,
                         const int8_t* status, int64_t p, double* dTx, cudaStream_t s);
cudaError_t prep_dtx_dense(const void* X, int prec, int64_t ld, int64_t n, const int8_t* status, int64_t p,
                           double* dTx, cudaStream_t s);
cudaError_t prep_warp_groups(const int32_t* gend, int32_t K, int64_t n, int32_t nwarps, int64_t rows_per_warp,
                             int32_t* wk0, cudaStream_t s);
cudaError_t prep_warp_offsets(const int64_t* col_ptr, const int32_t* row_idx, int64_t p, int64_t n,
                              int32_t nwarps, int64_t rows_per_warp, int32_t* woff, cudaStream_t s);
cudaError_t prep_eta_dense(const void* X, int prec, int64_t ld, int64_t n, int64_t p, const double* beta,
                           void* eta, void* e, cudaStream_t s);
cudaError_t prep_eta_zero(int prec, int64_t n, void* eta, void* e, cudaStream_t s);
cudaError_t prep_eta_axpy_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* values, int prec,
                              int64_t j, int64_t nnz_j, double delta, void* eta, cudaStream_t s);
cudaError_t prep_eta_exp(int prec, int64_t n, const void* eta, void* e, cudaStream_t s);
cudaError_t prep_fill_f64(double* v, double value, int64_t count, cudaStream_t s);
// Convert / pad a dense matrix into the working precision with leading
// dimension ld (src column-major, leading dimension n).
cudaError_t prep_convert_dense(const void* src, int src_dtype, int64_t n, int64_t p, void* dst, int prec,
                               int64_t ld, cudaStream_t s);
cudaError_t prep_convert_vec(const void* src, int src_dtype, int64_t count, void* dst, int prec, cudaStream_t s);

// ---- cross-validated path and lambda_max (cv.cu) -------------------------
// fold ids outside [0, nfolds) set PREP_FOLD in *perr
cudaError_t cv_check_folds(const int8_t* fold_id, int64_t n, int nfolds, unsigned* perr, cudaStream_t s);
// dk [nfolds][K]: events of each group outside each fold; events [nfolds] (zeroed by the caller) += their totals
cudaError_t cv_fold_stats(const int32_t* gend, int32_t K, const int8_t* status, const int8_t* fold_id, int nfolds,
                          int32_t* dk, int32_t* events, cudaStream_t s);
// dTx [nfolds][p]: delta^T X_j over the subjects outside each fold (layout 0 CSC, 1 dense)
cudaError_t cv_dtx(int layout, int prec, const int64_t* col_ptr, const int32_t* row_idx, const void* values,
                   int64_t ld, int64_t n, int64_t p, const int8_t* status, const int8_t* fold_id, int nfolds,
                   double* dTx, cudaStream_t s);
// e [nfit][fit_n] = 1 outside the fit's fold (f % nfolds), 0 inside; eta = 0
// (rows 0..n-1 of each fit; fit_n >= n is the per-fit stride)
cudaError_t cv_init(int prec, int64_t n, int64_t fit_n, const int8_t* fold_id, int nfolds, int nfit, void* e,
                    void* eta, cudaStream_t s);
// heldout [nfit]: log partial likelihood of each fit's fold on its own risk
// sets at eta [nfit][fit_n]; den [nfit][K] scratch
cudaError_t cv_heldout(int prec, int64_t n, int64_t fit_n, const int32_t* time, const int8_t* status, const int8_t* fold_id,
                       int nfolds, int nfit, const void* eta, const int32_t* dk_all, const int32_t* dk_fold,
                       int32_t K, double* den, double* heldout, cudaStream_t s);
// cv_mean [nlambda] and *best (device)
cudaError_t cv_select(const double* heldout, int nlambda, int nfolds, double* cv_mean, int32_t* best,
                      cudaStream_t s);
// *out (device) = max_j |l'_j(0)| / pf_j for Cox; lam [K], r [n], g [p] scratch
cudaError_t lambda_max_device(int layout, int prec, const int64_t* col_ptr, const int32_t* row_idx,
                              const void* values, int64_t ld, int64_t n, int64_t p, const int8_t* status,
                              const int32_t* gend, const int32_t* dk, int32_t K, const double* pf, double* lam,
                              double* r, double* g, double* out, cudaStream_t s);

// Text returned by surv_last_error() on the calling thread (api.cu).
void set_last_error_text(const char* msg);

// ---- sort (sort.cu) -----------------------------------------------------
// Workspace bytes needed by radix_sort_desc for n elements.
size_t radix_sort_workspace(int64_t n);
cudaError_t radix_sort_desc(const int32_t* time, int64_t n, int32_t* perm, void* work, cudaStream_t s,
                            int* launches);

}  // namespace survgpu
