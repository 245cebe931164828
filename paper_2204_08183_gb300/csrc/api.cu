// C ABI of libsurvgpu.so (declared in include/survgpu.h): argument checks,
// staging of host buffers, workspace management and the launch sequence:
// prep kernels, then the CCD schedule (speculative coordinate batches for
// Cox fits of CSC data in FP32, one coordinate per pass otherwise, both as
// CUDA-graph replays; the persistent kernel on request and for single
// evaluations).  No arithmetic of the method runs on the host; the host
// reads back only sizes, error words and results.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "survgpu.h"

#include "workspace.h"

namespace {

using survgpu::CcdParams;

thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

struct DevCtrl {
  unsigned perr;
  unsigned err;
  int32_t K;
  int32_t total_events;
  unsigned counters[2];
  unsigned pad[2];
  double out[survgpu::OUT_COUNT];
  unsigned long long timing[survgpu::PH_COUNT];
  survgpu::GraphCtl gctl;
};

// Allocation failures map to SURV_E_NOMEM, anything else to SURV_E_CUDA.
int cuda_code(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SURV_E_NOMEM : SURV_E_CUDA; }

#define CUDA_TRY(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return cuda_code(e_);                                                     \
    }                                                                           \
  } while (0)

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

int survgpu::ws_ensure(surv_workspace* ws, int id, size_t bytes, void** out) {
  auto& b = ws->bufs[id];
  if (bytes == 0) bytes = 256;
  if (b.cap < bytes) {
    if (b.p) {
      cudaError_t e = cudaFree(b.p);
      b.p = nullptr;
      b.cap = 0;
      if (e != cudaSuccess) {
        set_error("cudaFree: %s", cudaGetErrorString(e));
        return SURV_E_CUDA;
      }
    }
    cudaError_t e = cudaMalloc(&b.p, align256(bytes));
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
      return SURV_E_NOMEM;
    }
    b.cap = align256(bytes);
  }
  *out = b.p;
  return SURV_OK;
}

namespace {

int ensure(surv_workspace* ws, int id, size_t bytes, void** out) { return survgpu::ws_ensure(ws, id, bytes, out); }

void free_all(surv_workspace* ws) {
  survgpu::graph_cache_free(&ws->graph);
  for (auto& b : ws->bufs) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
}

// Memory the kernels may read in place: device memory of the current device
// or managed memory.  Host memory and memory of another GPU are not.
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.device == cur;
}

// Device view of a caller array: the pointer itself if the kernels may read
// it in place, else a workspace copy made on `s` (from host memory or from
// another GPU).
int device_view(surv_workspace* ws, int id, const void* src, size_t bytes, cudaStream_t s, const void** out) {
  if (is_device_ptr(src) || bytes == 0) {
    *out = src;
    return SURV_OK;
  }
  void* d = nullptr;
  int rc = ensure(ws, id, bytes, &d);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(d, src, bytes, cudaMemcpyDefault, s));
  *out = d;
  return SURV_OK;
}

// Copy a caller array (host or device) into host memory.
int to_host(const void* src, size_t bytes, void* dst, cudaStream_t s) {
  if (bytes == 0) return SURV_OK;
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return SURV_OK;
}

struct WsGuard {
  surv_workspace* ws = nullptr;
  bool owned = false;
  ~WsGuard() {
    if (owned && ws) {
      free_all(ws);
      delete ws;
    }
  }
};

int map_prep_error(unsigned perr) {
  if (perr & survgpu::PREP_INDEX) { set_error("CSC row indices out of range or not increasing"); return SURV_E_INDEX; }
  if (perr & survgpu::PREP_UNSORTED) { set_error("time is not non-increasing"); return SURV_E_UNSORTED; }
  if (perr & survgpu::PREP_STATUS) { set_error("status code out of range"); return SURV_E_STATUS; }
  if (perr & survgpu::PREP_NONFINITE) { set_error("non-finite value in X, beta or penalty factors"); return SURV_E_NONFINITE; }
  return SURV_OK;
}

// Sizes, enums and pointers of a surv_data (SURV_OK or SURV_E_INVALID / NO_EVENTS).
int check_data(const surv_data* d) {
  if (!d) { set_error("null data"); return SURV_E_INVALID; }
  const int64_t n = d->n, p = d->p;
  if (n < 0 || p < 1 || n > 0x7fffffff || p > 0x7fffffff) { set_error("bad sizes n=%lld p=%lld", (long long)n, (long long)p); return SURV_E_INVALID; }
  if (d->layout != SURV_CSC && d->layout != SURV_DENSE) { set_error("bad layout"); return SURV_E_INVALID; }
  if (d->dtype != SURV_F32 && d->dtype != SURV_F64 && !(d->dtype == SURV_BF16 && d->layout == SURV_DENSE)) {
    set_error("bad dtype (bfloat16 is for dense X only)");
    return SURV_E_INVALID;
  }
  if (n == 0) { set_error("no subjects"); return SURV_E_NO_EVENTS; }
  if (!d->time || !d->status) { set_error("null time/status"); return SURV_E_INVALID; }
  if (d->layout == SURV_CSC && (!d->col_ptr || !d->row_idx)) { set_error("null CSC arrays"); return SURV_E_INVALID; }
  if (d->layout == SURV_DENSE && !d->values) { set_error("null dense values"); return SURV_E_INVALID; }
  return SURV_OK;
}

// Device views of the data in the working precision prec (0 float, 1 double):
// caller arrays used in place when they are device memory, else copied; X
// converted (and dense X padded to a leading dimension that is a multiple
// of 4) when its dtype or alignment differs.
struct Staged {
  const int32_t* time = nullptr;
  const int8_t* status = nullptr;
  const int64_t* colptr = nullptr;
  const int32_t* rowidx = nullptr;
  const void* vals = nullptr;  // CSC values (null: indicators) or dense X
  int64_t ld = 0;
  int64_t nnz = 0;
  std::vector<int64_t> colptr_h;
};

int stage_data(const surv_data* d, int prec, surv_workspace* ws, cudaStream_t s, Staged* st, int64_t* launches) {
  using W = surv_workspace;
  const int64_t n = d->n, p = d->p;
  const size_t tsz = prec == 0 ? 4 : 8;
  int rc;
  const void *time_d = nullptr, *status_d = nullptr, *colptr_d = nullptr, *rowidx_d = nullptr, *vals_d = nullptr;
  if ((rc = device_view(ws, W::TIME, d->time, 4 * (size_t)n, s, &time_d))) return rc;
  if ((rc = device_view(ws, W::STATUS, d->status, (size_t)n, s, &status_d))) return rc;
  if (d->layout == SURV_CSC) {
    st->colptr_h.resize(p + 1);
    if ((rc = to_host(d->col_ptr, 8 * (size_t)(p + 1), st->colptr_h.data(), s))) return rc;
    if (st->colptr_h[0] != 0) { set_error("col_ptr[0] != 0"); return SURV_E_INDEX; }
    for (int64_t j = 0; j < p; ++j)
      if (st->colptr_h[j + 1] < st->colptr_h[j]) { set_error("col_ptr decreases at %lld", (long long)j); return SURV_E_INDEX; }
    st->nnz = st->colptr_h[p];
    if ((rc = device_view(ws, W::COLPTR, d->col_ptr, 8 * (size_t)(p + 1), s, &colptr_d))) return rc;
    if ((rc = device_view(ws, W::ROWIDX, d->row_idx, 4 * (size_t)st->nnz, s, &rowidx_d))) return rc;
    if (d->values) {
      const size_t vsz = d->dtype == SURV_F32 ? 4 : 8;
      if ((rc = device_view(ws, W::VALUES, d->values, vsz * (size_t)st->nnz, s, &vals_d))) return rc;
      if (d->dtype != prec) {
        void* conv = nullptr;
        if ((rc = ensure(ws, W::XD, tsz * (size_t)st->nnz, &conv))) return rc;
        CUDA_TRY(survgpu::prep_convert_vec(vals_d, d->dtype, st->nnz, conv, prec, s));
        ++*launches;
        vals_d = conv;
      }
    }
  }
  st->ld = n;
  if (d->layout == SURV_DENSE) {
    const size_t vsz = d->dtype == SURV_F32 ? 4 : (d->dtype == SURV_F64 ? 8 : 2);
    if ((rc = device_view(ws, W::VALUES, d->values, vsz * (size_t)n * (size_t)p, s, &vals_d))) return rc;
    const bool aligned = ((uintptr_t)vals_d % 16) == 0 && (n % 4) == 0;
    if (d->dtype != prec || !aligned) {
      st->ld = (n + 3) / 4 * 4;
      void* conv = nullptr;
      if ((rc = ensure(ws, W::XD, tsz * (size_t)st->ld * (size_t)p, &conv))) return rc;
      CUDA_TRY(survgpu::prep_convert_dense(vals_d, d->dtype, n, p, conv, prec, st->ld, s));
      ++*launches;
      vals_d = conv;
    }
  }
  st->time = static_cast<const int32_t*>(time_d);
  st->status = static_cast<const int8_t*>(status_d);
  st->colptr = static_cast<const int64_t*>(colptr_d);
  st->rowidx = static_cast<const int32_t*>(rowidx_d);
  st->vals = vals_d;
  return SURV_OK;
}

// Validation kernels on the staged data and the tie-group count: *K after a
// synchronisation (ctrl zeroed here; prep errors mapped to return codes).
// CSC values that are all exactly 1 are dropped from st (the kernels then
// take every nonzero as 1, an indicator matrix): the arithmetic is the same
// bit for bit (x e = e, x^2 = x, delta x = delta) and the values are not read
// again.
int validate_and_count(int model, int layout, int prec, int64_t n, int64_t p, Staged& st, DevCtrl* ctrl,
                       surv_workspace* ws, cudaStream_t s, void** blockcnt, int32_t* K, int64_t* launches) {
  CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(DevCtrl), s));
  CUDA_TRY(survgpu::prep_check_times(st.time, st.status, n, model, &ctrl->perr, s));
  ++*launches;
  if (layout == SURV_CSC)
    CUDA_TRY(survgpu::prep_check_csc(st.colptr, st.rowidx, st.vals, prec, p, n, &ctrl->perr, s));
  else
    CUDA_TRY(survgpu::prep_check_dense(st.vals, prec, st.ld, n, p, &ctrl->perr, s));
  ++*launches;
  const int64_t nb = survgpu::prep_end_blocks(n);
  int rc;
  if ((rc = ensure(ws, surv_workspace::BLOCKCNT, 4 * (size_t)nb, blockcnt))) return rc;
  CUDA_TRY(survgpu::prep_count_ends(st.time, n, static_cast<int32_t*>(*blockcnt), &ctrl->K, s));
  *launches += 2;
  DevCtrl hc;
  CUDA_TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if ((rc = map_prep_error(hc.perr))) return rc;
  *K = hc.K;
  if (layout == SURV_CSC && st.vals && !(hc.perr & survgpu::PREP_VALUES_NOT_ONE)) st.vals = nullptr;
  return SURV_OK;
}

int fit_common(int model, const surv_data* d, const surv_opts* o_in, double* beta_inout, surv_fit_info* info,
               int single_j, double* out_l, double* out_g, double* out_h) {
  g_last_error[0] = '\0';
  surv_opts o;
  if (o_in) o = *o_in; else surv_opts_default(&o);
  if (!d || !beta_inout) { set_error("null data or beta"); return SURV_E_INVALID; }
  const int64_t n = d->n, p = d->p;
  if (n < 0 || p < 1 || n > 0x7fffffff || p > 0x7fffffff) { set_error("bad sizes n=%lld p=%lld", (long long)n, (long long)p); return SURV_E_INVALID; }
  if (d->layout != SURV_CSC && d->layout != SURV_DENSE) { set_error("bad layout"); return SURV_E_INVALID; }
  if (d->dtype != SURV_F32 && d->dtype != SURV_F64 && !(d->dtype == SURV_BF16 && d->layout == SURV_DENSE)) {
    set_error("bad dtype (bfloat16 is for dense X only)");
    return SURV_E_INVALID;
  }
  if (o.penalty < 0 || o.penalty > 2 || o.precision < 0 || o.precision > 1) { set_error("bad penalty/precision"); return SURV_E_INVALID; }
  if (!(o.lambda >= 0.0) || !std::isfinite(o.lambda) || !(o.tol >= 0.0) || o.max_sweeps < 0) { set_error("bad lambda/tol/max_sweeps"); return SURV_E_INVALID; }
  if ((o.flags & ~(SURV_FLAG_TEST_STALL | SURV_FLAG_PERSISTENT | SURV_FLAG_SPARSE_NUMERATOR | SURV_FLAG_ONE_COORDINATE |
                   SURV_FLAG_SPEC_B8 | SURV_FLAG_NO_PDL)) !=
      0) {
    set_error("unknown flags");
    return SURV_E_INVALID;
  }
  // the sparse-numerator form: Cox, CSC, FP32 mode, a full fit on the default schedule
  const bool sn = (o.flags & SURV_FLAG_SPARSE_NUMERATOR) != 0;
  if (sn && (model != SURV_COX || d->layout != SURV_CSC || o.precision != SURV_PREC_F32C || single_j >= 0 ||
             (o.flags & (SURV_FLAG_TEST_STALL | SURV_FLAG_PERSISTENT)) != 0)) {
    set_error("SURV_FLAG_SPARSE_NUMERATOR needs a Cox fit of CSC data in the FP32 mode on the default schedule");
    return SURV_E_INVALID;
  }
  if (single_j >= 0 && single_j >= p) { set_error("coordinate j=%d out of range", single_j); return SURV_E_INVALID; }
  if (n == 0) { set_error("no subjects"); return SURV_E_NO_EVENTS; }
  if (!d->time || !d->status) { set_error("null time/status"); return SURV_E_INVALID; }
  if (d->layout == SURV_CSC && (!d->col_ptr || !d->row_idx)) { set_error("null CSC arrays"); return SURV_E_INVALID; }
  if (d->layout == SURV_DENSE && !d->values) { set_error("null dense values"); return SURV_E_INVALID; }

  cudaStream_t s = static_cast<cudaStream_t>(o.stream);
  int64_t launches = 0;
  WsGuard guard;
  surv_workspace* ws = o.workspace;
  if (!ws) {
    ws = new surv_workspace();
    guard.ws = ws;
    guard.owned = true;
  }
  CUDA_TRY(cudaGetDevice(&ws->device));
  const int prec = o.precision;              // 0: float / float-float, 1: double
  const size_t tsz = prec == 0 ? 4 : 8;
  const int layout = d->layout;
  const int M = model == SURV_COX ? 3 : 6;
  using W = surv_workspace;

  // fits run as per-coordinate kernels replayed in a CUDA graph; the single
  // evaluation of loglik_grad_hess, the stall test and SURV_FLAG_PERSISTENT
  // use the persistent kernel
  const bool graph = single_j < 0 && (o.flags & (SURV_FLAG_TEST_STALL | SURV_FLAG_PERSISTENT)) == 0;
  int G = 0, wpc = 0;
  if (graph) CUDA_TRY(survgpu::graph_grid_size(model, layout, prec, &G, &wpc));
  else CUDA_TRY(survgpu::ccd_grid_size(model, layout, prec, &G, &wpc));
  if (G < 1) { set_error("CCD kernel cannot be made co-resident"); return SURV_E_CUDA; }
  const int32_t nwarps = G * wpc;
  const int64_t nwords = (n + 31) / 32;
  const int32_t wpw = (int32_t)((nwords + nwarps - 1) / nwarps);
  const int64_t rows_per_warp = (int64_t)wpw * 32;

  // ---------------------------------------------------------- staging
  int rc;
  Staged stg;
  if ((rc = stage_data(d, prec, ws, s, &stg, &launches))) return rc;
  const void *colptr_d = stg.colptr, *rowidx_d = stg.rowidx;
  const int64_t ld = stg.ld;
  const std::vector<int64_t>& colptr_h = stg.colptr_h;

  // host copies of beta and penalty factors (p values each)
  std::vector<double> beta_h(p), pf_h(p, 1.0), pen_h(p);
  if ((rc = to_host(beta_inout, 8 * (size_t)p, beta_h.data(), s))) return rc;
  if (o.penalty_factor && (rc = to_host(o.penalty_factor, 8 * (size_t)p, pf_h.data(), s))) return rc;
  for (int64_t j = 0; j < p; ++j) {
    if (!std::isfinite(beta_h[j]) || !std::isfinite(pf_h[j]) || pf_h[j] < 0.0) {
      set_error("non-finite beta or invalid penalty factor at %lld", (long long)j);
      return SURV_E_NONFINITE;
    }
    pen_h[j] = o.lambda * pf_h[j];
  }

  // ---------------------------------------------------------- validation, K
  void* ctrl_v = nullptr;
  if ((rc = ensure(ws, W::CTRL, sizeof(DevCtrl), &ctrl_v))) return rc;
  DevCtrl* ctrl = static_cast<DevCtrl*>(ctrl_v);
  const int32_t* time_p = stg.time;
  const int8_t* status_p = stg.status;
  void* blockcnt = nullptr;
  int32_t K = 0;
  if ((rc = validate_and_count(model, layout, prec, n, p, stg, ctrl, ws, s, &blockcnt, &K, &launches))) return rc;
  const void* vals_d = stg.vals;  // null for indicator CSC data (all values 1)
  DevCtrl hc;

  // ---------------------------------------------------------- tables
  void *gend, *dk, *ck, *Gk, *rec, *e, *eta, *w2 = nullptr, *wk0, *woff = nullptr, *dTx, *beta, *width, *pen, *slots;
  constexpr size_t accsz = 8;  // an accumulator: ff (2 floats) or double
  if ((rc = ensure(ws, W::GEND, 4 * (size_t)K, &gend))) return rc;
  if ((rc = ensure(ws, W::DK, 4 * (size_t)K, &dk))) return rc;
  if ((rc = ensure(ws, W::CK, 4 * (size_t)K, &ck))) return rc;
  if ((rc = ensure(ws, W::GK, 8 * (size_t)K, &Gk))) return rc;
  void* Gkff = nullptr;
  if ((rc = ensure(ws, W::GKFF, 8 * (size_t)K, &Gkff))) return rc;
  // speculative coordinate batches (the default for Cox fits of CSC data in
  // the FP32 mode): 4 columns per row pass, the fastest measured at N = 10^7
  // (8 columns: SURV_FLAG_SPEC_B8, for comparison).  Not when the tie groups
  // outnumber twice the warps: the transform of 4 columns at ~10^6 group
  // ends costs more than the passes saved (measured 107 against 68 ms per
  // fit at N = 2 x 10^6 with unique times).
  int spec_b = 0;
  if (!(o.flags & SURV_FLAG_ONE_COORDINATE) && graph && !sn && model == SURV_COX && layout == SURV_CSC &&
      prec == 0 && p >= 2 && (int64_t)K < 2 * (int64_t)nwarps) {
    spec_b = (o.flags & SURV_FLAG_SPEC_B8) ? 8 : 4;
  }
  const int R = spec_b ? 1 + 2 * spec_b : M;  // record / aggregate components
  if ((rc = ensure(ws, W::REC, accsz * (size_t)K * R, &rec))) return rc;
  if ((rc = ensure(ws, W::E, tsz * (size_t)n, &e))) return rc;
  if ((rc = ensure(ws, W::ETA, 8 * (size_t)n, &eta))) return rc;
  if (model == SURV_FG && (rc = ensure(ws, W::W2, tsz * (size_t)n, &w2))) return rc;
  if ((rc = ensure(ws, W::WK0, 4 * (size_t)(nwarps + 1), &wk0))) return rc;
  if (layout == SURV_CSC && (rc = ensure(ws, W::WOFF, 4 * (size_t)p * (nwarps + 1), &woff))) return rc;
  if ((rc = ensure(ws, W::DTX, 8 * (size_t)p, &dTx))) return rc;
  if ((rc = ensure(ws, W::BETA, 8 * (size_t)p, &beta))) return rc;
  if ((rc = ensure(ws, W::WIDTH, 8 * (size_t)p, &width))) return rc;
  if ((rc = ensure(ws, W::PEN, 8 * (size_t)p, &pen))) return rc;
  const size_t slot_bytes = 4 * (size_t)survgpu::kSlotWords * 2 * G;
  if ((rc = ensure(ws, W::SLOTS, 2 * slot_bytes, &slots))) return rc;
  void* wt = nullptr;
  void* aggr = nullptr;
  if (graph && (rc = ensure(ws, W::WT, 8 * (size_t)R * nwarps, &wt))) return rc;
  if (graph && (rc = ensure(ws, W::AGG, 8 * (size_t)survgpu::kRep * R * G, &aggr))) return rc;
  survgpu::SnParams S;
  std::memset(&S, 0, sizeof(S));
  if (sn) {
    void *grp, *den, *v1, *v2, *lamv, *Wv, *pden, *ll, *pcol;
    if ((rc = ensure(ws, W::SN_GRP, 4 * (size_t)n, &grp))) return rc;
    if ((rc = ensure(ws, W::SN_DEN, 8 * (size_t)K, &den))) return rc;
    if ((rc = ensure(ws, W::SN_V1, 8 * (size_t)K, &v1))) return rc;
    if ((rc = ensure(ws, W::SN_V2, 8 * (size_t)K, &v2))) return rc;
    if ((rc = ensure(ws, W::SN_LAM, 8 * (size_t)K, &lamv))) return rc;
    if ((rc = ensure(ws, W::SN_W, 8 * (size_t)(K + 1), &Wv))) return rc;
    if ((rc = ensure(ws, W::SN_PDEN, 8 * 3 * (size_t)G, &pden))) return rc;
    if ((rc = ensure(ws, W::SN_LL, 8, &ll))) return rc;
    // column kernels: at most 8 entries per thread of 256 (the longest column)
    int64_t maxnnz = 0;
    for (int64_t j = 0; j < p; ++j) maxnnz = std::max(maxnnz, colptr_h[j + 1] - colptr_h[j]);
    const int G2 = (int)std::max<int64_t>(G, (maxnnz + 2047) / 2048);
    if ((rc = ensure(ws, W::SN_PCOL, 8 * 4 * (size_t)G2, &pcol))) return rc;
    S.grp = static_cast<const int32_t*>(grp);
    S.den = static_cast<double*>(den);
    S.v1 = static_cast<double*>(v1);
    S.v2 = static_cast<double*>(v2);
    S.lam = static_cast<float2*>(lamv);
    S.W = static_cast<float2*>(Wv);
    S.part_den = static_cast<double*>(pden);
    S.ll_den = static_cast<double*>(ll);
    S.part_col = static_cast<uint64_t*>(pcol);
    S.G2 = G2;
    S.multi = (int64_t)K >= 2 * (int64_t)nwarps ? 1 : 0;
  }

  CUDA_TRY(survgpu::prep_write_ends(time_p, n, static_cast<const int32_t*>(blockcnt), static_cast<int32_t*>(gend), s));
  CUDA_TRY(survgpu::prep_group_stats(static_cast<int32_t*>(gend), K, status_p, n, static_cast<int32_t*>(dk),
                                     static_cast<int32_t*>(ck), &ctrl->total_events, s));
  launches += 2;
  if (model == SURV_FG) {
    CUDA_TRY(survgpu::prep_km(static_cast<int32_t*>(gend), static_cast<int32_t*>(ck), K, static_cast<double*>(Gk),
                              static_cast<float2*>(Gkff), s));
    CUDA_TRY(survgpu::prep_w2(static_cast<int32_t*>(gend), K, status_p, static_cast<double*>(Gk), w2, prec, s));
    launches += 2;
  }
  if (layout == SURV_CSC) {
    CUDA_TRY(survgpu::prep_dtx_csc(static_cast<const int64_t*>(colptr_d), static_cast<const int32_t*>(rowidx_d),
                                   vals_d, prec, status_p, p, static_cast<double*>(dTx), s));
    CUDA_TRY(survgpu::prep_warp_offsets(static_cast<const int64_t*>(colptr_d), static_cast<const int32_t*>(rowidx_d),
                                        p, n, nwarps, rows_per_warp, static_cast<int32_t*>(woff), s));
    launches += 2;
  } else {
    CUDA_TRY(survgpu::prep_dtx_dense(vals_d, prec, ld, n, status_p, p, static_cast<double*>(dTx), s));
    ++launches;
  }
  CUDA_TRY(survgpu::prep_warp_groups(static_cast<int32_t*>(gend), K, n, nwarps, rows_per_warp,
                                     static_cast<int32_t*>(wk0), s));
  ++launches;
  CUDA_TRY(cudaMemcpyAsync(beta, beta_h.data(), 8 * (size_t)p, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(pen, pen_h.data(), 8 * (size_t)p, cudaMemcpyHostToDevice, s));
  CUDA_TRY(survgpu::prep_fill_f64(static_cast<double*>(width), 1.0, p, s));
  ++launches;
  bool any_beta = false;
  for (double b : beta_h) any_beta |= (b != 0.0);
  if (!any_beta) {
    CUDA_TRY(survgpu::prep_eta_zero(prec, n, eta, e, s));
    ++launches;
  } else if (layout == SURV_DENSE) {
    CUDA_TRY(survgpu::prep_eta_dense(vals_d, prec, ld, n, p, static_cast<double*>(beta), eta, e, s));
    ++launches;
  } else {
    CUDA_TRY(survgpu::prep_eta_zero(prec, n, eta, e, s));
    ++launches;
    const size_t vsz = prec == 0 ? 4 : 8;
    for (int64_t j = 0; j < p; ++j) {
      if (beta_h[j] == 0.0) continue;
      const int64_t a = colptr_h[j], b = colptr_h[j + 1];
      const void* vj = vals_d ? static_cast<const char*>(vals_d) + vsz * (size_t)a : nullptr;
      CUDA_TRY(survgpu::prep_eta_axpy_csc(nullptr, static_cast<const int32_t*>(rowidx_d) + a, vj, prec, j, b - a,
                                          beta_h[j], eta, s));
      ++launches;
    }
    CUDA_TRY(survgpu::prep_eta_exp(prec, n, eta, e, s));
    ++launches;
  }
  CUDA_TRY(cudaMemsetAsync(slots, 0, 2 * slot_bytes, s));
  {
    const unsigned long long big = ~0ull;
    CUDA_TRY(cudaMemcpyAsync(&ctrl->timing[survgpu::PH_PASS_MIN], &big, sizeof(big), cudaMemcpyHostToDevice, s));
  }
  CUDA_TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hc.total_events <= 0) { set_error("no events"); return SURV_E_NO_EVENTS; }

  // ---------------------------------------------------------- CCD kernel
  CcdParams P;
  std::memset(&P, 0, sizeof(P));
  P.n = n;
  P.ld = ld;
  P.p = (int32_t)p;
  P.K = K;
  P.G = G;
  P.wpc = wpc;
  P.wpw = wpw;
  P.nwarps = nwarps;
  P.gend = static_cast<const int32_t*>(gend);
  P.dk = static_cast<const int32_t*>(dk);
  P.Gk = static_cast<const double*>(Gk);
  P.Gkff = static_cast<const float2*>(Gkff);
  P.wk0 = static_cast<const int32_t*>(wk0);
  P.col_ptr = static_cast<const int64_t*>(colptr_d);
  P.row_idx = static_cast<const int32_t*>(rowidx_d);
  P.values = layout == SURV_CSC ? vals_d : nullptr;
  P.woff = static_cast<const int32_t*>(woff);
  P.X = layout == SURV_DENSE ? vals_d : nullptr;
  P.e = e;
  P.eta = eta;
  P.w2 = w2;
  P.dTx = static_cast<const double*>(dTx);
  P.beta = static_cast<double*>(beta);
  P.width = static_cast<double*>(width);
  P.pen = static_cast<const double*>(pen);
  P.rec = rec;
  P.slot_agg = static_cast<unsigned*>(slots);
  P.slot_part = static_cast<unsigned*>(slots) + survgpu::kSlotWords * 2 * G;
  P.counters = ctrl->counters;
  P.err = &ctrl->err;
  P.out = ctrl->out;
  P.timing = ctrl->timing;
  P.penalty = single_j >= 0 ? 0 : o.penalty;
  P.max_sweeps = o.max_sweeps;
  P.tol = o.tol;
  P.single_j = single_j;
  P.withhold_cta = (o.flags & SURV_FLAG_TEST_STALL) ? 0 : -1;
  P.no_pdl = (o.flags & SURV_FLAG_NO_PDL) ? 1 : 0;
  P.timeout_ns = (uint64_t)((o.wait_limit_s > 0.0 ? o.wait_limit_s : 2.0) * 1e9);
  if (graph) {
    P.wt = static_cast<uint64_t*>(wt);
    P.agg = static_cast<uint64_t*>(aggr);
    P.gctl = &ctrl->gctl;
  }
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  CUDA_TRY(cudaEventCreate(&ev.a));
  CUDA_TRY(cudaEventCreate(&ev.b));
  int replays = 0;
  if (graph) {
    int glaunches = 0;
    CUDA_TRY(survgpu::graph_init(P, s));
    ++launches;
    if (spec_b) {
      CUDA_TRY(survgpu::run_spec_graph(P, spec_b, s, o_in && o_in->workspace ? &ws->graph : nullptr, ev.a, &replays,
                                       &glaunches));
    } else if (sn) {
      CUDA_TRY(survgpu::sn_groups(static_cast<const int32_t*>(gend), K, n, const_cast<int32_t*>(S.grp), s));
      ++launches;
      CUDA_TRY(survgpu::run_sn_graph(P, S, s, o_in && o_in->workspace ? &ws->graph : nullptr, ev.a, &replays,
                                     &glaunches));
    } else {
      CUDA_TRY(survgpu::run_ccd_graph(model, layout, prec, P, s, o_in && o_in->workspace ? &ws->graph : nullptr,
                                      ev.a, &replays, &glaunches));
    }
    launches += glaunches;
  } else {
    CUDA_TRY(cudaEventRecord(ev.a, s));
    CUDA_TRY(survgpu::launch_ccd(model, layout, prec, P, s));
    ++launches;
  }
  CUDA_TRY(cudaEventRecord(ev.b, s));
  CUDA_TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  std::vector<double> beta_out(p);
  CUDA_TRY(cudaMemcpyAsync(beta_out.data(), beta, 8 * (size_t)p, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  float kernel_ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&kernel_ms, ev.a, ev.b));

  if (single_j < 0) {
    CUDA_TRY(cudaMemcpyAsync(beta_inout, beta_out.data(), 8 * (size_t)p, cudaMemcpyDefault, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->sweeps = (int32_t)hc.out[survgpu::OUT_SWEEPS];
    info->converged = (int32_t)hc.out[survgpu::OUT_CONVERGED];
    int nz = 0;
    for (double b : beta_out) nz += b != 0.0;
    info->nnz_beta = nz;
    info->device_error = (int32_t)hc.err;
    info->loglik = hc.out[survgpu::OUT_LOGLIK];
    info->objective = hc.out[survgpu::OUT_OBJECTIVE];
    info->objective_prev = hc.out[survgpu::OUT_OBJECTIVE_PREV];
    info->n_groups = K;
    info->coordinate_passes = (int64_t)hc.out[survgpu::OUT_PASSES];
    info->eta_updates = (int64_t)hc.out[survgpu::OUT_ETA_UPDATES];
    info->kernel_launches = launches;
    info->ccd_kernel_ms = kernel_ms;
    for (int i = 0; i < 16; ++i) info->phase_ms[i] = (double)hc.timing[i] * 1e-6;
    info->phase_ms[survgpu::PH_PASS_SUM] /= (double)G;  // mean over CTAs
    info->row_passes = (int64_t)hc.out[spec_b ? survgpu::OUT_BATCHES : survgpu::OUT_PASSES];
  }
  if (graph && hc.gctl.done != 1) {
    set_error("CCD stopped after %d sweep replays without a stop decision", replays);
    return SURV_E_CUDA;
  }
  if (hc.err != 0) {
    set_error("device-side wait expired (error word 0x%x)", hc.err);
    return SURV_E_DEVICE_TIMEOUT;
  }
  if (single_j >= 0) {
    if (out_l) *out_l = hc.out[survgpu::OUT_LOGLIK];
    if (out_g) *out_g = hc.out[survgpu::OUT_GRAD];
    if (out_h) *out_h = hc.out[survgpu::OUT_HESS];
    return SURV_OK;
  }
  return hc.out[survgpu::OUT_CONVERGED] != 0.0 ? SURV_OK : SURV_W_NOT_CONVERGED;
}

// ---------------------------------------------------------------- lambda_max
int lambda_max_impl(const surv_data* d, const double* pf_in, double* out, void* stream) {
  g_last_error[0] = '\0';
  if (!out) { set_error("null lambda_max"); return SURV_E_INVALID; }
  int rc;
  if ((rc = check_data(d))) return rc;
  const int64_t n = d->n, p = d->p;
  const int layout = d->layout;
  const int prec = d->dtype == SURV_F64 ? 1 : 0;  // the data's own precision (bfloat16 widens to FP32); FP64 sums
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  surv_workspace ws;
  struct Free { surv_workspace* w; ~Free() { free_all(w); } } fr{&ws};
  using W = surv_workspace;
  CUDA_TRY(cudaGetDevice(&ws.device));
  int64_t launches = 0;
  Staged stg;
  if ((rc = stage_data(d, prec, &ws, s, &stg, &launches))) return rc;
  const double* pf_d = nullptr;
  if (pf_in) {
    std::vector<double> pf_h(p);
    if ((rc = to_host(pf_in, 8 * (size_t)p, pf_h.data(), s))) return rc;
    for (int64_t j = 0; j < p; ++j)
      if (!std::isfinite(pf_h[j]) || pf_h[j] < 0.0) { set_error("invalid penalty factor at %lld", (long long)j); return SURV_E_NONFINITE; }
    const void* v = nullptr;
    if ((rc = device_view(&ws, W::PF, pf_in, 8 * (size_t)p, s, &v))) return rc;
    pf_d = static_cast<const double*>(v);
  }
  void* ctrl_v = nullptr;
  if ((rc = ensure(&ws, W::CTRL, sizeof(DevCtrl), &ctrl_v))) return rc;
  DevCtrl* ctrl = static_cast<DevCtrl*>(ctrl_v);
  void* blockcnt = nullptr;
  int32_t K = 0;
  if ((rc = validate_and_count(SURV_COX, layout, prec, n, p, stg, ctrl, &ws, s, &blockcnt, &K, &launches))) return rc;
  void *gend, *dk, *ck, *lam, *r, *g;
  if ((rc = ensure(&ws, W::GEND, 4 * (size_t)K, &gend))) return rc;
  if ((rc = ensure(&ws, W::DK, 4 * (size_t)K, &dk))) return rc;
  if ((rc = ensure(&ws, W::CK, 4 * (size_t)K, &ck))) return rc;
  if ((rc = ensure(&ws, W::LM_LAM, 8 * (size_t)K, &lam))) return rc;
  if ((rc = ensure(&ws, W::LM_R, 8 * (size_t)n, &r))) return rc;
  if ((rc = ensure(&ws, W::LM_G, 8 * (size_t)(p + 1), &g))) return rc;
  CUDA_TRY(survgpu::prep_write_ends(stg.time, n, static_cast<const int32_t*>(blockcnt), static_cast<int32_t*>(gend), s));
  CUDA_TRY(survgpu::prep_group_stats(static_cast<int32_t*>(gend), K, stg.status, n, static_cast<int32_t*>(dk),
                                     static_cast<int32_t*>(ck), &ctrl->total_events, s));
  double* gd = static_cast<double*>(g);
  CUDA_TRY(survgpu::lambda_max_device(layout, prec, stg.colptr, stg.rowidx, stg.vals, stg.ld, n, p, stg.status,
                                      static_cast<const int32_t*>(gend), static_cast<const int32_t*>(dk), K, pf_d,
                                      static_cast<double*>(lam), static_cast<double*>(r), gd, gd + p, s));
  DevCtrl hc;
  double v = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&v, gd + p, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hc.total_events <= 0) { set_error("no events"); return SURV_E_NO_EVENTS; }
  *out = v;
  return SURV_OK;
}

// ------------------------------------------------------ cross-validated path
struct CvCtrl {
  unsigned perr;
  unsigned done;         // fits that have stopped
  int32_t best;          // index of the chosen lambda
  int32_t pad;
  int32_t events[128];   // training events per fold
};

// CTAs per fit when neither the caller nor the tuner chose: about ten waves
// of co-resident CTAs over all fits (measured best at N = 10^6, 200 fits:
// 16 CTAs per fit; 1 gave 98 fits/s, 3 gave 142, 16 gave 179, 48 gave 147),
// within the rows available (at least one 32-row word per warp).
int cv_ctas_default(int F, int Gmax, int max_by_rows) {
  const int lim = std::max(1, std::min(Gmax, max_by_rows));
  const int g = (int)((10LL * Gmax + F / 2) / F);
  return std::max(1, std::min(g, lim));
}

int cv_impl(const surv_data* d, const int8_t* fold_id, int nfolds, const double* lambdas, int nlambda,
            const surv_opts* o_in, int ctas_per_fit, double* beta_out, double* heldout_out, double* cv_mean_out,
            int32_t* sweeps_out, surv_cv_info* info) {
  g_last_error[0] = '\0';
  surv_opts o;
  if (o_in) o = *o_in; else surv_opts_default(&o);
  int rc;
  if ((rc = check_data(d))) return rc;
  if (!fold_id || !lambdas || !beta_out) { set_error("null fold_id, lambdas or beta_out"); return SURV_E_INVALID; }
  if (nfolds < 1 || nfolds > 127 || nlambda < 1 || (int64_t)nfolds * nlambda > 65535) {
    set_error("bad nfolds=%d / nlambda=%d", nfolds, nlambda);
    return SURV_E_INVALID;
  }
  if (ctas_per_fit < 0) { set_error("negative ctas_per_fit"); return SURV_E_INVALID; }
  if (o.penalty < 0 || o.penalty > 2 || o.precision < 0 || o.precision > 1) { set_error("bad penalty/precision"); return SURV_E_INVALID; }
  if (!(o.tol >= 0.0) || o.max_sweeps < 0) { set_error("bad tol/max_sweeps"); return SURV_E_INVALID; }
  if ((o.flags & ~(SURV_FLAG_CV_TUNE | SURV_FLAG_CV_TILE1 | SURV_FLAG_CV_TILE2)) != 0 ||
      (o.flags & SURV_FLAG_CV_TILE1 && o.flags & SURV_FLAG_CV_TILE2)) {
    set_error("unknown flags for cox_cv_path");
    return SURV_E_INVALID;
  }
  const int64_t n = d->n, p = d->p;
  const int F = nfolds * nlambda;
  const int layout = d->layout;
  const int prec = o.precision;
  const size_t tsz = prec == 0 ? 4 : 8;
  constexpr int M = 3;
  // per-fit strides: every fit's arrays start on a 256-byte boundary (the
  // pass reads e with 16-byte vector loads)
  auto pad = [](size_t elems, size_t esz) { return (elems * esz + 255) / 256 * 256 / esz; };
  const int64_t fit_n = (int64_t)pad((size_t)n, 8);  // elements of e and eta per fit
  cudaStream_t s = static_cast<cudaStream_t>(o.stream);
  int64_t launches = 0;
  WsGuard guard;
  surv_workspace* ws = o.workspace;
  if (!ws) {
    ws = new surv_workspace();
    guard.ws = ws;
    guard.owned = true;
  }
  CUDA_TRY(cudaGetDevice(&ws->device));
  using W = surv_workspace;

  // lambdas and penalty factors (host copies; pen[f][j] = lambda_l * pf_j)
  std::vector<double> lam_h(nlambda), pf_h(p, 1.0);
  if ((rc = to_host(lambdas, 8 * (size_t)nlambda, lam_h.data(), s))) return rc;
  for (double l : lam_h)
    if (!std::isfinite(l) || l < 0.0) { set_error("lambdas must be finite and >= 0"); return SURV_E_INVALID; }
  if (o.penalty_factor && (rc = to_host(o.penalty_factor, 8 * (size_t)p, pf_h.data(), s))) return rc;
  for (int64_t j = 0; j < p; ++j)
    if (!std::isfinite(pf_h[j]) || pf_h[j] < 0.0) { set_error("invalid penalty factor at %lld", (long long)j); return SURV_E_NONFINITE; }

  // CTAs per fit: the caller's, else the tuned value kept in the workspace
  // for this shape, else the default; SURV_FLAG_CV_TUNE times one sweep for
  // each candidate first and keeps the fastest
  int Gmax = 0, wpc = 0;
  CUDA_TRY(survgpu::graph_grid_size(SURV_COX, layout, prec, &Gmax, &wpc));
  if (Gmax < 1) { set_error("CCD kernels do not fit on the device"); return SURV_E_CUDA; }
  const int64_t nwords = (n + 31) / 32;
  const int max_by_rows = (int)std::min<int64_t>(Gmax, std::max<int64_t>(1, nwords / wpc));
  const bool tune = ctas_per_fit == 0 && (o.flags & SURV_FLAG_CV_TUNE) != 0;
  const int64_t tkey[6] = {n, p, (int64_t)F, (int64_t)layout * 2 + prec, (int64_t)d->dtype,
                           d->layout == SURV_CSC ? (int64_t)-1 : (int64_t)0};
  int G = ctas_per_fit > 0 ? std::min(ctas_per_fit, Gmax) : cv_ctas_default(F, Gmax, max_by_rows);
  int form = 0;  // row-pass form: 0 by the ends per warp
  int tile = 0;  // tile shape of the CSC FP32 row pass
  if (ctas_per_fit == 0 && !tune && ws->cv_tuned_ctas > 0 && std::memcmp(ws->cv_tune_key, tkey, sizeof(tkey)) == 0) {
    G = ws->cv_tuned_ctas;
    form = ws->cv_tuned_form;
    tile = ws->cv_tuned_tile;
  }
  const int tile_forced = (o.flags & SURV_FLAG_CV_TILE1) ? 1 : ((o.flags & SURV_FLAG_CV_TILE2) ? 2 : -1);
  const bool tile_ok = layout == SURV_CSC && prec == 0;  // the shapes exist for CSC data in the FP32 mode
  if (tile_forced >= 0) tile = tile_ok ? tile_forced : 0;
  std::vector<int> cands;
  if (tune) {
    for (int g : {G / 2, G, 2 * G, 3 * G})
      if (g >= 1 && g <= max_by_rows && std::find(cands.begin(), cands.end(), g) == cands.end()) cands.push_back(g);
    if (cands.empty()) cands.push_back(G);
  }
  const int Galloc = tune ? *std::max_element(cands.begin(), cands.end()) : G;

  // staging and validation
  Staged stg;
  if ((rc = stage_data(d, prec, ws, s, &stg, &launches))) return rc;
  void* ctrl_v = nullptr;
  if ((rc = ensure(ws, W::CTRL, sizeof(DevCtrl), &ctrl_v))) return rc;
  DevCtrl* ctrl = static_cast<DevCtrl*>(ctrl_v);
  void* blockcnt = nullptr;
  int32_t K = 0;
  if ((rc = validate_and_count(SURV_COX, layout, prec, n, p, stg, ctrl, ws, s, &blockcnt, &K, &launches))) return rc;
  const void* fold_v = nullptr;
  if ((rc = device_view(ws, W::CV_FOLD, fold_id, (size_t)n, s, &fold_v))) return rc;
  const int8_t* fold_d = static_cast<const int8_t*>(fold_v);

  // shared tables, per-fold tables, per-fit state (scratch sized for the
  // largest grid tried)
  const int32_t nwarps_alloc = Galloc * wpc;
  // one coordinate per pass: the fits run in lockstep, so speculative
  // batches would be as many as the slowest fit needs (measured slower:
  // 180 against 237 fits/s at N = 10^6, 200 fits)
  const int RC = M, NPART = 3;
  void *gend, *dk, *ck, *wk0, *woff = nullptr, *dkf, *dtxf, *cvc_v;
  void *e, *eta, *rec, *wt, *agg, *part, *gctl, *beta, *width, *pen, *out, *fits, *den, *held, *mean;
  const size_t rec_f = pad((size_t)K * RC, 8), wt_f = pad((size_t)RC * nwarps_alloc, 8);
  const size_t agg_f = pad((size_t)survgpu::kRep * RC * Galloc, 8), part_f = pad((size_t)NPART * Galloc, 8);
  if ((rc = ensure(ws, W::GEND, 4 * (size_t)K, &gend))) return rc;
  if ((rc = ensure(ws, W::DK, 4 * (size_t)K, &dk))) return rc;
  if ((rc = ensure(ws, W::CK, 4 * (size_t)K, &ck))) return rc;
  if ((rc = ensure(ws, W::WK0, 4 * (size_t)(nwarps_alloc + 1), &wk0))) return rc;
  if (layout == SURV_CSC && (rc = ensure(ws, W::WOFF, 4 * (size_t)p * (nwarps_alloc + 1), &woff))) return rc;
  if ((rc = ensure(ws, W::CV_DK, 4 * (size_t)nfolds * K, &dkf))) return rc;
  if ((rc = ensure(ws, W::CV_DTX, 8 * (size_t)nfolds * p, &dtxf))) return rc;
  if ((rc = ensure(ws, W::CV_CTRL, sizeof(CvCtrl), &cvc_v))) return rc;
  if ((rc = ensure(ws, W::CV_E, tsz * (size_t)F * fit_n, &e))) return rc;
  if ((rc = ensure(ws, W::CV_ETA, 8 * (size_t)F * fit_n, &eta))) return rc;
  if ((rc = ensure(ws, W::CV_REC, 8 * (size_t)F * rec_f, &rec))) return rc;
  if ((rc = ensure(ws, W::CV_WT, 8 * (size_t)F * wt_f, &wt))) return rc;
  if ((rc = ensure(ws, W::CV_AGG, 8 * (size_t)F * agg_f, &agg))) return rc;
  if ((rc = ensure(ws, W::CV_PART, 8 * (size_t)F * part_f, &part))) return rc;
  if ((rc = ensure(ws, W::CV_GCTL, sizeof(survgpu::GraphCtl) * (size_t)F, &gctl))) return rc;
  if ((rc = ensure(ws, W::CV_BETA, 8 * (size_t)F * p, &beta))) return rc;
  if ((rc = ensure(ws, W::CV_WIDTH, 8 * (size_t)F * p, &width))) return rc;
  if ((rc = ensure(ws, W::CV_PEN, 8 * (size_t)F * p, &pen))) return rc;
  if ((rc = ensure(ws, W::CV_OUT, 8 * (size_t)F * survgpu::OUT_COUNT, &out))) return rc;
  if ((rc = ensure(ws, W::CV_FITS, sizeof(CcdParams) * (size_t)F, &fits))) return rc;
  if ((rc = ensure(ws, W::CV_DEN, 8 * (size_t)F * K, &den))) return rc;
  if ((rc = ensure(ws, W::CV_HELD, 8 * (size_t)F, &held))) return rc;
  if ((rc = ensure(ws, W::CV_MEAN, 8 * (size_t)nlambda, &mean))) return rc;
  CvCtrl* cvc = static_cast<CvCtrl*>(cvc_v);

  CUDA_TRY(cudaMemsetAsync(cvc, 0, sizeof(CvCtrl), s));
  CUDA_TRY(survgpu::cv_check_folds(fold_d, n, nfolds, &cvc->perr, s));
  CUDA_TRY(survgpu::prep_write_ends(stg.time, n, static_cast<const int32_t*>(blockcnt), static_cast<int32_t*>(gend), s));
  CUDA_TRY(survgpu::prep_group_stats(static_cast<int32_t*>(gend), K, stg.status, n, static_cast<int32_t*>(dk),
                                     static_cast<int32_t*>(ck), &ctrl->total_events, s));
  CUDA_TRY(survgpu::cv_fold_stats(static_cast<int32_t*>(gend), K, stg.status, fold_d, nfolds,
                                  static_cast<int32_t*>(dkf), cvc->events, s));
  CUDA_TRY(survgpu::cv_dtx(layout == SURV_CSC ? 0 : 1, prec, stg.colptr, stg.rowidx, stg.vals, stg.ld, n, p,
                           stg.status, fold_d, nfolds, static_cast<double*>(dtxf), s));
  launches += 5;
  std::vector<double> pen_h((size_t)F * p);
  for (int f = 0; f < F; ++f)
    for (int64_t j = 0; j < p; ++j) pen_h[(size_t)f * p + j] = lam_h[f / nfolds] * pf_h[j];
  CUDA_TRY(cudaMemcpyAsync(pen, pen_h.data(), 8 * pen_h.size(), cudaMemcpyHostToDevice, s));
  CvCtrl hcv;
  DevCtrl hc;
  CUDA_TRY(cudaMemcpyAsync(&hcv, cvc, sizeof(CvCtrl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hcv.perr & survgpu::PREP_FOLD) { set_error("fold_id outside [0, %d)", nfolds); return SURV_E_INVALID; }
  if (hc.total_events <= 0) { set_error("no events"); return SURV_E_NO_EVENTS; }
  for (int k = 0; k < nfolds; ++k)
    if (hcv.events[k] <= 0) { set_error("no events outside fold %d", k); return SURV_E_NO_EVENTS; }

  // Grid tables, per-fit parameters and a cold start for G CTAs per fit;
  // *P0 receives the launch parameters (fit 0's, with the table of all fits).
  std::vector<CcdParams> fits_h(F);
  auto setup = [&](int Gc, int form_c, int tile_c, CcdParams* P0) -> int {
    const int32_t nwarps = Gc * wpc;
    const int32_t wpw = (int32_t)((nwords + nwarps - 1) / nwarps);
    const int64_t rows_per_warp = (int64_t)wpw * 32;
    if (layout == SURV_CSC) {
      CUDA_TRY(survgpu::prep_warp_offsets(stg.colptr, stg.rowidx, p, n, nwarps, rows_per_warp,
                                          static_cast<int32_t*>(woff), s));
      ++launches;
    }
    CUDA_TRY(survgpu::prep_warp_groups(static_cast<int32_t*>(gend), K, n, nwarps, rows_per_warp,
                                       static_cast<int32_t*>(wk0), s));
    CUDA_TRY(survgpu::cv_init(prec, n, fit_n, fold_d, nfolds, F, e, eta, s));
    CUDA_TRY(survgpu::prep_fill_f64(static_cast<double*>(width), 1.0, (int64_t)F * p, s));
    launches += 3;
    CUDA_TRY(cudaMemsetAsync(beta, 0, 8 * (size_t)F * p, s));
    CUDA_TRY(cudaMemsetAsync(gctl, 0, sizeof(survgpu::GraphCtl) * (size_t)F, s));
    CUDA_TRY(cudaMemsetAsync(out, 0, 8 * (size_t)F * survgpu::OUT_COUNT, s));
    CUDA_TRY(cudaMemsetAsync(&cvc->done, 0, sizeof(unsigned), s));
    CcdParams P;
    std::memset(&P, 0, sizeof(P));
    P.pass_form = form_c;
    P.tile_form = tile_c;
    P.n = n;
    P.ld = stg.ld;
    P.p = (int32_t)p;
    P.K = K;
    P.G = Gc;
    P.wpc = wpc;
    P.wpw = wpw;
    P.nwarps = nwarps;
    P.gend = static_cast<const int32_t*>(gend);
    P.wk0 = static_cast<const int32_t*>(wk0);
    P.col_ptr = stg.colptr;
    P.row_idx = stg.rowidx;
    P.values = layout == SURV_CSC ? stg.vals : nullptr;
    P.woff = static_cast<const int32_t*>(woff);
    P.X = layout == SURV_DENSE ? stg.vals : nullptr;
    P.penalty = o.penalty;
    P.max_sweeps = o.max_sweeps;
    P.tol = o.tol;
    P.single_j = -1;
    P.withhold_cta = -1;
    P.done_count = &cvc->done;
    P.nfit = F;
    P.fold_id = fold_d;
    for (int f = 0; f < F; ++f) {
      const int k = f % nfolds;
      CcdParams& Q = fits_h[f];
      Q = P;
      Q.fold = k;
      Q.dk = static_cast<const int32_t*>(dkf) + (size_t)k * K;
      Q.dTx = static_cast<const double*>(dtxf) + (size_t)k * p;
      Q.e = static_cast<char*>(e) + tsz * (size_t)f * fit_n;
      Q.eta = static_cast<char*>(eta) + 8 * (size_t)f * fit_n;
      Q.rec = static_cast<char*>(rec) + 8 * (size_t)f * rec_f;
      Q.wt = static_cast<uint64_t*>(wt) + (size_t)f * wt_f;
      Q.agg = static_cast<uint64_t*>(agg) + (size_t)f * agg_f;
      Q.slot_part = reinterpret_cast<unsigned*>(static_cast<uint64_t*>(part) + (size_t)f * part_f);
      Q.gctl = static_cast<survgpu::GraphCtl*>(gctl) + f;
      Q.beta = static_cast<double*>(beta) + (size_t)f * p;
      Q.width = static_cast<double*>(width) + (size_t)f * p;
      Q.pen = static_cast<const double*>(pen) + (size_t)f * p;
      Q.out = static_cast<double*>(out) + (size_t)f * survgpu::OUT_COUNT;
      Q.fits = nullptr;
    }
    CUDA_TRY(cudaMemcpyAsync(fits, fits_h.data(), sizeof(CcdParams) * (size_t)F, cudaMemcpyHostToDevice, s));
    *P0 = fits_h[0];
    P0->fits = static_cast<const CcdParams*>(fits);
    CUDA_TRY(survgpu::graph_init(*P0, s));
    ++launches;
    return SURV_OK;
  };

  const int lmode = layout == SURV_CSC ? 0 : 1;
  CcdParams P0;
  if (tune) {
    // one full sweep of every candidate from the same cold start: CTAs per
    // fit x, for CSC data, the two forms of the row pass (one reduction per
    // group end, or lane scans per tile) x, in the FP32 mode, three tile
    // shapes (the configured one, half the loads of e per lane, half the
    // rounds of nonzeros per load)
    float best_ms = 0.f;
    int best_g = G, best_form = 0, best_tile = 0;
    const std::vector<int> forms = layout == SURV_CSC ? std::vector<int>{1, 2} : std::vector<int>{0};
    const std::vector<int> tiles = tile_forced >= 0 ? std::vector<int>{tile}
                                   : (tile_ok ? std::vector<int>{0, 1, 2} : std::vector<int>{0});
    for (int g : cands)
      for (int fm : forms)
        for (int tw : tiles) {
          if ((rc = setup(g, fm, tw, &P0))) return rc;
          float ms = 0.f;
          CUDA_TRY(survgpu::time_one_sweep(SURV_COX, lmode, prec, P0, s, &ms));
          launches += 2 * p;
          if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            best_g = g;
            best_form = fm;
            best_tile = tw;
          }
        }
    G = best_g;
    form = best_form;
    tile = best_tile;
    ws->cv_tuned_ctas = G;
    ws->cv_tuned_form = form;
    ws->cv_tuned_tile = tile;
    std::memcpy(ws->cv_tune_key, tkey, sizeof(tkey));
  }
  if ((rc = setup(G, form, tile, &P0))) return rc;

  struct Events {
    cudaEvent_t a = nullptr, b = nullptr, c = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (c) cudaEventDestroy(c);
    }
  } ev;
  CUDA_TRY(cudaEventCreate(&ev.a));
  CUDA_TRY(cudaEventCreate(&ev.b));
  CUDA_TRY(cudaEventCreate(&ev.c));
  int replays = 0, glaunches = 0;
  CUDA_TRY(survgpu::run_ccd_graph(SURV_COX, lmode, prec, P0, s, o_in && o_in->workspace ? &ws->graph : nullptr,
                                  ev.a, &replays, &glaunches));
  launches += glaunches;
  CUDA_TRY(cudaEventRecord(ev.b, s));
  CUDA_TRY(survgpu::cv_heldout(prec, n, fit_n, stg.time, stg.status, fold_d, nfolds, F, eta,
                               static_cast<const int32_t*>(dk), static_cast<const int32_t*>(dkf), K,
                               static_cast<double*>(den), static_cast<double*>(held), s));
  CUDA_TRY(survgpu::cv_select(static_cast<const double*>(held), nlambda, nfolds, static_cast<double*>(mean),
                              &cvc->best, s));
  launches += 2;
  CUDA_TRY(cudaEventRecord(ev.c, s));
  std::vector<double> out_h((size_t)F * survgpu::OUT_COUNT);
  CUDA_TRY(cudaMemcpyAsync(out_h.data(), out, 8 * out_h.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&hcv, cvc, sizeof(CvCtrl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hcv.done != (unsigned)F) {
    set_error("%u of %d fits stopped after %d sweep replays", hcv.done, F, replays);
    return SURV_E_CUDA;
  }
  CUDA_TRY(cudaMemcpyAsync(beta_out, beta, 8 * (size_t)F * p, cudaMemcpyDefault, s));
  if (heldout_out) CUDA_TRY(cudaMemcpyAsync(heldout_out, held, 8 * (size_t)F, cudaMemcpyDefault, s));
  if (cv_mean_out) CUDA_TRY(cudaMemcpyAsync(cv_mean_out, mean, 8 * (size_t)nlambda, cudaMemcpyDefault, s));
  std::vector<int32_t> sw((size_t)F);
  int conv = 0, maxsw = 0;
  int64_t passes = 0, updates = 0;
  for (int f = 0; f < F; ++f) {
    const double* of = out_h.data() + (size_t)f * survgpu::OUT_COUNT;
    sw[f] = (int32_t)of[survgpu::OUT_SWEEPS];
    conv += of[survgpu::OUT_CONVERGED] != 0.0;
    maxsw = std::max(maxsw, sw[f]);
    passes += (int64_t)of[survgpu::OUT_PASSES];
    updates += (int64_t)of[survgpu::OUT_ETA_UPDATES];
  }
  if (sweeps_out) CUDA_TRY(cudaMemcpyAsync(sweeps_out, sw.data(), 4 * (size_t)F, cudaMemcpyDefault, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->nfits = F;
    info->best_lambda = hcv.best;
    info->max_sweeps_used = maxsw;
    info->fits_converged = conv;
    info->graph_replays = replays;
    info->ctas_per_fit = G;
    info->row_pass_form = layout == SURV_CSC ? (form == 2 || (form == 0 && (int64_t)K >= 2 * (int64_t)G * wpc) ? 2 : 1) : 0;
    info->tile_form = tile;
    info->kernel_launches = launches;
    info->n_groups = K;
    info->coordinate_passes = passes;
    info->eta_updates = updates;
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b));
    info->ccd_kernel_ms = ms;
    CUDA_TRY(cudaEventElapsedTime(&ms, ev.b, ev.c));
    info->heldout_ms = ms;
  }
  return conv == F ? SURV_OK : SURV_W_NOT_CONVERGED;
}

}  // namespace

namespace survgpu {
void set_last_error_text(const char* msg) { set_error("%s", msg ? msg : ""); }
}  // namespace survgpu

extern "C" {

void surv_opts_default(surv_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->penalty = SURV_PEN_NONE;
  o->precision = SURV_PREC_F32C;
  o->lambda = 0.0;
  o->tol = 1e-8;
  o->max_sweeps = 1000;
}

int surv_workspace_create(surv_workspace** ws) {
  if (!ws) { set_error("null handle pointer"); return SURV_E_INVALID; }
  *ws = new surv_workspace();
  return SURV_OK;
}

int surv_workspace_destroy(surv_workspace* ws) {
  if (!ws) return SURV_OK;
  free_all(ws);
  delete ws;
  return SURV_OK;
}

int surv_sort_desc(const int32_t* time, int64_t n, int32_t* perm, void* stream) {
  g_last_error[0] = '\0';
  if (n < 0 || n > 0x7fffffff) { set_error("bad n"); return SURV_E_INVALID; }
  if (n == 0) return SURV_OK;
  if (!time || !perm) { set_error("null time/perm"); return SURV_E_INVALID; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  surv_workspace ws;
  struct Free { surv_workspace* w; ~Free() { free_all(w); } } fr{&ws};
  const void* tdev = nullptr;
  int rc = device_view(&ws, surv_workspace::TIME, time, 4 * (size_t)n, s, &tdev);
  if (rc) return rc;
  void* work = nullptr;
  if ((rc = ensure(&ws, surv_workspace::SORTWORK, survgpu::radix_sort_workspace(n), &work))) return rc;
  const bool perm_dev = is_device_ptr(perm);
  void* pdev = perm;
  if (!perm_dev && (rc = ensure(&ws, surv_workspace::PERM, 4 * (size_t)n, &pdev))) return rc;
  int launches = 0;
  CUDA_TRY(survgpu::radix_sort_desc(static_cast<const int32_t*>(tdev), n, static_cast<int32_t*>(pdev), work, s,
                                    &launches));
  if (!perm_dev) CUDA_TRY(cudaMemcpyAsync(perm, pdev, 4 * (size_t)n, cudaMemcpyDefault, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return SURV_OK;
}

int cox_fit(const surv_data* data, const surv_opts* opts, double* beta_inout, surv_fit_info* info) {
  return fit_common(SURV_COX, data, opts, beta_inout, info, -1, nullptr, nullptr, nullptr);
}

int fg_fit(const surv_data* data, const surv_opts* opts, double* beta_inout, surv_fit_info* info) {
  return fit_common(SURV_FG, data, opts, beta_inout, info, -1, nullptr, nullptr, nullptr);
}

int loglik_grad_hess(const surv_data* data, int32_t model, const double* beta, int32_t j, double* loglik,
                     double* grad, double* hess, const surv_opts* opts) {
  if (model != SURV_COX && model != SURV_FG) { set_error("bad model"); return SURV_E_INVALID; }
  if (j < 0) { set_error("negative j"); return SURV_E_INVALID; }
  return fit_common(model, data, opts, const_cast<double*>(beta), nullptr, j, loglik, grad, hess);
}

int surv_groups(const int32_t* time, const int8_t* status, int64_t n, int64_t max_groups, int64_t* K_out,
                int32_t* gend_out, int32_t* dk_out, double* Gk_out, void* stream) {
  g_last_error[0] = '\0';
  if (n < 0 || n > 0x7fffffff || !K_out) { set_error("bad n or null K"); return SURV_E_INVALID; }
  *K_out = 0;
  if (n == 0) return SURV_OK;
  if (!time || !status) { set_error("null time/status"); return SURV_E_INVALID; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  surv_workspace ws;
  struct Free { surv_workspace* w; ~Free() { free_all(w); } } fr{&ws};
  using W = surv_workspace;
  const void *time_d = nullptr, *status_d = nullptr;
  int rc;
  if ((rc = device_view(&ws, W::TIME, time, 4 * (size_t)n, s, &time_d))) return rc;
  if ((rc = device_view(&ws, W::STATUS, status, (size_t)n, s, &status_d))) return rc;
  void *ctrl_v, *blockcnt;
  if ((rc = ensure(&ws, W::CTRL, sizeof(DevCtrl), &ctrl_v))) return rc;
  DevCtrl* ctrl = static_cast<DevCtrl*>(ctrl_v);
  CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(DevCtrl), s));
  const int32_t* tp = static_cast<const int32_t*>(time_d);
  const int8_t* sp = static_cast<const int8_t*>(status_d);
  CUDA_TRY(survgpu::prep_check_times(tp, sp, n, 1, &ctrl->perr, s));
  if ((rc = ensure(&ws, W::BLOCKCNT, 4 * (size_t)survgpu::prep_end_blocks(n), &blockcnt))) return rc;
  CUDA_TRY(survgpu::prep_count_ends(tp, n, static_cast<int32_t*>(blockcnt), &ctrl->K, s));
  DevCtrl hc;
  CUDA_TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if ((rc = map_prep_error(hc.perr))) return rc;
  const int32_t K = hc.K;
  *K_out = K;
  if (!gend_out && !dk_out && !Gk_out) return SURV_OK;
  if (K > max_groups) { set_error("K=%d exceeds max_groups", K); return SURV_E_INVALID; }
  void *gend, *dk, *ck, *Gk;
  if ((rc = ensure(&ws, W::GEND, 4 * (size_t)K, &gend))) return rc;
  if ((rc = ensure(&ws, W::DK, 4 * (size_t)K, &dk))) return rc;
  if ((rc = ensure(&ws, W::CK, 4 * (size_t)K, &ck))) return rc;
  if ((rc = ensure(&ws, W::GK, 8 * (size_t)K, &Gk))) return rc;
  CUDA_TRY(survgpu::prep_write_ends(tp, n, static_cast<const int32_t*>(blockcnt), static_cast<int32_t*>(gend), s));
  CUDA_TRY(survgpu::prep_group_stats(static_cast<int32_t*>(gend), K, sp, n, static_cast<int32_t*>(dk),
                                     static_cast<int32_t*>(ck), &ctrl->total_events, s));
  CUDA_TRY(survgpu::prep_km(static_cast<int32_t*>(gend), static_cast<int32_t*>(ck), K, static_cast<double*>(Gk), nullptr, s));
  if (gend_out) CUDA_TRY(cudaMemcpyAsync(gend_out, gend, 4 * (size_t)K, cudaMemcpyDefault, s));
  if (dk_out) CUDA_TRY(cudaMemcpyAsync(dk_out, dk, 4 * (size_t)K, cudaMemcpyDefault, s));
  if (Gk_out) CUDA_TRY(cudaMemcpyAsync(Gk_out, Gk, 8 * (size_t)K, cudaMemcpyDefault, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return SURV_OK;
}

int cox_lambda_max(const surv_data* data, const double* penalty_factor, double* lambda_max, void* stream) {
  return lambda_max_impl(data, penalty_factor, lambda_max, stream);
}

int cox_cv_path(const surv_data* data, const int8_t* fold_id, int32_t nfolds, const double* lambdas,
                int32_t nlambda, const surv_opts* opts, int32_t ctas_per_fit, double* beta_out, double* heldout,
                double* cv_mean, int32_t* sweeps, surv_cv_info* info) {
  return cv_impl(data, fold_id, nfolds, lambdas, nlambda, opts, ctas_per_fit, beta_out, heldout, cv_mean, sweeps,
                 info);
}

const char* surv_strerror(int code) {
  switch (code) {
    case SURV_OK: return "ok";
    case SURV_W_NOT_CONVERGED: return "not converged";
    case SURV_E_INVALID: return "invalid argument";
    case SURV_E_UNSORTED: return "time not sorted in decreasing order";
    case SURV_E_STATUS: return "invalid status code";
    case SURV_E_NONFINITE: return "non-finite value";
    case SURV_E_NO_EVENTS: return "no events";
    case SURV_E_CUDA: return "CUDA error";
    case SURV_E_DEVICE_TIMEOUT: return "device wait timed out";
    case SURV_E_NOMEM: return "out of device memory";
    case SURV_E_INDEX: return "malformed CSC indices";
    default: return "unknown code";
  }
}

const char* surv_last_error(void) { return g_last_error; }

int surv_version(void) { return 100; }

}  // extern "C"
