// loglik_grad_hess_noalloc: the one-pass gradient/Hessian entry point with all
// of its scratch carved from a fixed file-scope device array instead of
// cudaMalloc'd workspace.  The paper has no counterpart; it exists for callers
// that cannot allocate device memory (see include/survgpu.h).
//
// The array below is reserved on every GPU that loads this library, for the
// life of the process.  Host code must not use the symbol `g_scratch` as an
// address (it names a host-side shadow); the device address comes from
// cudaGetSymbolAddress, once per device, cached below.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "survgpu.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;
constexpr int64_t kMaxP = 4096;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

thread_local char g_err[256] = "";

struct Ctrl {
  unsigned perr;
  unsigned err;
  int32_t K;
  int32_t total_events;
  unsigned counters[2];
  unsigned pad[2];
  double out[survgpu::OUT_COUNT];
  unsigned long long timing[survgpu::PH_COUNT];
};

// Device address of the scratch array on the current device.  First call on a
// device resolves it (before any stream capture, see the header).
int scratch_base(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    snprintf(g_err, sizeof(g_err), "cudaGetDevice: %s", cudaGetErrorString(e));
    return SURV_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    snprintf(g_err, sizeof(g_err), "device index %d not supported", dev);
    return SURV_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(g_err, sizeof(g_err), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return SURV_E_CUDA;
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return SURV_OK;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carve {
  char* base;
  size_t used = 0;
  bool overflow = false;
  void* take(size_t bytes) {
    const size_t b = (bytes + 255) & ~size_t(255);
    if (used + b > kScratchBytes) {
      overflow = true;
      return nullptr;
    }
    void* p = base + used;
    used += b;
    return p;
  }
};

// Device memory of the current device (or managed memory, which any device
// may read).  Memory of another GPU is refused: the kernels run here.
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Host copies of beta and col_ptr (each at most kMaxP + 1 entries) for the
// calling thread: the column bounds are checked here before any kernel reads
// through them.
thread_local double g_beta_h[kMaxP];
thread_local int64_t g_colptr_h[kMaxP + 1];

int map_prep(unsigned perr) {
  if (perr & survgpu::PREP_INDEX) { snprintf(g_err, sizeof(g_err), "malformed CSC indices"); return SURV_E_INDEX; }
  if (perr & survgpu::PREP_UNSORTED) { snprintf(g_err, sizeof(g_err), "time is not non-increasing"); return SURV_E_UNSORTED; }
  if (perr & survgpu::PREP_STATUS) { snprintf(g_err, sizeof(g_err), "status code out of range"); return SURV_E_STATUS; }
  if (perr & survgpu::PREP_NONFINITE) { snprintf(g_err, sizeof(g_err), "non-finite value"); return SURV_E_NONFINITE; }
  return SURV_OK;
}

#define TRY(call)                                                                               \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      snprintf(g_err, sizeof(g_err), "%s: %s", #call, cudaGetErrorString(e_));                  \
      return SURV_E_CUDA;                                                                       \
    }                                                                                           \
  } while (0)

#define TAKE(ptr, bytes)                                                                        \
  do {                                                                                          \
    (ptr) = cv.take(bytes);                                                                     \
    if (!(ptr)) {                                                                               \
      snprintf(g_err, sizeof(g_err), "problem needs more than the %zu bytes of static scratch", \
               kScratchBytes);                                                                  \
      return SURV_E_INVALID;                                                                    \
    }                                                                                           \
  } while (0)

int run(const surv_data* d, int model, const double* beta, int32_t j, double* out_l, double* out_g, double* out_h,
        int prec, cudaStream_t s) {
  g_err[0] = '\0';
  if (!d || !beta) { snprintf(g_err, sizeof(g_err), "null data or beta"); return SURV_E_INVALID; }
  if (model != SURV_COX && model != SURV_FG) { snprintf(g_err, sizeof(g_err), "bad model"); return SURV_E_INVALID; }
  if (prec != SURV_PREC_F32C && prec != SURV_PREC_F64) { snprintf(g_err, sizeof(g_err), "bad precision"); return SURV_E_INVALID; }
  const int64_t n = d->n, p = d->p;
  if (n < 1 || p < 1 || p > kMaxP || n > 0x7fffffff || j < 0 || j >= p) {
    snprintf(g_err, sizeof(g_err), "sizes out of range (n=%lld p=%lld j=%d; p <= %lld)", (long long)n, (long long)p,
             j, (long long)kMaxP);
    return SURV_E_INVALID;
  }
  if (d->layout != SURV_CSC && d->layout != SURV_DENSE) { snprintf(g_err, sizeof(g_err), "bad layout"); return SURV_E_INVALID; }
  if (d->dtype != prec && !(d->layout == SURV_CSC && !d->values)) {
    snprintf(g_err, sizeof(g_err), "values dtype must match the precision (no conversion buffer)");
    return SURV_E_INVALID;
  }
  const bool csc = d->layout == SURV_CSC;
  if (!csc && ((uintptr_t)d->values % 16 != 0 || n % 4 != 0)) {
    snprintf(g_err, sizeof(g_err), "dense X needs a 16-byte aligned base and n divisible by 4");
    return SURV_E_INVALID;
  }
  int cur = 0;
  TRY(cudaGetDevice(&cur));
  if (!on_device(d->time, cur) || !on_device(d->status, cur) ||
      (csc && (!on_device(d->col_ptr, cur) || !on_device(d->row_idx, cur))) ||
      ((!csc || d->values) && !on_device(d->values, cur))) {
    snprintf(g_err, sizeof(g_err), "time, status and X must be arrays on the current device");
    return SURV_E_INVALID;
  }

  void* base = nullptr;
  int rc = scratch_base(&base);
  if (rc) return rc;
  Carve cv{static_cast<char*>(base)};

  int G = 0, wpc = 0;
  TRY(survgpu::ccd_grid_size(model, d->layout, prec, &G, &wpc));
  const int32_t nwarps = G * wpc;
  const int64_t nwords = (n + 31) / 32;
  const int32_t wpw = (int32_t)((nwords + nwarps - 1) / nwarps);
  const int64_t rows_per_warp = (int64_t)wpw * 32;
  const size_t tsz = prec == SURV_PREC_F32C ? 4 : 8;
  const int M = model == SURV_COX ? 3 : 6;

  // host copies of beta (the caller's beta may be host or device memory) and
  // of col_ptr, checked before any kernel indexes row_idx through it
  double* beta_h = g_beta_h;
  int64_t* colptr_h = g_colptr_h;
  TRY(cudaMemcpyAsync(beta_h, beta, 8 * (size_t)p, cudaMemcpyDefault, s));
  if (csc) TRY(cudaMemcpyAsync(colptr_h, d->col_ptr, 8 * (size_t)(p + 1), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (csc) {
    if (colptr_h[0] != 0) { snprintf(g_err, sizeof(g_err), "col_ptr[0] != 0"); return SURV_E_INDEX; }
    for (int64_t q = 0; q < p; ++q)
      if (colptr_h[q + 1] < colptr_h[q]) {
        snprintf(g_err, sizeof(g_err), "col_ptr decreases at %lld", (long long)q);
        return SURV_E_INDEX;
      }
    if (colptr_h[p] > 0x7fffffffLL) { snprintf(g_err, sizeof(g_err), "more than 2^31 - 1 nonzeros"); return SURV_E_INDEX; }
  }
  for (int64_t q = 0; q < p; ++q)
    if (!std::isfinite(beta_h[q])) { snprintf(g_err, sizeof(g_err), "non-finite beta"); return SURV_E_NONFINITE; }

  void *ctrl_v, *blockcnt, *e, *eta, *w2 = nullptr, *wk0, *woff = nullptr, *dTx, *beta_d, *width, *pen, *slots;
  TAKE(ctrl_v, sizeof(Ctrl));
  Ctrl* ctrl = static_cast<Ctrl*>(ctrl_v);
  TAKE(blockcnt, 4 * (size_t)survgpu::prep_end_blocks(n));
  TAKE(e, tsz * (size_t)n);
  TAKE(eta, 8 * (size_t)n);
  if (model == SURV_FG) TAKE(w2, tsz * (size_t)n);
  TAKE(wk0, 4 * (size_t)(nwarps + 1));
  if (csc) TAKE(woff, 4 * (size_t)p * (nwarps + 1));
  TAKE(dTx, 8 * (size_t)p);
  TAKE(beta_d, 8 * (size_t)p);
  TAKE(width, 8 * (size_t)p);
  TAKE(pen, 8 * (size_t)p);
  const size_t slot_bytes = 4 * (size_t)survgpu::kSlotWords * 2 * G;
  TAKE(slots, 2 * slot_bytes);

  // state that must start at zero: the control block (error words, counters)
  TRY(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
  const int32_t* tp = static_cast<const int32_t*>(static_cast<const void*>(d->time));
  const int8_t* sp = d->status;
  TRY(survgpu::prep_check_times(tp, sp, n, model, &ctrl->perr, s));
  if (csc) {
    TRY(survgpu::prep_check_csc(d->col_ptr, d->row_idx, d->values, prec, p, n, &ctrl->perr, s));
  } else {
    TRY(survgpu::prep_check_dense(d->values, prec, n, n, p, &ctrl->perr, s));
  }
  TRY(survgpu::prep_count_ends(tp, n, static_cast<int32_t*>(blockcnt), &ctrl->K, s));
  Ctrl hc;
  TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if ((rc = map_prep(hc.perr))) return rc;
  const int32_t K = hc.K;

  void *gend, *dk, *ck, *Gk, *Gkff, *rec;
  TAKE(gend, 4 * (size_t)K);
  TAKE(dk, 4 * (size_t)K);
  TAKE(ck, 4 * (size_t)K);
  TAKE(Gk, 8 * (size_t)K);
  TAKE(Gkff, 8 * (size_t)K);
  TAKE(rec, 8 * (size_t)K * M);

  TRY(survgpu::prep_write_ends(tp, n, static_cast<const int32_t*>(blockcnt), static_cast<int32_t*>(gend), s));
  TRY(survgpu::prep_group_stats(static_cast<int32_t*>(gend), K, sp, n, static_cast<int32_t*>(dk),
                                static_cast<int32_t*>(ck), &ctrl->total_events, s));
  if (model == SURV_FG) {
    TRY(survgpu::prep_km(static_cast<int32_t*>(gend), static_cast<int32_t*>(ck), K, static_cast<double*>(Gk),
                         static_cast<float2*>(Gkff), s));
    TRY(survgpu::prep_w2(static_cast<int32_t*>(gend), K, sp, static_cast<double*>(Gk), w2, prec, s));
  }
  if (csc) {
    TRY(survgpu::prep_dtx_csc(d->col_ptr, d->row_idx, d->values, prec, sp, p, static_cast<double*>(dTx), s));
    TRY(survgpu::prep_warp_offsets(d->col_ptr, d->row_idx, p, n, nwarps, rows_per_warp, static_cast<int32_t*>(woff), s));
  } else {
    TRY(survgpu::prep_dtx_dense(d->values, prec, n, n, sp, p, static_cast<double*>(dTx), s));
  }
  TRY(survgpu::prep_warp_groups(static_cast<int32_t*>(gend), K, n, nwarps, rows_per_warp, static_cast<int32_t*>(wk0), s));
  TRY(cudaMemcpyAsync(beta_d, beta_h, 8 * (size_t)p, cudaMemcpyHostToDevice, s));
  TRY(survgpu::prep_fill_f64(static_cast<double*>(width), 1.0, p, s));
  TRY(survgpu::prep_fill_f64(static_cast<double*>(pen), 0.0, p, s));
  bool any_beta = false;
  for (int64_t q = 0; q < p; ++q) any_beta |= beta_h[q] != 0.0;
  if (!any_beta) {
    TRY(survgpu::prep_eta_zero(prec, n, eta, e, s));
  } else if (!csc) {
    TRY(survgpu::prep_eta_dense(d->values, prec, n, n, p, static_cast<double*>(beta_d), eta, e, s));
  } else {
    TRY(survgpu::prep_eta_zero(prec, n, eta, e, s));
    for (int64_t q = 0; q < p; ++q) {
      if (beta_h[q] == 0.0) continue;
      const void* vq = d->values ? static_cast<const char*>(d->values) + tsz * (size_t)colptr_h[q] : nullptr;
      TRY(survgpu::prep_eta_axpy_csc(nullptr, d->row_idx + colptr_h[q], vq, prec, q, colptr_h[q + 1] - colptr_h[q],
                                     beta_h[q], eta, s));
    }
    TRY(survgpu::prep_eta_exp(prec, n, eta, e, s));
  }
  TRY(cudaMemsetAsync(slots, 0, 2 * slot_bytes, s));
  TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (hc.total_events <= 0) { snprintf(g_err, sizeof(g_err), "no events"); return SURV_E_NO_EVENTS; }

  survgpu::CcdParams P;
  std::memset(&P, 0, sizeof(P));
  P.n = n;
  P.ld = n;
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
  P.col_ptr = csc ? d->col_ptr : nullptr;
  P.row_idx = csc ? d->row_idx : nullptr;
  P.values = csc ? d->values : nullptr;
  P.woff = static_cast<const int32_t*>(woff);
  P.X = csc ? nullptr : d->values;
  P.e = e;
  P.eta = eta;
  P.w2 = w2;
  P.dTx = static_cast<const double*>(dTx);
  P.beta = static_cast<double*>(beta_d);
  P.width = static_cast<double*>(width);
  P.pen = static_cast<const double*>(pen);
  P.rec = rec;
  P.slot_agg = static_cast<unsigned*>(slots);
  P.slot_part = static_cast<unsigned*>(slots) + survgpu::kSlotWords * 2 * G;
  P.counters = ctrl->counters;
  P.err = &ctrl->err;
  P.out = ctrl->out;
  P.timing = ctrl->timing;
  P.penalty = 0;
  P.max_sweeps = 0;
  P.tol = 0.0;
  P.single_j = j;
  P.withhold_cta = -1;
  P.timeout_ns = 2000000000ull;
  TRY(survgpu::launch_ccd(model, d->layout, prec, P, s));
  TRY(cudaMemcpyAsync(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (hc.err != 0) {
    snprintf(g_err, sizeof(g_err), "device-side wait expired (error word 0x%x)", hc.err);
    return SURV_E_DEVICE_TIMEOUT;
  }
  if (out_l) *out_l = hc.out[survgpu::OUT_LOGLIK];
  if (out_g) *out_g = hc.out[survgpu::OUT_GRAD];
  if (out_h) *out_h = hc.out[survgpu::OUT_HESS];
  return SURV_OK;
}

}  // namespace

extern "C" {

int loglik_grad_hess_noalloc(const surv_data* data, int32_t model, const double* beta, int32_t j, double* loglik,
                             double* grad, double* hess, int32_t precision, void* stream) {
  const int rc = run(data, model, beta, j, loglik, grad, hess, precision, static_cast<cudaStream_t>(stream));
  survgpu::set_last_error_text(rc == SURV_OK ? "" : g_err);
  return rc;
}

}  // extern "C"
