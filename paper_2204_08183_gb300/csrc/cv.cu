// Kernels of the cross-validated penalty path (Section 2.8) around the
// batched CCD schedule of ccd_graph.cu, and of the L1 path's starting
// strength lambda_max:
//
//   k_cv_check_folds   fold ids in range
//   k_cv_dk            per fold: events d_k of each tie group outside the fold
//   k_cv_dtx_*         per fold: delta^T X_j over the subjects outside it
//   k_cv_init          per fit: eta = 0, e = 1 outside the fold, 0 inside
//   k_cv_heldout       per fit: log partial likelihood of the fold's own
//                      subjects on their own risk sets at the fit's beta
//   k_cv_select        mean held-out score per lambda and its first maximum
//   k_lmax_*           lambda_max = max_j |l'_j(0)| / pf_j (Cox)
//
// Fits are numbered f = l * nfolds + k (lambda l, fold k).  Every sum runs in
// a fixed order, so results do not depend on timing.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace survgpu {
namespace {

constexpr int kCvThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kRowsPerThread = 4;

inline unsigned grid_for(int64_t count, int threads, int64_t cap = 65535) {
  int64_t g = (count + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

__global__ void k_cv_check_folds(const int8_t* fold_id, int64_t n, int nfolds, unsigned* perr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int f = fold_id[i];
    if (f < 0 || f >= nfolds) atomicOr(perr, PREP_FOLD);
  }
}

// one warp per tie group, fold = blockIdx.y: events (status 1) of the group
// whose subject is outside the fold (exact integer counts)
__global__ void k_cv_dk(const int32_t* gend, int32_t K, const int8_t* status, const int8_t* fold_id, int32_t* dk,
                        int32_t* events) {
  const int fold = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < K; k += nwarp) {
    const int64_t a = k == 0 ? 0 : (int64_t)gend[k - 1] + 1, b = gend[k];
    int d = 0;
    for (int64_t i = a + lane; i <= b; i += 32) d += (status[i] == 1 && fold_id[i] != fold);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if (lane == 0) {
      dk[(size_t)fold * K + k] = d;
      if (d) atomicAdd(events + fold, d);
    }
  }
}

template <typename A>
__device__ __forceinline__ A block_sum(A v) {
  __shared__ A s[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();  // s may hold the previous call's values
  if (lane == 0) s[w] = v;
  __syncthreads();
  A u;
  acc_zero(u);
  if (lane < (int)(blockDim.x >> 5)) u = s[lane];
  return warp_sum(u);
}

// delta^T X_j over the subjects outside fold blockIdx.y (block per column)
template <typename T>
__global__ void k_cv_dtx_csc(const int64_t* col_ptr, const int32_t* row_idx, const T* values, const int8_t* status,
                             const int8_t* fold_id, int64_t p, double* dTx) {
  using A = typename AccOf<T>::type;
  const int fold = blockIdx.y;
  const int64_t j = blockIdx.x;
  const int64_t a = col_ptr[j], b = col_ptr[j + 1];
  A acc;
  acc_zero(acc);
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
    const int r = row_idx[i];
    if (status[r] == 1 && fold_id[r] != fold) acc = acc_add_v(acc, values ? values[i] : T(1));
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) dTx[(size_t)fold * p + j] = acc_to_d(acc);
}

template <typename T>
__global__ void k_cv_dtx_dense(const T* X, int64_t ld, int64_t n, const int8_t* status, const int8_t* fold_id,
                               int64_t p, double* dTx) {
  using A = typename AccOf<T>::type;
  const int fold = blockIdx.y;
  const int64_t j = blockIdx.x;
  A acc;
  acc_zero(acc);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    if (status[i] == 1 && fold_id[i] != fold) acc = acc_add_v(acc, X[j * ld + i]);
  acc = block_sum(acc);
  if (threadIdx.x == 0) dTx[(size_t)fold * p + j] = acc_to_d(acc);
}

// eta = 0 and e = 1 (0 for the subjects of the fit's fold), fit = blockIdx.y
template <typename T, typename E>
__global__ void k_cv_init(int64_t n, int64_t fit_n, const int8_t* fold_id, int nfolds, T* e, E* eta) {
  const int f = blockIdx.y;
  const int fold = f % nfolds;
  T* ef = e + (size_t)f * fit_n;
  E* etaf = eta + (size_t)f * fit_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ef[i] = fold_id[i] == fold ? T(0) : T(1);
    etaf[i] = E{};
  }
}

// exp(eta) of a held-out subject in the fit's working precision (the same
// rounding as the fit's own e) and eta as a double
__device__ __forceinline__ float held_exp(float2 q) {
  const float ev = expf(q.x);
  return fmaf(ev, q.y, ev);
}
__device__ __forceinline__ double held_exp(double q) { return exp(q); }
__device__ __forceinline__ double eta_d(float2 q) { return (double)q.x + (double)q.y; }
__device__ __forceinline__ double eta_d(double q) { return q; }

// Held-out score of fit blockIdx.x (fold k = f % nfolds): Breslow log
// partial likelihood of the fold's subjects on their own risk sets,
//   sum_{i in fold, delta_i = 1} eta_i - sum_g dh_g log den_g,
//   den_g = sum_{r <= e_g, r in fold} exp(eta_r),
// dh_g = events of group g inside the fold = d_g(all) - d_g(outside fold).
// One CTA per fit: rows in tiles of kScanThreads * kRowsPerThread, a block
// scan of the held-out exp(eta) and of the group-end count per tile gives
// den_g at each group end (stored to den[f][g]); a second loop takes the
// FP64 logs.
template <typename T, typename E>
__global__ void __launch_bounds__(kScanThreads) k_cv_heldout(int64_t n, int64_t fit_n, const int32_t* time,
                                                              const int8_t* status,
                                                              const int8_t* fold_id, int nfolds, const E* eta_all,
                                                              const int32_t* dk_all, const int32_t* dk_fold,
                                                              int32_t K, double* den_all, double* heldout) {
  using A = typename AccOf<T>::type;
  __shared__ A s_ws[32];
  __shared__ int s_wc[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int f = blockIdx.x;
  const int fold = f % nfolds;
  const E* eta = eta_all + (size_t)f * fit_n;
  double* den = den_all + (size_t)f * K;
  A carry;
  acc_zero(carry);
  int carry_c = 0;
  double lin = 0.0;
  constexpr int R = kRowsPerThread;
  for (int64_t base = 0; base < n; base += (int64_t)kScanThreads * R) {
    const int64_t r0 = base + (int64_t)tid * R;
    A s[R];
    int c[R];
    bool end[R];
    A run;
    acc_zero(run);
    int runc = 0;
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int64_t i = r0 + u;
      T ev = T(0);
      end[u] = false;
      if (i < n) {
        end[u] = (i + 1 == n) || time[i + 1] != time[i];
        if (fold_id[i] == fold) {
          const E q = eta[i];
          ev = held_exp(q);
          if (status[i] == 1) lin += eta_d(q);
        }
      }
      run = acc_add_v(run, ev);
      s[u] = run;
      c[u] = runc;  // group ends before row i inside this thread's rows
      runc += end[u] ? 1 : 0;
    }
    // block exclusive scan of the thread totals (sum and end count)
    A incl = warp_inclusive_scan(run, lane);
    int inclc = runc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inclc, d);
      if (lane >= d) inclc += v;
    }
    __syncthreads();  // the previous tile's readers of s_ws are done
    if (lane == 31) {
      s_ws[w] = incl;
      s_wc[w] = inclc;
    }
    __syncthreads();
    A woff, tile_tot;
    acc_zero(woff);
    acc_zero(tile_tot);
    int woffc = 0, tile_c = 0;
    for (int q = 0; q < kScanThreads / 32; ++q) {
      if (q < w) {
        woff = acc_add(woff, s_ws[q]);
        woffc += s_wc[q];
      }
      tile_tot = acc_add(tile_tot, s_ws[q]);
      tile_c += s_wc[q];
    }
    // prefix before this thread's rows: carry + warps before + lanes before
    A ex = shfl_up(incl, 1);
    int exc = __shfl_up_sync(0xffffffffu, inclc, 1);
    if (lane == 0) {
      acc_zero(ex);
      exc = 0;
    }
    const A base_s = acc_add(acc_add(carry, woff), ex);
    const int base_c = carry_c + woffc + exc;
#pragma unroll
    for (int u = 0; u < R; ++u)
      if (end[u]) den[base_c + c[u]] = acc_to_d(acc_add(base_s, s[u]));
    carry = acc_add(carry, tile_tot);
    carry_c += tile_c;
  }
  __syncthreads();  // den[] of every thread written
  double acc = 0.0;
  for (int k = tid; k < K; k += kScanThreads) {
    const int dh = dk_all[k] - dk_fold[(size_t)fold * K + k];
    if (dh > 0) acc += (double)dh * log(den[k]);
  }
  double v = block_sum(lin - acc);
  if (tid == 0) heldout[f] = v;
}

// cv_mean[l] = mean over folds of heldout[l * nfolds + k] (fixed order) and
// the first l with the largest mean
__global__ void k_cv_select(const double* heldout, int nlambda, int nfolds, double* cv_mean, int32_t* best) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int b = 0;
  double bv = 0.0;
  for (int l = 0; l < nlambda; ++l) {
    double s = 0.0;
    for (int k = 0; k < nfolds; ++k) s += heldout[(size_t)l * nfolds + k];
    const double m = s / (double)nfolds;
    cv_mean[l] = m;
    if (l == 0 || m > bv) {
      bv = m;
      b = l;
    }
  }
  *best = b;
}

// ---------------------------------------------------------------- lambda_max
// Lambda_k = sum_{k' >= k} d_k' / (e_k' + 1): at beta = 0 every e_r = 1, so
// the risk set of group k' (subjects 0..e_k') has e_k' + 1 members.  One CTA,
// groups taken from the last one down in chunks of the block size (FP64).
__global__ void __launch_bounds__(kScanThreads) k_lmax_lambda(const int32_t* gend, const int32_t* dk, int32_t K,
                                                               double* lam) {
  __shared__ double s_w[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double carry = 0.0;
  for (int64_t base = 0; base < K; base += kScanThreads) {
    const int64_t k = (int64_t)K - 1 - (base + tid);
    const double v = k >= 0 ? (double)dk[k] / ((double)gend[k] + 1.0) : 0.0;
    const double incl = warp_inclusive_scan(v, lane);
    __syncthreads();
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    double woff = 0.0, tot = 0.0;
    for (int q = 0; q < kScanThreads / 32; ++q) {
      if (q < w) woff += s_w[q];
      tot += s_w[q];
    }
    if (k >= 0) lam[k] = carry + woff + incl;
    carry += tot;
  }
}

// r_i = delta_i - Lambda_{g(i)}, g(i) the tie group of subject i (the first
// group whose end is at or after i)
__global__ void k_lmax_resid(const int32_t* gend, int32_t K, const int8_t* status, const double* lam, int64_t n,
                             double* r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (gend[mid] >= i) hi = mid; else lo = mid + 1;
    }
    r[i] = (status[i] == 1 ? 1.0 : 0.0) - lam[lo];
  }
}

// l'_j(0) = sum_i x_ij r_i (block per column, FP64)
template <typename T>
__global__ void k_lmax_grad_csc(const int64_t* col_ptr, const int32_t* row_idx, const T* values, const double* r,
                                double* g) {
  const int64_t j = blockIdx.x;
  const int64_t a = col_ptr[j], b = col_ptr[j + 1];
  double acc = 0.0;
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) acc += (values ? (double)values[i] : 1.0) * r[row_idx[i]];
  acc = block_sum(acc);
  if (threadIdx.x == 0) g[j] = acc;
}

template <typename T>
__global__ void k_lmax_grad_dense(const T* X, int64_t ld, int64_t n, const double* r, double* g) {
  const int64_t j = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += (double)X[j * ld + i] * r[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) g[j] = acc;
}

// max over penalised j of |g_j| / pf_j (pf null: all ones)
__global__ void k_lmax_max(const double* g, const double* pf, int64_t p, double* out) {
  double m = 0.0;
  for (int64_t j = threadIdx.x; j < p; j += blockDim.x) {
    const double f = pf ? pf[j] : 1.0;
    if (f > 0.0) m = fmax(m, fabs(g[j]) / f);
  }
  __shared__ double s[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if (lane == 0) s[w] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v = fmax(v, s[q]);
    *out = v;
  }
}

}  // namespace

cudaError_t cv_check_folds(const int8_t* fold_id, int64_t n, int nfolds, unsigned* perr, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_cv_check_folds<<<grid_for(n, kCvThreads, 4096), kCvThreads, 0, s>>>(fold_id, n, nfolds, perr);
  return cudaGetLastError();
}

cudaError_t cv_fold_stats(const int32_t* gend, int32_t K, const int8_t* status, const int8_t* fold_id, int nfolds,
                          int32_t* dk, int32_t* events, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  const dim3 g(grid_for((int64_t)K * 32, kCvThreads, 4096), nfolds);
  k_cv_dk<<<g, kCvThreads, 0, s>>>(gend, K, status, fold_id, dk, events);
  return cudaGetLastError();
}

cudaError_t cv_dtx(int layout, int prec, const int64_t* col_ptr, const int32_t* row_idx, const void* values,
                   int64_t ld, int64_t n, int64_t p, const int8_t* status, const int8_t* fold_id, int nfolds,
                   double* dTx, cudaStream_t s) {
  if (p <= 0) return cudaSuccess;
  const dim3 g((unsigned)p, nfolds);
  if (layout == 0) {
    if (prec == 0)
      k_cv_dtx_csc<float><<<g, kCvThreads, 0, s>>>(col_ptr, row_idx, (const float*)values, status, fold_id, p, dTx);
    else
      k_cv_dtx_csc<double><<<g, kCvThreads, 0, s>>>(col_ptr, row_idx, (const double*)values, status, fold_id, p, dTx);
  } else {
    if (prec == 0)
      k_cv_dtx_dense<float><<<g, 1024, 0, s>>>((const float*)values, ld, n, status, fold_id, p, dTx);
    else
      k_cv_dtx_dense<double><<<g, 1024, 0, s>>>((const double*)values, ld, n, status, fold_id, p, dTx);
  }
  return cudaGetLastError();
}

cudaError_t cv_init(int prec, int64_t n, int64_t fit_n, const int8_t* fold_id, int nfolds, int nfit, void* e,
                    void* eta, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 g(grid_for(n, kCvThreads, std::max<int64_t>(1, 8192 / nfit)), nfit);
  if (prec == 0)
    k_cv_init<float, float2><<<g, kCvThreads, 0, s>>>(n, fit_n, fold_id, nfolds, (float*)e, (float2*)eta);
  else
    k_cv_init<double, double><<<g, kCvThreads, 0, s>>>(n, fit_n, fold_id, nfolds, (double*)e, (double*)eta);
  return cudaGetLastError();
}

cudaError_t cv_heldout(int prec, int64_t n, int64_t fit_n, const int32_t* time, const int8_t* status, const int8_t* fold_id,
                       int nfolds, int nfit, const void* eta, const int32_t* dk_all, const int32_t* dk_fold,
                       int32_t K, double* den, double* heldout, cudaStream_t s) {
  if (prec == 0)
    k_cv_heldout<float, float2><<<nfit, kScanThreads, 0, s>>>(n, fit_n, time, status, fold_id, nfolds, (const float2*)eta,
                                                              dk_all, dk_fold, K, den, heldout);
  else
    k_cv_heldout<double, double><<<nfit, kScanThreads, 0, s>>>(n, fit_n, time, status, fold_id, nfolds, (const double*)eta,
                                                               dk_all, dk_fold, K, den, heldout);
  return cudaGetLastError();
}

cudaError_t cv_select(const double* heldout, int nlambda, int nfolds, double* cv_mean, int32_t* best,
                      cudaStream_t s) {
  k_cv_select<<<1, 32, 0, s>>>(heldout, nlambda, nfolds, cv_mean, best);
  return cudaGetLastError();
}

cudaError_t lambda_max_device(int layout, int prec, const int64_t* col_ptr, const int32_t* row_idx,
                              const void* values, int64_t ld, int64_t n, int64_t p, const int8_t* status,
                              const int32_t* gend, const int32_t* dk, int32_t K, const double* pf, double* lam,
                              double* r, double* g, double* out, cudaStream_t s) {
  k_lmax_lambda<<<1, kScanThreads, 0, s>>>(gend, dk, K, lam);
  k_lmax_resid<<<grid_for(n, kCvThreads, 8192), kCvThreads, 0, s>>>(gend, K, status, lam, n, r);
  if (layout == 0) {
    if (prec == 0) k_lmax_grad_csc<float><<<(unsigned)p, kCvThreads, 0, s>>>(col_ptr, row_idx, (const float*)values, r, g);
    else k_lmax_grad_csc<double><<<(unsigned)p, kCvThreads, 0, s>>>(col_ptr, row_idx, (const double*)values, r, g);
  } else {
    if (prec == 0) k_lmax_grad_dense<float><<<(unsigned)p, 1024, 0, s>>>((const float*)values, ld, n, r, g);
    else k_lmax_grad_dense<double><<<(unsigned)p, 1024, 0, s>>>((const double*)values, ld, n, r, g);
  }
  k_lmax_max<<<1, 1024, 0, s>>>(g, pf, p, out);
  return cudaGetLastError();
}

}  // namespace survgpu
