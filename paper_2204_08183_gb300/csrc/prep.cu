// Once-per-fit preparation kernels (the "precomputed" parts of Section 2.7):
// input validation, the Breslow tie-group table (group ends e_k and event
// counts d_k), the Kaplan-Meier censoring survival G(t_k) and the competing
// weights W_r = I(status_r = 2) / G(y_r) (Section 2.2), delta^T X_j (the
// constant first term of Eq. cox_g), the warp/row partition tables of the
// persistent kernel, and eta = X beta for a warm start.
//
// Integer work (ends, counts) is exact; G(t_k) is a sequential FP64 product
// from the smallest time upward in a single thread, so its rounding follows
// one fixed order.
#include <climits>
#include <cuda_bf16.h>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace survgpu {
namespace {

constexpr int kPrepThreads = 256;

inline unsigned grid_for(int64_t count, int threads, unsigned cap = 65535u * 32u) {
  int64_t g = (count + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > (int64_t)cap) g = cap;
  return (unsigned)g;
}

__global__ void k_check_times(const int32_t* time, const int8_t* status, int64_t n, int model, unsigned* perr) {
  unsigned bits = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i + 1 < n && time[i] < time[i + 1]) bits |= PREP_UNSORTED;
    const int s = status[i];
    if (s < 0 || s > (model == 1 ? 2 : 1)) bits |= PREP_STATUS;
  }
  if (bits) atomicOr(perr, bits);
}

template <typename T>
__global__ void k_check_csc(const int64_t* col_ptr, const int32_t* row_idx, const T* values, int64_t p,
                            int64_t n, unsigned* perr) {
  unsigned bits = 0;
  for (int64_t j = blockIdx.y; j < p; j += gridDim.y) {
    const int64_t a = col_ptr[j], b = col_ptr[j + 1];
    for (int64_t i = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b;
         i += (int64_t)gridDim.x * blockDim.x) {
      const int32_t r = row_idx[i];
      if (r < 0 || r >= n) bits |= PREP_INDEX;
      if (i > a && row_idx[i - 1] >= r) bits |= PREP_INDEX;
      if (values && !isfinite(values[i])) bits |= PREP_NONFINITE;
      if (values && values[i] != T(1)) bits |= PREP_VALUES_NOT_ONE;
    }
  }
  if (bits) atomicOr(perr, bits);
}

template <typename T>
__global__ void k_check_dense(const T* X, int64_t ld, int64_t n, int64_t p, unsigned* perr) {
  unsigned bits = 0;
  const int64_t total = n * p;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / n, i = t - j * n;
    if (!isfinite(X[j * ld + i])) bits |= PREP_NONFINITE;
  }
  if (bits) atomicOr(perr, bits);
}

__global__ void k_check_finite(const double* v, int64_t count, unsigned* perr) {
  unsigned bits = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) bits |= PREP_NONFINITE;
  if (bits) atomicOr(perr, bits);
}

// --- tie groups: i is a group end iff i == n-1 or time[i] != time[i+1]
constexpr int kEndBlock = 1024;

__device__ __forceinline__ bool is_end(const int32_t* time, int64_t n, int64_t i) {
  return i < n && (i == n - 1 || time[i] != time[i + 1]);
}

__global__ void k_count_ends(const int32_t* time, int64_t n, int32_t* blockcnt) {
  const int64_t i = (int64_t)blockIdx.x * kEndBlock + threadIdx.x;
  const int c = __syncthreads_count(is_end(time, n, i) ? 1 : 0);
  if (threadIdx.x == 0) blockcnt[blockIdx.x] = c;
}

// single block: exclusive scan of block counts in place, total into *K
__global__ void k_scan_counts(int32_t* cnt, int64_t nb, int32_t* K) {
  __shared__ int32_t s_part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t lo = t * per, hi = lo + per < nb ? lo + per : nb;
  int32_t sum = 0;
  for (int64_t b = lo; b < hi; ++b) sum += cnt[b];
  s_part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int q = 0; q < (int)blockDim.x; ++q) {
      const int32_t v = s_part[q];
      s_part[q] = run;
      run += v;
    }
    *K = run;
  }
  __syncthreads();
  int32_t run = s_part[t];
  for (int64_t b = lo; b < hi; ++b) {
    const int32_t v = cnt[b];
    cnt[b] = run;
    run += v;
  }
}

__global__ void k_write_ends(const int32_t* time, int64_t n, const int32_t* blockoff, int32_t* gend) {
  __shared__ int32_t s_w[kEndBlock / 32];
  const int64_t i = (int64_t)blockIdx.x * kEndBlock + threadIdx.x;
  const bool f = is_end(time, n, i);
  const unsigned m = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s_w[w] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int q = 0; q < kEndBlock / 32; ++q) {
      const int v = s_w[q];
      s_w[q] = run;
      run += v;
    }
  }
  __syncthreads();
  if (f) gend[blockoff[blockIdx.x] + s_w[w] + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
}

// Events (status 1) and censored (status 0) per tie group.  Each warp takes
// a chunk of kStatChunk consecutive subjects and adds the counts of every
// group segment inside it to the group's total (integer atomics: the
// result does not depend on their order).  A group spanning many chunks is
// counted by many warps, so one large group does not hold up the kernel.
constexpr int kStatChunk = 2048;
__global__ void k_group_stats(const int32_t* gend, int32_t K, const int8_t* status, int64_t n, int32_t* dk,
                              int32_t* ck, int32_t* total_events) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nchunk = (n + kStatChunk - 1) / kStatChunk;
  for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; ch < nchunk; ch += nwarp) {
    const int64_t r0 = ch * kStatChunk, r1 = min(r0 + kStatChunk, n);
    // first group whose end is at or after r0
    int lo = 0, hi = K - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)gend[mid] >= r0) hi = mid; else lo = mid + 1;
    }
    int k = lo;
    int evs = 0;
    for (int64_t pos = r0; pos < r1 && k < K; ++k) {
      const int64_t g_end = min((int64_t)gend[k], r1 - 1);
      int d = 0, c = 0;
      for (int64_t i = pos + lane; i <= g_end; i += 32) {
        const int sv = status[i];
        d += sv == 1;
        c += sv == 0;
      }
      d = __reduce_add_sync(0xffffffffu, d);
      c = __reduce_add_sync(0xffffffffu, c);
      if (lane == 0) {
        if (d) atomicAdd(dk + k, d);
        if (ck && c) atomicAdd(ck + k, c);
      }
      evs += d;
      pos = g_end + 1;
    }
    if (lane == 0 && evs) atomicAdd(total_events, evs);
  }
}

// Kaplan-Meier censoring survival (Section 2.2):
//   G(t_k) = prod_{k' >= k} f_k',  f_k' = 1 - c_k' / n_k',  n_k' = e_k' + 1
// (groups k' >= k have t_k' <= t_k).  The factors are independent: one
// thread each (k_km_factor writes them into Gk).  The product is ordered:
// up to kKmSerial groups one thread multiplies them in the order of the
// definition, k = K - 1 down to 0, exactly as a sequential loop does; above
// that the groups are cut into 1024 contiguous chunks, each thread forms
// its chunk's product, a fixed-shape suffix scan over the chunks gives each
// chunk the product of the chunks after it, and each thread walks its chunk
// downward from there.  That order is fixed (the result does not depend on
// timing) and keeps the relative error below (2 L + 12) u, L = ceil(K /
// 1024), against (K - 1) u for the sequential product.
constexpr int kKmSerial = 4096;
constexpr int kKmThreads = 1024;

__global__ void k_km_factor(const int32_t* gend, const int32_t* ck, int32_t K, double* f) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x)
    f[k] = 1.0 - (double)ck[k] / (double)((int64_t)gend[k] + 1);
}

__device__ __forceinline__ void km_put(double* Gk, float2* Gkff, int64_t k, double v) {
  Gk[k] = v;
  if (Gkff) {
    const ff q = d_to_ff(v);
    Gkff[k] = make_float2(q.hi, q.lo);
  }
}

// Gk holds the factors on entry and G(t_k) on exit (one block).
__global__ void __launch_bounds__(kKmThreads) k_km_product(int32_t K, double* Gk, float2* Gkff) {
  if (K <= kKmSerial) {
    if (threadIdx.x != 0) return;
    double acc = 1.0;
    for (int64_t k = (int64_t)K - 1; k >= 0; --k) {
      acc = acc * Gk[k];
      km_put(Gk, Gkff, k, acc);
    }
    return;
  }
  __shared__ double s_w[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t L = ((int64_t)K + kKmThreads - 1) / kKmThreads;
  const int64_t a = min((int64_t)t * L, (int64_t)K), b = min(a + L, (int64_t)K);
  double v = 1.0;
  for (int64_t k = b - 1; k >= a; --k) v = v * Gk[k];
  // inclusive suffix products over the lanes, then over the warps
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, d);
    if (lane + d < 32) v = v * u;
  }
  if (lane == 0) s_w[w] = v;
  __syncthreads();
  if (w == 0) {
    double q = s_w[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const double u = __shfl_down_sync(0xffffffffu, q, d);
      if (lane + d < 32) q = q * u;
    }
    __syncwarp();
    s_w[lane] = q;
  }
  __syncthreads();
  double in_warp = __shfl_down_sync(0xffffffffu, v, 1);
  if (lane == 31) in_warp = 1.0;
  const double later_warps = w < 31 ? s_w[w + 1] : 1.0;
  double acc = later_warps * in_warp;   // product of the chunks after this one
  for (int64_t k = b - 1; k >= a; --k) {
    acc = acc * Gk[k];
    km_put(Gk, Gkff, k, acc);
  }
}

template <typename T>
__global__ void k_w2(const int32_t* gend, int32_t K, const int8_t* status, const double* Gk, T* w2) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < K; k += nwarp) {
    const int64_t a = k == 0 ? 0 : (int64_t)gend[k - 1] + 1, b = gend[k];
    const T inv = (T)(1.0 / Gk[k]);
    for (int64_t i = a + lane; i <= b; i += 32) w2[i] = status[i] == 2 ? inv : T(0);
  }
}

template <typename T>
__device__ __forceinline__ void block_sum_store(typename AccOf<T>::type v, double* dst) {
  using A = typename AccOf<T>::type;
  __shared__ A s[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) s[w] = v;
  __syncthreads();
  if (w == 0) {
    A u;
    acc_zero(u);
    if (lane < (int)(blockDim.x >> 5)) u = s[lane];
    u = warp_sum(u);
    if (lane == 0) *dst = acc_to_d(u);
  }
}

// delta^T X_j over the nonzeros of column j (one block per column)
template <typename T>
__global__ void k_dtx_csc(const int64_t* col_ptr, const int32_t* row_idx, const T* values, const int8_t* status,
                          double* dTx) {
  using A = typename AccOf<T>::type;
  const int64_t j = blockIdx.x;
  const int64_t a = col_ptr[j], b = col_ptr[j + 1];
  const int64_t NT = blockDim.x;
  A acc;
  acc_zero(acc);
  // eight independent gathers in flight per thread
  int64_t i = a + threadIdx.x;
  for (; i + 7 * NT < b; i += 8 * NT) {
    int32_t r[8];
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      r[u] = row_idx[i + u * NT];
      v[u] = values ? values[i + u * NT] : T(1);
    }
    int8_t st[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) st[u] = status[r[u]];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (st[u] == 1) acc = acc_add_v(acc, v[u]);
  }
  for (; i < b; i += NT)
    if (status[row_idx[i]] == 1) acc = acc_add_v(acc, values ? values[i] : T(1));
  block_sum_store<T>(acc, dTx + j);
}

template <typename T>
__global__ void k_dtx_dense(const T* X, int64_t ld, int64_t n, const int8_t* status, double* dTx) {
  using A = typename AccOf<T>::type;
  const int64_t j = blockIdx.x;
  A acc;
  acc_zero(acc);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    if (status[i] == 1) acc = acc_add_v(acc, X[j * ld + i]);
  block_sum_store<T>(acc, dTx + j);
}

// first group whose end is at or after the warp's first row
__global__ void k_warp_groups(const int32_t* gend, int32_t K, int64_t n, int32_t nwarps, int64_t rows_per_warp,
                              int32_t* wk0) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g > nwarps) return;
  int64_t R = g * rows_per_warp;
  if (R > n) R = n;
  int64_t lo = 0, hi = K;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)gend[mid] < R) lo = mid + 1; else hi = mid;
  }
  wk0[g] = (int32_t)lo;
}

// entry offset (relative to col_ptr[j]) of the first nonzero at or after
// each warp's first row
__global__ void k_warp_offsets(const int64_t* col_ptr, const int32_t* row_idx, int64_t p, int64_t n,
                               int32_t nwarps, int64_t rows_per_warp, int32_t* woff) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nw1 = (int64_t)nwarps + 1;
  if (t >= p * nw1) return;
  const int64_t j = t / nw1, g = t - j * nw1;
  int64_t R = g * rows_per_warp;
  if (R > n) R = n;
  const int64_t a = col_ptr[j], b = col_ptr[j + 1];
  int64_t lo = 0, hi = b - a;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)row_idx[a + mid] < R) lo = mid + 1; else hi = mid;
  }
  woff[t] = (int32_t)lo;
}

// eta (float-float or double) and e = exp(eta)
__device__ __forceinline__ void eta_store(float2* eta, float* e, int64_t i, ff v) {
  eta[i] = make_float2(v.hi, v.lo);
  const float ev = expf(v.hi);
  e[i] = fmaf(ev, v.lo, ev);
}
__device__ __forceinline__ void eta_store(double* eta, double* e, int64_t i, double v) {
  eta[i] = v;
  e[i] = exp(v);
}

template <typename T>
__global__ void k_eta_dense(const T* X, int64_t ld, int64_t n, int64_t p, const double* beta, void* eta, T* e) {
  using A = typename AccOf<T>::type;
  using E = typename std::conditional<sizeof(T) == 4, float2, double>::type;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    A v;
    acc_zero(v);
    for (int64_t j = 0; j < p; ++j) {
      const double b = beta[j];
      if (b == 0.0) continue;
      if constexpr (sizeof(T) == 4) v = ff_add(v, ff_mul_f(d_to_ff(b), X[j * ld + i]));
      else v = v + X[j * ld + i] * b;
    }
    eta_store(reinterpret_cast<E*>(eta), e, i, v);
  }
}

template <typename T>
__global__ void k_eta_zero(int64_t n, void* eta, T* e) {
  using E = typename std::conditional<sizeof(T) == 4, float2, double>::type;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) reinterpret_cast<E*>(eta)[i] = make_float2(0.f, 0.f);
    else reinterpret_cast<E*>(eta)[i] = 0.0;
    e[i] = T(1);
  }
}

template <typename T>
__global__ void k_eta_axpy_csc(const int32_t* rows, const T* vals, int64_t nnz, double delta, void* eta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rows[i];
    const T x = vals ? vals[i] : T(1);
    if constexpr (sizeof(T) == 4) {
      float2* et = reinterpret_cast<float2*>(eta);
      const float2 q = et[r];
      const ff v = ff_add({q.x, q.y}, ff_mul_f(d_to_ff(delta), x));
      et[r] = make_float2(v.hi, v.lo);
    } else {
      double* et = reinterpret_cast<double*>(eta);
      et[r] = et[r] + x * delta;
    }
  }
}

template <typename T>
__global__ void k_eta_exp(int64_t n, const void* eta, T* e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) {
      const float2 q = reinterpret_cast<const float2*>(eta)[i];
      const float ev = expf(q.x);
      e[i] = fmaf(ev, q.y, ev);
    } else {
      e[i] = exp(reinterpret_cast<const double*>(eta)[i]);
    }
  }
}

__global__ void k_fill_f64(double* v, double value, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = value;
}

template <typename D, typename S>
__device__ __forceinline__ D to_wide(S v) { return (D)v; }
template <>
__device__ __forceinline__ float to_wide<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ double to_wide<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <typename S, typename D>
__global__ void k_convert_dense(const S* src, int64_t n, int64_t p, D* dst, int64_t ld) {
  const int64_t total = ld * p;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / ld, i = t - j * ld;
    dst[t] = i < n ? to_wide<D>(src[j * n + i]) : D(0);
  }
}

template <typename S, typename D>
__global__ void k_convert_vec(const S* src, int64_t count, D* dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (D)src[t];
}

}  // namespace

cudaError_t prep_check_times(const int32_t* time, const int8_t* status, int64_t n, int model, unsigned* perr,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_check_times<<<grid_for(n, kPrepThreads, 4096), kPrepThreads, 0, s>>>(time, status, n, model, perr);
  return cudaGetLastError();
}

cudaError_t prep_check_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* values, int prec, int64_t p,
                           int64_t n, unsigned* perr, cudaStream_t s) {
  if (p <= 0) return cudaSuccess;
  dim3 grid(64, (unsigned)(p < 65535 ? p : 65535));
  if (prec == 0) k_check_csc<float><<<grid, kPrepThreads, 0, s>>>(col_ptr, row_idx, (const float*)values, p, n, perr);
  else k_check_csc<double><<<grid, kPrepThreads, 0, s>>>(col_ptr, row_idx, (const double*)values, p, n, perr);
  return cudaGetLastError();
}

cudaError_t prep_check_dense(const void* X, int prec, int64_t ld, int64_t n, int64_t p, unsigned* perr,
                             cudaStream_t s) {
  if (n <= 0 || p <= 0) return cudaSuccess;
  const unsigned g = grid_for(n * p, kPrepThreads, 8192);
  if (prec == 0) k_check_dense<float><<<g, kPrepThreads, 0, s>>>((const float*)X, ld, n, p, perr);
  else k_check_dense<double><<<g, kPrepThreads, 0, s>>>((const double*)X, ld, n, p, perr);
  return cudaGetLastError();
}

cudaError_t prep_check_finite_f64(const double* v, int64_t count, unsigned* perr, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_check_finite<<<grid_for(count, kPrepThreads, 1024), kPrepThreads, 0, s>>>(v, count, perr);
  return cudaGetLastError();
}

int64_t prep_end_blocks(int64_t n) { return (n + kEndBlock - 1) / kEndBlock; }

cudaError_t prep_count_ends(const int32_t* time, int64_t n, int32_t* blockcnt, int32_t* K_dev, cudaStream_t s) {
  const int64_t nb = prep_end_blocks(n);
  if (nb > 0) k_count_ends<<<(unsigned)nb, kEndBlock, 0, s>>>(time, n, blockcnt);
  cudaError_t st = cudaGetLastError();
  if (st != cudaSuccess) return st;
  k_scan_counts<<<1, 1024, 0, s>>>(blockcnt, nb, K_dev);
  return cudaGetLastError();
}

cudaError_t prep_write_ends(const int32_t* time, int64_t n, const int32_t* blockoff, int32_t* gend, cudaStream_t s) {
  const int64_t nb = prep_end_blocks(n);
  if (nb > 0) k_write_ends<<<(unsigned)nb, kEndBlock, 0, s>>>(time, n, blockoff, gend);
  return cudaGetLastError();
}

cudaError_t prep_group_stats(const int32_t* gend, int32_t K, const int8_t* status, int64_t n, int32_t* dk,
                             int32_t* ck, int32_t* total_events, cudaStream_t s) {
  if (K <= 0 || n <= 0) return cudaSuccess;
  cudaError_t st = cudaMemsetAsync(dk, 0, sizeof(int32_t) * (size_t)K, s);
  if (st == cudaSuccess && ck) st = cudaMemsetAsync(ck, 0, sizeof(int32_t) * (size_t)K, s);
  if (st != cudaSuccess) return st;
  const int64_t nchunk = (n + kStatChunk - 1) / kStatChunk;
  k_group_stats<<<grid_for(nchunk * 32, kPrepThreads, 16384), kPrepThreads, 0, s>>>(gend, K, status, n, dk, ck,
                                                                                  total_events);
  return cudaGetLastError();
}

cudaError_t prep_km(const int32_t* gend, const int32_t* ck, int32_t K, double* Gk, float2* Gkff, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  k_km_factor<<<grid_for(K, kPrepThreads, 16384), kPrepThreads, 0, s>>>(gend, ck, K, Gk);
  cudaError_t st = cudaGetLastError();
  if (st != cudaSuccess) return st;
  k_km_product<<<1, kKmThreads, 0, s>>>(K, Gk, Gkff);
  return cudaGetLastError();
}

cudaError_t prep_w2(const int32_t* gend, int32_t K, const int8_t* status, const double* Gk, void* w2, int prec,
                    cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  const unsigned g = grid_for((int64_t)K * 32, kPrepThreads, 16384);
  if (prec == 0) k_w2<float><<<g, kPrepThreads, 0, s>>>(gend, K, status, Gk, (float*)w2);
  else k_w2<double><<<g, kPrepThreads, 0, s>>>(gend, K, status, Gk, (double*)w2);
  return cudaGetLastError();
}

cudaError_t prep_dtx_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* values, int prec,
                         const int8_t* status, int64_t p, double* dTx, cudaStream_t s) {
  if (p <= 0) return cudaSuccess;
  if (prec == 0)
    k_dtx_csc<float><<<(unsigned)p, 1024, 0, s>>>(col_ptr, row_idx, (const float*)values, status, dTx);
  else
    k_dtx_csc<double><<<(unsigned)p, 1024, 0, s>>>(col_ptr, row_idx, (const double*)values, status, dTx);
  return cudaGetLastError();
}

cudaError_t prep_dtx_dense(const void* X, int prec, int64_t ld, int64_t n, const int8_t* status, int64_t p,
                           double* dTx, cudaStream_t s) {
  if (p <= 0) return cudaSuccess;
  if (prec == 0) k_dtx_dense<float><<<(unsigned)p, 1024, 0, s>>>((const float*)X, ld, n, status, dTx);
  else k_dtx_dense<double><<<(unsigned)p, 1024, 0, s>>>((const double*)X, ld, n, status, dTx);
  return cudaGetLastError();
}

cudaError_t prep_warp_groups(const int32_t* gend, int32_t K, int64_t n, int32_t nwarps, int64_t rows_per_warp,
                             int32_t* wk0, cudaStream_t s) {
  k_warp_groups<<<grid_for((int64_t)nwarps + 1, kPrepThreads), kPrepThreads, 0, s>>>(gend, K, n, nwarps,
                                                                                       rows_per_warp, wk0);
  return cudaGetLastError();
}

cudaError_t prep_warp_offsets(const int64_t* col_ptr, const int32_t* row_idx, int64_t p, int64_t n, int32_t nwarps,
                              int64_t rows_per_warp, int32_t* woff, cudaStream_t s) {
  const int64_t total = p * ((int64_t)nwarps + 1);
  if (total <= 0) return cudaSuccess;
  k_warp_offsets<<<grid_for(total, kPrepThreads, 1u << 30), kPrepThreads, 0, s>>>(col_ptr, row_idx, p, n, nwarps,
                                                                                   rows_per_warp, woff);
  return cudaGetLastError();
}

cudaError_t prep_eta_dense(const void* X, int prec, int64_t ld, int64_t n, int64_t p, const double* beta, void* eta,
                           void* e, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n, kPrepThreads, 8192);
  if (prec == 0) k_eta_dense<float><<<g, kPrepThreads, 0, s>>>((const float*)X, ld, n, p, beta, eta, (float*)e);
  else k_eta_dense<double><<<g, kPrepThreads, 0, s>>>((const double*)X, ld, n, p, beta, eta, (double*)e);
  return cudaGetLastError();
}

cudaError_t prep_eta_zero(int prec, int64_t n, void* eta, void* e, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n, kPrepThreads, 8192);
  if (prec == 0) k_eta_zero<float><<<g, kPrepThreads, 0, s>>>(n, eta, (float*)e);
  else k_eta_zero<double><<<g, kPrepThreads, 0, s>>>(n, eta, (double*)e);
  return cudaGetLastError();
}

cudaError_t prep_eta_axpy_csc(const int64_t* col_ptr, const int32_t* row_idx, const void* values, int prec,
                              int64_t j, int64_t nnz_j, double delta, void* eta, cudaStream_t s) {
  (void)col_ptr;
  if (nnz_j <= 0) return cudaSuccess;
  (void)j;
  const unsigned g = grid_for(nnz_j, kPrepThreads, 8192);
  if (prec == 0) k_eta_axpy_csc<float><<<g, kPrepThreads, 0, s>>>(row_idx, (const float*)values, nnz_j, delta, eta);
  else k_eta_axpy_csc<double><<<g, kPrepThreads, 0, s>>>(row_idx, (const double*)values, nnz_j, delta, eta);
  return cudaGetLastError();
}

cudaError_t prep_eta_exp(int prec, int64_t n, const void* eta, void* e, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n, kPrepThreads, 8192);
  if (prec == 0) k_eta_exp<float><<<g, kPrepThreads, 0, s>>>(n, eta, (float*)e);
  else k_eta_exp<double><<<g, kPrepThreads, 0, s>>>(n, eta, (double*)e);
  return cudaGetLastError();
}

cudaError_t prep_fill_f64(double* v, double value, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_fill_f64<<<grid_for(count, kPrepThreads, 1024), kPrepThreads, 0, s>>>(v, value, count);
  return cudaGetLastError();
}

cudaError_t prep_convert_dense(const void* src, int src_dtype, int64_t n, int64_t p, void* dst, int prec, int64_t ld,
                               cudaStream_t s) {
  if (ld * p <= 0) return cudaSuccess;
  const unsigned g = grid_for(ld * p, kPrepThreads, 16384);
  if (src_dtype == 0 && prec == 0) k_convert_dense<float, float><<<g, kPrepThreads, 0, s>>>((const float*)src, n, p, (float*)dst, ld);
  else if (src_dtype == 0) k_convert_dense<float, double><<<g, kPrepThreads, 0, s>>>((const float*)src, n, p, (double*)dst, ld);
  else if (src_dtype == 2 && prec == 0)
    k_convert_dense<__nv_bfloat16, float><<<g, kPrepThreads, 0, s>>>((const __nv_bfloat16*)src, n, p, (float*)dst, ld);
  else if (src_dtype == 2)
    k_convert_dense<__nv_bfloat16, double><<<g, kPrepThreads, 0, s>>>((const __nv_bfloat16*)src, n, p, (double*)dst, ld);
  else if (prec == 0) k_convert_dense<double, float><<<g, kPrepThreads, 0, s>>>((const double*)src, n, p, (float*)dst, ld);
  else k_convert_dense<double, double><<<g, kPrepThreads, 0, s>>>((const double*)src, n, p, (double*)dst, ld);
  return cudaGetLastError();
}

cudaError_t prep_convert_vec(const void* src, int src_dtype, int64_t count, void* dst, int prec, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const unsigned g = grid_for(count, kPrepThreads, 16384);
  if (src_dtype == 0 && prec == 0) k_convert_vec<float, float><<<g, kPrepThreads, 0, s>>>((const float*)src, count, (float*)dst);
  else if (src_dtype == 0) k_convert_vec<float, double><<<g, kPrepThreads, 0, s>>>((const float*)src, count, (double*)dst);
  else if (prec == 0) k_convert_vec<double, float><<<g, kPrepThreads, 0, s>>>((const double*)src, count, (float*)dst);
  else k_convert_vec<double, double><<<g, kPrepThreads, 0, s>>>((const double*)src, count, (double*)dst);
  return cudaGetLastError();
}

}  // namespace survgpu
