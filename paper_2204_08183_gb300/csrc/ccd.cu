// Persistent cyclic-coordinate-descent kernel for the Cox and Fine-Gray
// partial likelihoods (Sections 2.4 and 2.7).
//
// One cooperative launch runs a whole fit: for every coordinate j it does
// the paper's four steps over all N subjects (arranged by decreasing time)
// and the conditional update, without returning to the host:
//
//   step 1  e = exp(eta) is kept up to date by the conditional update below;
//   step 2  the tuple scan S_pre[e], S_pre[e x_j], S_pre[e x_j^2] (Cox), plus
//           the competing-risk suffix sums of the same tuple weighted by
//           W_r = I(status_r = 2) / G(y_r) (Fine-Gray, Eqs. fg_g, fg_h);
//   step 3  the transform G = num1 / den, H = num2 / den at each tie-group
//           end (Breslow: the risk set of a tied time is read at the last
//           subject of the run);
//   step 4  the reductions delta^T G and delta^T (H - G*G) (Eqs. cox_g,
//           cox_h) and, on the first coordinate of a sweep, delta^T log den
//           for the log-likelihood;
//   then    the trust-region Newton step with the L1/L2 penalty (Section
//           2.4) and, if the step is nonzero, eta += x_j * step and
//           e = exp(eta) on the nonzeros of column j (the sparse update).
//
// Layout of the work: subjects are split into 32-row words; every warp of
// the grid owns a contiguous range of words, every CTA the union of its
// warps.  A warp streams its rows with 16-byte loads and keeps per-lane
// float-float (or double) running sums.  The scan result is needed only at
// group ends, so instead of a full scan the warp reduces its lanes at each
// group end that falls in its range and stores the warp-relative prefix.
// The CTA combines warp totals; the grid combines CTA aggregates through
// 128-byte exchange slots (one per CTA, double-buffered by epoch parity):
// every CTA reads all slots in a fixed order, so every CTA derives the same
// prefix and the same Newton step without a host round trip.  Every wait is
// bounded by a wall-clock limit and turns into an error word on expiry.
#include <cfloat>
#include <climits>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace survgpu {
namespace {

template <typename T> struct Vec;
template <> struct Vec<float> {
  static constexpr int n = 4;
  __device__ static __forceinline__ void load(const float* p, float (&v)[4]) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <> struct Vec<double> {
  static constexpr int n = 2;
  __device__ static __forceinline__ void load(const double* p, double (&v)[2]) {
    double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
};

// eta storage: float-float (float2) in the FP32 mode, double in the FP64 mode
__device__ __forceinline__ void eta_axpy(float2* eta, float* e, int64_t i, float x, ff delta) {
  float2 q = eta[i];
  ff v = ff_add({q.x, q.y}, ff_mul_f(delta, x));
  eta[i] = make_float2(v.hi, v.lo);
  float ev = expf(v.hi);
  e[i] = fmaf(ev, v.lo, ev);  // exp(hi + lo) to first order in lo
}
__device__ __forceinline__ void eta_axpy(double* eta, double* e, int64_t i, double x, double delta) {
  double v = eta[i] + x * delta;
  eta[i] = v;
  e[i] = exp(v);
}

// Slot (de)serialisation of accumulators: 2 words each.
__device__ __forceinline__ void put_acc(unsigned* w, ff a) {
  w[0] = __float_as_uint(a.hi);
  w[1] = __float_as_uint(a.lo);
}
__device__ __forceinline__ void put_acc(unsigned* w, double a) {
  unsigned long long b = __double_as_longlong(a);
  w[0] = (unsigned)(b & 0xffffffffull);
  w[1] = (unsigned)(b >> 32);
}
template <typename A> __device__ __forceinline__ A get_acc(const unsigned* w);
template <> __device__ __forceinline__ ff get_acc<ff>(const unsigned* w) {
  return {__uint_as_float(__ldcg(w)), __uint_as_float(__ldcg(w + 1))};
}
template <> __device__ __forceinline__ double get_acc<double>(const unsigned* w) {
  unsigned long long lo = __ldcg(w), hi = __ldcg(w + 1);
  return __longlong_as_double((long long)(lo | (hi << 32)));
}

__device__ __forceinline__ ff acc_from_d(double d, ff*) { return d_to_ff(d); }
__device__ __forceinline__ double acc_from_d(double d, double*) { return d; }
__device__ __forceinline__ ff acc_div(ff a, ff b) { return ff_div(a, b); }
__device__ __forceinline__ double acc_div(double a, double b) { return a / b; }
__device__ __forceinline__ ff acc_mul(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ double acc_mul(double a, double b) { return a * b; }
__device__ __forceinline__ ff acc_scale(ff a, int d) { return ff_mul_f(a, (float)d); }
__device__ __forceinline__ double acc_scale(double a, int d) { return a * (double)d; }

// Grid exchange: every CTA writes its payload slot, then thread 0 fences and
// adds 1 to the exchange counter; waiters poll the counter with relaxed loads
// until it reaches `target` (= exchanges so far x G) and fence once before
// reading the payloads through L2.  A counter costs one L2 atomic per CTA and
// one polled word, which measured faster on GB300 than polling one flag per
// CTA.  The wait is bounded by limit_ns.
__device__ __forceinline__ void exchange_arrive(unsigned* counter) {
  __threadfence();
  atomicAdd(counter, 1u);
}

__device__ __forceinline__ bool exchange_wait(const unsigned* counter, unsigned target, unsigned* err,
                                              uint64_t limit_ns) {
  const int lane = threadIdx.x & 31;
  uint64_t t0 = 0;
  bool timed = false;
  for (;;) {
    unsigned v = 0, bad = 0;
    if (lane == 0) {
      asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
      bad = ld_volatile(err);
    }
    v = __shfl_sync(0xffffffffu, v, 0);
    bad = __shfl_sync(0xffffffffu, bad, 0);
    if (v >= target) break;
    if (bad) return false;
    if (!timed) { t0 = global_ns(); timed = true; }
    if (global_ns() - t0 > limit_ns) {
      if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
      return false;
    }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return true;
}

// Newton step on g = l + pi for one coordinate (Section 2.4); grad, hess are
// the log-likelihood derivatives.  Mirrors the CPU reading exactly.
__device__ double newton_step(double b, double grad, double hess, int penalty, double lam) {
  double h = -hess;
  if (!(h > 0.0)) return 0.0;
  if (penalty == 0) return grad / h;
  if (penalty == 2) return (grad - lam * b) / (h + lam);
  // L1
  if (b == 0.0) {
    if (grad > lam) return (grad - lam) / h;
    if (grad < -lam) return (grad + lam) / h;
    return 0.0;
  }
  double s = b > 0.0 ? 1.0 : -1.0;
  double step = (grad - lam * s) / h;
  double nb = b + step;
  bool keeps_sign = s > 0.0 ? (nb > 0.0) : (nb < 0.0);
  if (!keeps_sign) step = -b;
  return step;
}

template <int MODEL, int LAYOUT, typename T>
struct Cfg {
  static constexpr int M = MODEL == 0 ? 3 : 6;              // tuple components
  static constexpr int VEC = Vec<T>::n;                      // rows per 16-byte load
  static constexpr int U = LAYOUT == 0 ? 8 : 4;              // loads per lane per tile
  static constexpr int TILE = 32 * U * VEC;                  // rows per warp tile
  // components produced by the dense row pass
  static constexpr int ND = LAYOUT == 1 ? M : (MODEL == 0 ? 1 : 2);
  // components produced by the sparse (CSC entry) pass
  static constexpr int NS = LAYOUT == 1 ? 0 : (MODEL == 0 ? 2 : 4);
  // threads per CTA the kernel is compiled for: 1024 (64 registers) where that
  // does not spill, else 512 (128 registers)
  static constexpr int MAXT = (MODEL == 0 && sizeof(T) == 4) ? 1024 : 512;
  __device__ static constexpr int dmap(int d) { return LAYOUT == 1 ? d : (d == 0 ? 0 : 3); }
  __device__ static constexpr int smap(int s) { return s < 2 ? 1 + s : 4 + (s - 2); }
};

// Value of dense component d for one row: e, e x, e x^2, w e, w e x, w e x^2
template <int MODEL, int LAYOUT, typename T>
__device__ __forceinline__ T dense_comp(int d, T e, T x, T w) {
  using C = Cfg<MODEL, LAYOUT, T>;
  const int m = C::dmap(d);
  T v = e;
  if (m == 1 || m == 2 || m == 4 || m == 5) v = v * x;
  if (m == 2 || m == 5) v = v * x;
  if (m >= 3) v = v * w;
  return v;
}

template <int MODEL, int LAYOUT, typename T>
__global__ void __launch_bounds__(Cfg<MODEL, LAYOUT, T>::MAXT, 1) ccd_kernel(const __grid_constant__ CcdParams P) {
  using A = typename AccOf<T>::type;
  using C = Cfg<MODEL, LAYOUT, T>;
  constexpr int M = C::M;
  constexpr int VEC = C::VEC;
  constexpr int U = C::U;
  constexpr int TILE = C::TILE;
  constexpr int ND = C::ND;
  constexpr int NS = C::NS;

  __shared__ A s_wtot[kMaxWarpsPerCta][M];
  __shared__ A s_woff[kMaxWarpsPerCta][M];
  __shared__ A s_T[M];
  __shared__ A s_tot[M];
  __shared__ A s_red[kMaxWarpsPerCta][2];
  __shared__ double s_redl[kMaxWarpsPerCta];
  __shared__ double s_scal[8];
  __shared__ int s_flag[2];

  const int tid = threadIdx.x;
  const int WPC = P.wpc;
  const int NT = 32 * WPC;
  const int lane = tid & 31;
  const int w = tid >> 5;
  const int c = blockIdx.x;
  const int G = P.G;
  const int64_t n = P.n;
  const int64_t nwords = (n + 31) >> 5;
  const int gw = c * WPC + w;
  const int64_t word_lo = min((int64_t)gw * P.wpw, nwords);
  const int64_t word_hi = min(word_lo + P.wpw, nwords);
  const int64_t row_lo = word_lo * 32;
  const int64_t row_hi = min(word_hi * 32, n);
  const int64_t cta_row_lo = min((int64_t)c * WPC * P.wpw, nwords) * 32;
  const int64_t cta_row_hi = min(min((int64_t)(c + 1) * WPC * P.wpw, nwords) * 32, n);
  const int k_lo = P.wk0[gw], k_hi = P.wk0[gw + 1];
  const int kc_lo = P.wk0[c * WPC], kc_hi = P.wk0[(c + 1) * WPC];

  const T* e = reinterpret_cast<const T*>(P.e);
  const T* w2 = reinterpret_cast<const T*>(P.w2);
  A* rec = reinterpret_cast<A*>(P.rec);
  const int nw1 = P.nwarps + 1;

  unsigned epoch = P.epoch0;
  int sweep = 0;
  double f_prev = 0.0, f_prev2 = 0.0, ll_last = 0.0;
  int converged = 0;
  long long eta_updates = 0, passes = 0;
  const bool single = P.single_j >= 0;

  for (;;) {
    bool finished = false;
    for (int jj = 0; jj < P.p && !finished; ++jj) {
      const int j = single ? P.single_j : jj;
      const bool eval = single || jj == 0;
      ++epoch;
      ++passes;
      const int par = epoch & 1;
      if (ld_volatile(P.err) != 0u) { finished = true; break; }
      // beta_j and Delta_j are read before this CTA publishes anything for
      // this coordinate: CTA 0 rewrites them only after exchange #2, which
      // needs every CTA's partial.  L2 loads: the writer is another SM.
      const double bj = __ldcg(P.beta + j);
      const double wj = __ldcg(P.width + j);

      // ------------------------------------------------ step 2: warp pass
      A tot[M];
#pragma unroll
      for (int m = 0; m < M; ++m) acc_zero(tot[m]);
      {
        // dense part: rows [row_lo, row_hi) in tiles of TILE rows
        A acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc_zero(acc[d]);
        int kn = k_lo;
        int64_t next_end = kn < k_hi ? (int64_t)P.gend[kn] : LLONG_MAX;
        const T* xcol = LAYOUT == 1 ? reinterpret_cast<const T*>(P.X) + (size_t)j * P.ld : nullptr;
        for (int64_t t0 = row_lo; t0 < row_hi; t0 += TILE) {
          T ev[U][VEC], xv[U][VEC], wv[U][VEC];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int64_t r = t0 + (int64_t)(lane + 32 * u) * VEC;
            if (r + VEC <= row_hi) {
              Vec<T>::load(e + r, ev[u]);
              if (LAYOUT == 1) Vec<T>::load(xcol + r, xv[u]);
              if (MODEL == 1) Vec<T>::load(w2 + r, wv[u]);
            } else {
#pragma unroll
              for (int q = 0; q < VEC; ++q) {
                const bool in = r + q < row_hi;
                ev[u][q] = in ? e[r + q] : T(0);
                xv[u][q] = (LAYOUT == 1 && in) ? xcol[r + q] : T(0);
                wv[u][q] = (MODEL == 1 && in) ? w2[r + q] : T(0);
              }
            }
          }
          const int64_t t_end = min(t0 + (int64_t)TILE, row_hi);
          // group ends inside this tile: warp-relative prefix at each end
          while (next_end < t_end) {
#pragma unroll
            for (int d = 0; d < ND; ++d) {
              T part = T(0);
#pragma unroll
              for (int u = 0; u < U; ++u)
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                  const int64_t r = t0 + (int64_t)(lane + 32 * u) * VEC + q;
                  if (r <= next_end) part += dense_comp<MODEL, LAYOUT, T>(d, ev[u][q], xv[u][q], wv[u][q]);
                }
              A pref = warp_sum(acc_add_v(acc[d], part));
              if (lane == 0) rec[(size_t)kn * M + C::dmap(d)] = pref;
            }
            ++kn;
            next_end = kn < k_hi ? (int64_t)P.gend[kn] : LLONG_MAX;
          }
          // tile sums (pairwise within the lane) into the running sums
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            T su[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              T a0 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][0], xv[u][0], wv[u][0]);
              T a1 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][1], xv[u][1], wv[u][1]);
              if (VEC == 4) {
                T a2 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][VEC > 2 ? 2 : 0], xv[u][VEC > 2 ? 2 : 0],
                                                    wv[u][VEC > 2 ? 2 : 0]);
                T a3 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][VEC > 3 ? 3 : 0], xv[u][VEC > 3 ? 3 : 0],
                                                    wv[u][VEC > 3 ? 3 : 0]);
                su[u] = (a0 + a1) + (a2 + a3);
              } else {
                su[u] = a0 + a1;
              }
            }
#pragma unroll
            for (int s = 1; s < U; s <<= 1)
#pragma unroll
              for (int u = 0; u + s < U; u += 2 * s) su[u] += su[u + s];
            acc[d] = acc_add_v(acc[d], su[0]);
          }
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) tot[C::dmap(d)] = warp_sum(acc[d]);
      }
      if (LAYOUT == 0 && NS > 0) {
        // sparse part: nonzeros of column j inside the warp's rows
        const int64_t cb = P.col_ptr[j];
        const int32_t* ri = P.row_idx + cb;
        const T* vals = P.values ? reinterpret_cast<const T*>(P.values) + cb : nullptr;
        const int a = P.woff[(size_t)j * nw1 + gw];
        const int b = P.woff[(size_t)j * nw1 + gw + 1];
        A sacc[NS > 0 ? NS : 1];
#pragma unroll
        for (int s = 0; s < NS; ++s) acc_zero(sacc[s]);
        int kn = k_lo;
        int64_t next_end = kn < k_hi ? (int64_t)P.gend[kn] : LLONG_MAX;
        for (int base = a; base < b; base += 32) {
          const int i = base + lane;
          const bool valid = i < b;
          const int row = valid ? ri[i] : INT_MAX;
          const T x = valid ? (vals ? vals[i] : T(1)) : T(0);
          const T ev = valid ? e[row] : T(0);
          const T wv = (MODEL == 1 && valid) ? w2[row] : T(0);
          T sv[NS > 0 ? NS : 1];
          sv[0] = ev * x;
          if (NS > 1) sv[NS > 1 ? 1 : 0] = sv[0] * x;
          if (NS > 2) {
            sv[NS > 2 ? 2 : 0] = wv * sv[0];
            sv[NS > 3 ? 3 : 0] = wv * sv[NS > 1 ? 1 : 0];
          }
          const int nvalid = min(32, b - base);
          const int last_row = __shfl_sync(0xffffffffu, row, nvalid - 1);
          while (next_end < (int64_t)last_row) {
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              A pref = warp_sum(acc_add_v(sacc[s], (int64_t)row <= next_end ? sv[s] : T(0)));
              if (lane == 0) rec[(size_t)kn * M + C::smap(s)] = pref;
            }
            ++kn;
            next_end = kn < k_hi ? (int64_t)P.gend[kn] : LLONG_MAX;
          }
#pragma unroll
          for (int s = 0; s < NS; ++s) sacc[s] = acc_add_v(sacc[s], sv[s]);
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) tot[C::smap(s)] = warp_sum(sacc[s]);
        // ends after the last nonzero of the range see the whole warp total
        for (; kn < k_hi; ++kn)
          if (lane == 0)
#pragma unroll
            for (int s = 0; s < NS; ++s) rec[(size_t)kn * M + C::smap(s)] = tot[C::smap(s)];
      }
      if (lane == 0)
#pragma unroll
        for (int m = 0; m < M; ++m) s_wtot[w][m] = tot[m];
      __syncthreads();

      // ------------------------------ CTA combine and grid exchange #1
      if (w == 0) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          A v;
          acc_zero(v);
          if (lane < WPC) v = s_wtot[lane][m];
          A incl = warp_inclusive_scan(v, lane);
          A excl = shfl_up(incl, 1);
          if (lane == 0) acc_zero(excl);
          if (lane < WPC) s_woff[lane][m] = excl;
          A agg = shfl_idx(incl, WPC - 1);
          if (lane == 0) {
            unsigned* slot = P.slot_agg + ((size_t)par * G + c) * kSlotWords;
            put_acc(slot + 2 * m, agg);
          }
        }
        if (lane == 0 && c != P.withhold_cta) exchange_arrive(P.counters + 0);
        bool ok = exchange_wait(P.counters + 0, (unsigned)passes * (unsigned)G, P.err, P.timeout_ns);
        if (lane == 0) s_flag[0] = ok ? 0 : 1;
        if (ok) {
          // exclusive prefix over CTAs < c, and (Fine-Gray) the grand total
          A pre[M], all[M];
#pragma unroll
          for (int m = 0; m < M; ++m) { acc_zero(pre[m]); acc_zero(all[m]); }
          for (int q = lane; q < G; q += 32) {
            const unsigned* slot = P.slot_agg + ((size_t)par * G + q) * kSlotWords;
#pragma unroll
            for (int m = 0; m < M; ++m) {
              A v = get_acc<A>(slot + 2 * m);
              if (q < c) pre[m] = acc_add(pre[m], v);
              if (MODEL == 1) all[m] = acc_add(all[m], v);
            }
          }
#pragma unroll
          for (int m = 0; m < M; ++m) {
            A t = warp_sum(pre[m]);
            if (lane == 0) s_T[m] = t;
            if (MODEL == 1) {
              A a2 = warp_sum(all[m]);
              if (lane == 0) s_tot[m] = a2;
            }
          }
          // penalty and delta^T eta = sum_q beta_q (delta^T X_q) for the
          // objective.  Read here, before this CTA publishes its partial:
          // CTA 0 rewrites beta_j only after exchange #2.
          if (eval) {
            double pen = 0.0, lin = 0.0;
            for (int q = lane; q < P.p; q += 32) {
              const double bq = __ldcg(P.beta + q);
              lin += bq * P.dTx[q];
              if (P.penalty == 1) pen -= P.pen[q] * fabs(bq);
              else if (P.penalty == 2) pen -= P.pen[q] * bq * bq * 0.5;
            }
            lin = warp_sum(lin);
            pen = warp_sum(pen);
            if (lane == 0) { s_scal[4] = lin; s_scal[3] = pen; }
          }
        }
      }
      __syncthreads();
      if (s_flag[0]) { finished = true; break; }

      // ------------------------------ steps 3-4: transform at group ends
      A pg1, pg2;
      acc_zero(pg1);
      acc_zero(pg2);
      double pl = 0.0;
      for (int k = kc_lo + tid; k < kc_hi; k += NT) {
        const int d = P.dk[k];
        if (d == 0) continue;
        const int64_t row = P.gend[k];
        const int wl = (int)((row >> 5) / P.wpw) - c * WPC;
        A Pm[M];
#pragma unroll
        for (int m = 0; m < M; ++m) Pm[m] = acc_add(acc_add(s_T[m], s_woff[wl][m]), rec[(size_t)k * M + m]);
        A den = Pm[0], num1 = Pm[1], num2 = Pm[2];
        if (MODEL == 1) {
          // R_2 part: G(t_k) times the suffix strictly after the group end
          A Gk = acc_from_d(P.Gk[k], (A*)nullptr);
          A q0 = acc_add(s_tot[3], acc_neg(Pm[3]));
          A q1 = acc_add(s_tot[4], acc_neg(Pm[4]));
          A q2 = acc_add(s_tot[5], acc_neg(Pm[5]));
          den = acc_add(den, acc_mul(Gk, q0));
          num1 = acc_add(num1, acc_mul(Gk, q1));
          num2 = acc_add(num2, acc_mul(Gk, q2));
        }
        A Gr = acc_div(num1, den);
        A H = acc_div(num2, den);
        pg1 = acc_add(pg1, acc_scale(Gr, d));
        pg2 = acc_add(pg2, acc_scale(acc_add(H, acc_neg(acc_mul(Gr, Gr))), d));
        if (eval) pl += (double)d * log(acc_to_d(den));
      }
      pg1 = warp_sum(pg1);
      pg2 = warp_sum(pg2);
#pragma unroll
      for (int dlt = 16; dlt > 0; dlt >>= 1) pl += __shfl_down_sync(0xffffffffu, pl, dlt);
      if (lane == 0) { s_red[w][0] = pg1; s_red[w][1] = pg2; s_redl[w] = pl; }
      __syncthreads();

      // ------------------------------ grid exchange #2: (g1, g2, l) partials
      if (w == 0) {
        A a1, a2;
        acc_zero(a1);
        acc_zero(a2);
        double al = 0.0;
        if (lane < WPC) { a1 = s_red[lane][0]; a2 = s_red[lane][1]; al = s_redl[lane]; }
        a1 = warp_sum(a1);
        a2 = warp_sum(a2);
#pragma unroll
        for (int dlt = 16; dlt > 0; dlt >>= 1) al += __shfl_down_sync(0xffffffffu, al, dlt);
        al = __shfl_sync(0xffffffffu, al, 0);
        unsigned* slot = P.slot_part + ((size_t)par * G + c) * kSlotWords;
        if (lane == 0) {
          put_acc(slot + 0, a1);
          put_acc(slot + 2, a2);
          put_acc(slot + 4, al);
          if (c != P.withhold_cta) exchange_arrive(P.counters + 1);
        }
        bool ok = exchange_wait(P.counters + 1, (unsigned)passes * (unsigned)G, P.err, P.timeout_ns);
        if (lane == 0) s_flag[1] = ok ? 0 : 1;
        if (ok) {
          A g1, g2;
          acc_zero(g1);
          acc_zero(g2);
          double gl = 0.0;
          for (int q = lane; q < G; q += 32) {
            const unsigned* sq = P.slot_part + ((size_t)par * G + q) * kSlotWords;
            g1 = acc_add(g1, get_acc<A>(sq + 0));
            g2 = acc_add(g2, get_acc<A>(sq + 2));
            gl += get_acc<double>(sq + 4);
          }
          g1 = warp_sum(g1);
          g2 = warp_sum(g2);
          gl = warp_sum(gl);
          if (lane == 0) {
            s_scal[0] = P.dTx[j] - acc_to_d(g1);   // l'
            s_scal[1] = -acc_to_d(g2);             // l''
            s_scal[2] = s_scal[4] - gl;            // l = delta^T eta - sum_k d_k log den_k
          }
        }
      }
      __syncthreads();
      if (s_flag[1]) { finished = true; break; }

      const double grad = s_scal[0], hess = s_scal[1];
      if (eval) {
        const double ll = s_scal[2];
        const double f = ll + s_scal[3];
        ll_last = ll;
        if (single) {
          if (c == 0 && tid == 0) {
            P.out[OUT_GRAD] = grad;
            P.out[OUT_HESS] = hess;
            P.out[OUT_LOGLIK] = ll;
            P.out[OUT_OBJECTIVE] = f;
          }
          finished = true;
          break;
        }
        if (sweep >= 1 && fabs(f - f_prev) / fabs(f) < P.tol) {
          converged = 1;
          f_prev2 = f_prev;
          f_prev = f;
          finished = true;
          break;
        }
        f_prev2 = f_prev;
        f_prev = f;
        if (sweep >= P.max_sweeps) { finished = true; break; }
      }

      // ------------------------------ Newton step and conditional update
      const double step = newton_step(bj, grad, hess, P.penalty, P.pen[j]);
      double applied = 0.0;
      if (step != 0.0) applied = copysign(fmin(fabs(step), wj), step);
      const double wnew = fmax(2.0 * fabs(applied), wj / 2.0);
      if (c == 0 && tid == 0) {
        P.beta[j] = bj + applied;
        P.width[j] = wnew;
      }
      if (applied != 0.0) {
        ++eta_updates;
        if (LAYOUT == 0) {
          const int64_t cb = P.col_ptr[j];
          const int a = P.woff[(size_t)j * nw1 + c * WPC];
          const int b = P.woff[(size_t)j * nw1 + (c + 1) * WPC];
          const int32_t* ri = P.row_idx + cb;
          const T* vals = P.values ? reinterpret_cast<const T*>(P.values) + cb : nullptr;
          auto* etap = reinterpret_cast<typename std::conditional<sizeof(T) == 4, float2, double>::type*>(P.eta);
          for (int i = a + tid; i < b; i += NT) {
            const T x = vals ? vals[i] : T(1);
            if constexpr (sizeof(T) == 4)
              eta_axpy(etap, reinterpret_cast<float*>(P.e), ri[i], (float)x, d_to_ff(applied));
            else
              eta_axpy(etap, reinterpret_cast<double*>(P.e), ri[i], (double)x, applied);
          }
        } else {
          const T* xcol = reinterpret_cast<const T*>(P.X) + (size_t)j * P.ld;
          auto* etap = reinterpret_cast<typename std::conditional<sizeof(T) == 4, float2, double>::type*>(P.eta);
          for (int64_t i = cta_row_lo + tid; i < cta_row_hi; i += NT) {
            if constexpr (sizeof(T) == 4)
              eta_axpy(etap, reinterpret_cast<float*>(P.e), i, (float)xcol[i], d_to_ff(applied));
            else
              eta_axpy(etap, reinterpret_cast<double*>(P.e), i, (double)xcol[i], applied);
          }
        }
      }
      __syncthreads();
    }
    if (finished) break;
    ++sweep;
  }

  if (c == 0 && tid == 0) {
    P.out[OUT_SWEEPS] = (double)sweep;
    P.out[OUT_CONVERGED] = (double)converged;
    P.out[OUT_ETA_UPDATES] = (double)eta_updates;
    P.out[OUT_PASSES] = (double)passes;
    P.out[OUT_EPOCH_END] = (double)epoch;
    if (!single) {
      P.out[OUT_LOGLIK] = ll_last;
      P.out[OUT_OBJECTIVE] = f_prev;
      P.out[OUT_OBJECTIVE_PREV] = f_prev2;
    }
  }
}

template <int MODEL, int LAYOUT, typename T>
cudaError_t launch_one(const CcdParams& P, cudaStream_t s) {
  void* args[] = {const_cast<CcdParams*>(&P)};
  return cudaLaunchCooperativeKernel((const void*)ccd_kernel<MODEL, LAYOUT, T>, dim3(P.G), dim3(32 * P.wpc),
                                     args, 0, s);
}

// One CTA per SM, as many warps (<= 32) as the register budget allows.
template <int MODEL, int LAYOUT, typename T>
cudaError_t grid_one(int* G, int* wpc) {
  int dev = 0, sms = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st != cudaSuccess) return st;
  st = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (st != cudaSuccess) return st;
  for (int w = Cfg<MODEL, LAYOUT, T>::MAXT / 32; w >= 4; w /= 2) {
    int occ = 0;
    st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ccd_kernel<MODEL, LAYOUT, T>, 32 * w, 0);
    if (st != cudaSuccess) return st;
    if (occ >= 1) {
      *G = sms;
      *wpc = w;
      return cudaSuccess;
    }
  }
  return cudaErrorLaunchOutOfResources;
}

}  // namespace

#define SURV_DISPATCH(FN, ...)                                               \
  do {                                                                       \
    if (model == 0 && layout == 0 && prec == 0) return FN<0, 0, float>(__VA_ARGS__);  \
    if (model == 0 && layout == 0 && prec == 1) return FN<0, 0, double>(__VA_ARGS__); \
    if (model == 0 && layout == 1 && prec == 0) return FN<0, 1, float>(__VA_ARGS__);  \
    if (model == 0 && layout == 1 && prec == 1) return FN<0, 1, double>(__VA_ARGS__); \
    if (model == 1 && layout == 0 && prec == 0) return FN<1, 0, float>(__VA_ARGS__);  \
    if (model == 1 && layout == 0 && prec == 1) return FN<1, 0, double>(__VA_ARGS__); \
    if (model == 1 && layout == 1 && prec == 0) return FN<1, 1, float>(__VA_ARGS__);  \
    if (model == 1 && layout == 1 && prec == 1) return FN<1, 1, double>(__VA_ARGS__); \
    return cudaErrorInvalidValue;                                            \
  } while (0)

cudaError_t launch_ccd(int model, int layout, int prec, const CcdParams& P, cudaStream_t s) {
  SURV_DISPATCH(launch_one, P, s);
}

cudaError_t ccd_grid_size(int model, int layout, int prec, int* G, int* wpc) {
  SURV_DISPATCH(grid_one, G, wpc);
}

}  // namespace survgpu
