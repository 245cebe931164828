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

__device__ __forceinline__ ff acc_from_d(double d, ff*) { return d_to_ff(d); }
__device__ __forceinline__ double acc_from_d(double d, double*) { return d; }
__device__ __forceinline__ ff acc_div(ff a, ff b) { return ff_div(a, b); }
__device__ __forceinline__ double acc_div(double a, double b) { return a / b; }
__device__ __forceinline__ ff acc_mul(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ double acc_mul(double a, double b) { return a * b; }
__device__ __forceinline__ ff acc_scale(ff a, int d) { return ff_mul_f(a, (float)d); }
// a base value held both as double and as float-float: pick the accumulator's form
template <typename A> __device__ __forceinline__ A acc_base(double d, ff f);
template <> __device__ __forceinline__ ff acc_base<ff>(double, ff f) { return f; }
template <> __device__ __forceinline__ double acc_base<double>(double d, ff) { return d; }
__device__ __forceinline__ ff acc_recip(ff a) { return ff_div({1.f, 0.f}, a); }
__device__ __forceinline__ double acc_recip(double a) { return 1.0 / a; }
__device__ __forceinline__ double acc_scale(double a, int d) { return a * (double)d; }

// Grid exchange: every CTA writes its payload slot, then thread 0 fences and
// adds 1 to the exchange counter; lane 0 of the waiting warp polls the counter
// with acquire loads until it reaches `target` (= exchanges so far x G), then
// the warp reads the payloads through L2.  One counter measured faster on
// GB300 than one flag per CTA or counters spread over several lines.  The
// wait is bounded by limit_ns.
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
      v = ld_acquire(counter);
      if (v < target) bad = ld_volatile(err);
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
  __syncwarp();
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
  // loads per lane per tile: CSC streams only e, so a lane keeps 16 loads in
  // flight; dense X and Fine-Gray stream two or three arrays
  static constexpr int U = LAYOUT == 0 ? (MODEL == 0 ? (sizeof(T) == 4 ? 16 : 8) : 8) : 4;
  static constexpr int TILE = 32 * U * VEC;                  // rows per warp tile
  // components produced by the dense row pass
  static constexpr int ND = LAYOUT == 1 ? M : (MODEL == 0 ? 1 : 2);
  // components produced by the sparse (CSC entry) pass
  static constexpr int NS = LAYOUT == 1 ? 0 : (MODEL == 0 ? 2 : 4);
  // threads per CTA the kernel is compiled for: 512 (128 registers).  1024
  // threads cap a thread at 64 registers, which spills this kernel, and make
  // every block barrier slower.
  static constexpr int MAXT = 512;
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
  constexpr int SR = 4;  // rounds of 32 nonzeros whose loads are issued before the dense tiles

  __shared__ double s_wtot[kMaxWarpsPerCta][M];  // warp totals of the pass
  __shared__ double s_base[kMaxWarpsPerCta][M];  // prefix before each warp: CTAs before + warps before
  __shared__ ff s_baseff[kMaxWarpsPerCta][M];    // the same as float-float
  __shared__ double s_tot[M];                    // grand totals (Fine-Gray suffix)
  __shared__ ff s_totff[M];
  __shared__ double s_red[kMaxWarpsPerCta][3];
  __shared__ double s_bc[8];                     // scalars broadcast by thread 0
  __shared__ float s_delta[2];                   // applied step as float-float
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
  const int nends = kc_hi - kc_lo;

  const T* e = reinterpret_cast<const T*>(P.e);
  const T* w2 = reinterpret_cast<const T*>(P.w2);
  A* rec = reinterpret_cast<A*>(P.rec);
  const int nw1 = P.nwarps + 1;
  const bool single = P.single_j >= 0;

  // control state, meaningful in thread 0 only (identical in every CTA)
  int sweep = 0, converged = 0;
  double f_prev = 0.0, f_prev2 = 0.0, ll_last = 0.0;
  long long eta_updates = 0;
  unsigned passes = 0;
  bool finished = false;
  // phase timers (thread 0): CTA 0 reports its phases, every CTA its pass time
  unsigned long long ph[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  uint64_t tmark = 0;
  auto lap = [&](int i) {
    if (tid == 0) {
      const uint64_t t = global_ns();
      ph[i] += t - tmark;
      tmark = t;
    }
  };

  while (!finished) {
    for (int jj = 0; jj < P.p; ++jj) {
      const int j = single ? P.single_j : jj;
      const bool eval = single || jj == 0;
      ++passes;
      const int par = passes & 1;
      // beta_j and Delta_j are read before this CTA publishes anything for
      // this coordinate; CTA 0 rewrites them only after exchange #2, which
      // needs every CTA's partial.  L2 loads: the writer is another SM.
      if (tid == 0) {
        s_bc[5] = __ldcg(P.beta + j);
        s_bc[6] = __ldcg(P.width + j);
        s_bc[1] = P.dTx[j];
        s_bc[2] = P.pen[j];
        tmark = global_ns();
      }

      // ------------------------------------------------ step 2: warp pass
      // sparse part first issues the loads of its first SR rounds so their
      // latency overlaps the dense tiles
      int sa = 0, sb = 0;
      const int32_t* ri = nullptr;
      const T* vals = nullptr;
      int prow[SR];
      T pval[SR];
      if (LAYOUT == 0) {
        const int64_t cb = P.col_ptr[j];
        ri = P.row_idx + cb;
        vals = P.values ? reinterpret_cast<const T*>(P.values) + cb : nullptr;
        sa = P.woff[(size_t)j * nw1 + gw];
        sb = P.woff[(size_t)j * nw1 + gw + 1];
#pragma unroll
        for (int r = 0; r < SR; ++r) {
          const int i = sa + 32 * r + lane;
          const bool valid = i < sb;
          prow[r] = valid ? ri[i] : INT_MAX;
          pval[r] = valid ? (vals ? vals[i] : T(1)) : T(0);
        }
      }

      A tot[M];
#pragma unroll
      for (int m = 0; m < M; ++m) acc_zero(tot[m]);
      {
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
        // sparse part: the nonzeros of column j inside the warp's rows
        A sacc[NS > 0 ? NS : 1];
#pragma unroll
        for (int s = 0; s < NS; ++s) acc_zero(sacc[s]);
        int kn = k_lo;
        int64_t next_end = kn < k_hi ? (int64_t)P.gend[kn] : LLONG_MAX;
        auto round = [&](int row, T x, T ev, T wv, int nvalid) {
          T sv[NS > 0 ? NS : 1];
          sv[0] = ev * x;
          if (NS > 1) sv[NS > 1 ? 1 : 0] = sv[0] * x;
          if (NS > 2) {
            sv[NS > 2 ? 2 : 0] = wv * sv[0];
            sv[NS > 3 ? 3 : 0] = wv * sv[NS > 1 ? 1 : 0];
          }
          const int last_row = __shfl_sync(0xffffffffu, row, nvalid - 1);
          // ends before the round's last nonzero see only part of the round
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
        };
        T pe[SR], pw[SR];
#pragma unroll
        for (int r = 0; r < SR; ++r) {
          pe[r] = prow[r] != INT_MAX ? e[prow[r]] : T(0);
          pw[r] = (MODEL == 1 && prow[r] != INT_MAX) ? w2[prow[r]] : T(0);
        }
#pragma unroll
        for (int r = 0; r < SR; ++r)
          if (sa + 32 * r < sb) round(prow[r], pval[r], pe[r], pw[r], min(32, sb - sa - 32 * r));
        for (int base = sa + 32 * SR; base < sb; base += 32) {
          const int i = base + lane;
          const bool valid = i < sb;
          const int row = valid ? ri[i] : INT_MAX;
          const T x = valid ? (vals ? vals[i] : T(1)) : T(0);
          const T ev = valid ? e[row] : T(0);
          const T wv = (MODEL == 1 && valid) ? w2[row] : T(0);
          round(row, x, ev, wv, min(32, sb - base));
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
        for (int m = 0; m < M; ++m) s_wtot[w][m] = acc_to_d(tot[m]);
      __syncthreads();
      lap(PH_PASS);

      // ------------------------------ CTA combine and grid exchange #1
      // Exchange payloads are laid out [parity][component][CTA] in doubles so
      // that one warp reads every CTA's value with coalesced loads.
      if (w == 0) {
        double* agg_soa = reinterpret_cast<double*>(P.slot_agg) + (size_t)par * 6 * G;
        double wv[M], excl[M];
#pragma unroll
        for (int m = 0; m < M; ++m) wv[m] = lane < WPC ? s_wtot[lane][m] : 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const double a = warp_sum(wv[m]);
          if (lane == 0) agg_soa[(size_t)m * G + c] = a;
        }
        if (lane == 0 && c != P.withhold_cta) exchange_arrive(P.counters + 0);
        lap(PH_EX1_PRE);
        // CTA-local work while the other CTAs arrive: warp offsets, and the
        // loads of beta / dTx / penalty factors for the objective
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const double incl = warp_inclusive_scan(wv[m], lane);
          double ex = shfl_up(incl, 1);
          excl[m] = lane == 0 ? 0.0 : ex;
        }
        double pen = 0.0, lin = 0.0;
        if (eval) {
          for (int q0 = 0; q0 < P.p; q0 += 32 * 4) {
            double bq[4], dq[4], fq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int q = q0 + 32 * u + lane;
              bq[u] = q < P.p ? __ldcg(P.beta + q) : 0.0;
              dq[u] = q < P.p ? P.dTx[q] : 0.0;
              fq[u] = q < P.p ? P.pen[q] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              lin += bq[u] * dq[u];
              if (P.penalty == 1) pen -= fq[u] * fabs(bq[u]);
              else if (P.penalty == 2) pen -= fq[u] * bq[u] * bq[u] * 0.5;
            }
          }
          lin = warp_sum(lin);
          pen = warp_sum(pen);
        }
        bool ok = exchange_wait(P.counters + 0, passes * (unsigned)G, P.err, P.timeout_ns);
        lap(PH_EX1_WAIT);
        if (lane == 0) s_flag[0] = ok ? 0 : 1;
        if (ok) {
          // exclusive prefix over CTAs < c (fixed order) and grand totals
          double pre[M], all[M];
#pragma unroll
          for (int m = 0; m < M; ++m) { pre[m] = 0.0; all[m] = 0.0; }
          for (int q0 = 0; q0 < G; q0 += 32 * 5) {
            double v[M][5];
#pragma unroll
            for (int u = 0; u < 5; ++u) {
              const int q = q0 + 32 * u + lane;
#pragma unroll
              for (int m = 0; m < M; ++m) v[m][u] = q < G ? __ldcg(agg_soa + (size_t)m * G + q) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 5; ++u) {
              const int q = q0 + 32 * u + lane;
#pragma unroll
              for (int m = 0; m < M; ++m) {
                if (q < c) pre[m] += v[m][u];
                if (MODEL == 1) all[m] += v[m][u];
              }
            }
          }
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const double T_c = warp_sum(pre[m]);
            if (MODEL == 1) {
              const double a2 = warp_sum(all[m]);
              if (lane == 0) { s_tot[m] = a2; s_totff[m] = d_to_ff(a2); }
            }
            if (lane < WPC) {
              const double b = T_c + excl[m];
              s_base[lane][m] = b;
              s_baseff[lane][m] = d_to_ff(b);
            }
          }
          if (eval && lane == 0) { s_bc[3] = pen; s_bc[4] = lin; }
        }
      }
      __syncthreads();
      lap(PH_EX1_POST);
      if (s_flag[0]) { finished = true; break; }

      // ------------------------------ steps 3-4: transform at group ends
      // Few ends per CTA: one end per thread in FP64 (latency-bound).  Many
      // ends: float-float (FP64 throughput on GB300 is ~1/70 of FP32).
      double pg1 = 0.0, pg2 = 0.0, pl = 0.0;
      int nw_red;
      if (nends <= NT) {
        nw_red = (nends + 31) >> 5;
        if (tid < nends) {
          const int k = kc_lo + tid;
          const int d = P.dk[k];
          if (d != 0) {
            const int wl = (int)((P.gend[k] >> 5) / P.wpw) - c * WPC;
            double Pm[M];
#pragma unroll
            for (int m = 0; m < M; ++m) Pm[m] = s_base[wl][m] + acc_to_d(rec[(size_t)k * M + m]);
            double den = Pm[0], num1 = Pm[1], num2 = Pm[2];
            if (MODEL == 1) {
              const double g = P.Gk[k];
              den += g * (s_tot[3] - Pm[3]);
              num1 += g * (s_tot[4] - Pm[4]);
              num2 += g * (s_tot[5] - Pm[5]);
            }
            const double inv = 1.0 / den;
            const double Gr = num1 * inv, H = num2 * inv;
            pg1 = d * Gr;
            pg2 = d * (H - Gr * Gr);
            if (eval) pl = d * log(den);
          }
        }
        if (w < nw_red) {
          pg1 = warp_sum(pg1);
          pg2 = warp_sum(pg2);
          pl = warp_sum(pl);
          if (lane == 0) { s_red[w][0] = pg1; s_red[w][1] = pg2; s_red[w][2] = pl; }
        }
      } else {
        nw_red = WPC;
        A fg1, fg2;
        acc_zero(fg1);
        acc_zero(fg2);
        for (int k = kc_lo + tid; k < kc_hi; k += NT) {
          const int d = P.dk[k];
          if (d == 0) continue;
          const int wl = (int)((P.gend[k] >> 5) / P.wpw) - c * WPC;
          A Pm[M];
#pragma unroll
          for (int m = 0; m < M; ++m) Pm[m] = acc_add(acc_base<A>(s_base[wl][m], s_baseff[wl][m]), rec[(size_t)k * M + m]);
          A den = Pm[0], num1 = Pm[1], num2 = Pm[2];
          if (MODEL == 1) {
            const float2 gf = P.Gkff[k];
            const A g = acc_base<A>(P.Gk[k], ff{gf.x, gf.y});
            den = acc_add(den, acc_mul(g, acc_add(acc_base<A>(s_tot[3], s_totff[3]), acc_neg(Pm[3]))));
            num1 = acc_add(num1, acc_mul(g, acc_add(acc_base<A>(s_tot[4], s_totff[4]), acc_neg(Pm[4]))));
            num2 = acc_add(num2, acc_mul(g, acc_add(acc_base<A>(s_tot[5], s_totff[5]), acc_neg(Pm[5]))));
          }
          const A inv = acc_recip(den);
          const A Gr = acc_mul(num1, inv);
          const A H = acc_mul(num2, inv);
          fg1 = acc_add(fg1, acc_scale(Gr, d));
          fg2 = acc_add(fg2, acc_scale(acc_add(H, acc_neg(acc_mul(Gr, Gr))), d));
          if (eval) pl += (double)d * log(acc_to_d(den));
        }
        fg1 = warp_sum(fg1);
        fg2 = warp_sum(fg2);
#pragma unroll
        for (int dl = 16; dl > 0; dl >>= 1) pl += __shfl_down_sync(0xffffffffu, pl, dl);
        if (lane == 0) { s_red[w][0] = acc_to_d(fg1); s_red[w][1] = acc_to_d(fg2); s_red[w][2] = pl; }
      }
      __syncthreads();
      lap(PH_TRANSFORM);

      // ------------------------------ grid exchange #2, Newton step
      if (w == 0) {
        double* part_soa = reinterpret_cast<double*>(P.slot_part) + (size_t)par * 3 * G;
        const double a1 = warp_sum(lane < nw_red ? s_red[lane][0] : 0.0);
        const double a2 = warp_sum(lane < nw_red ? s_red[lane][1] : 0.0);
        const double al = warp_sum(lane < nw_red ? s_red[lane][2] : 0.0);
        if (lane == 0) {
          part_soa[c] = a1;
          part_soa[G + c] = a2;
          part_soa[2 * G + c] = al;
          if (c != P.withhold_cta) exchange_arrive(P.counters + 1);
        }
        lap(PH_EX2_PRE);
        bool ok = exchange_wait(P.counters + 1, passes * (unsigned)G, P.err, P.timeout_ns);
        lap(PH_EX2_WAIT);
        int fin = ok ? 0 : 2;
        if (ok) {
          double g1 = 0.0, g2 = 0.0, gl = 0.0;
          for (int q0 = 0; q0 < G; q0 += 32 * 5) {
            double v[3][5];
#pragma unroll
            for (int u = 0; u < 5; ++u) {
              const int q = q0 + 32 * u + lane;
#pragma unroll
              for (int m = 0; m < 3; ++m) v[m][u] = q < G ? __ldcg(part_soa + (size_t)m * G + q) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 5; ++u) { g1 += v[0][u]; g2 += v[1][u]; gl += v[2][u]; }
          }
          g1 = warp_sum(g1);
          g2 = warp_sum(g2);
          gl = warp_sum(gl);
          if (lane == 0) {
            const double grad = s_bc[1] - g1;    // l' = delta^T X_j - sum_k d_k G_k
            const double hess = -g2;             // l''
            double applied = 0.0;
            if (eval) {
              const double ll = s_bc[4] - gl;    // l = delta^T eta - sum_k d_k log den_k
              const double f = ll + s_bc[3];
              ll_last = ll;
              if (single) {
                if (c == 0) {
                  P.out[OUT_GRAD] = grad;
                  P.out[OUT_HESS] = hess;
                  P.out[OUT_LOGLIK] = ll;
                  P.out[OUT_OBJECTIVE] = f;
                }
                fin = 1;
              } else if (sweep >= 1 && fabs(f - f_prev) / fabs(f) < P.tol) {
                converged = 1;
                f_prev2 = f_prev;
                f_prev = f;
                fin = 1;
              } else {
                f_prev2 = f_prev;
                f_prev = f;
                if (sweep >= P.max_sweeps) fin = 1;
              }
            }
            if (!fin) {
              const double bj = s_bc[5], wj = s_bc[6];
              const double step = newton_step(bj, grad, hess, P.penalty, s_bc[2]);
              if (step != 0.0) applied = copysign(fmin(fabs(step), wj), step);
              const double wnew = fmax(2.0 * fabs(applied), wj / 2.0);
              if (c == 0) {
                P.beta[j] = bj + applied;
                P.width[j] = wnew;
              }
              if (applied != 0.0) ++eta_updates;
            }
            s_bc[0] = applied;
            const ff dl = d_to_ff(applied);
            s_delta[0] = dl.hi;
            s_delta[1] = dl.lo;
          }
        }
        if (lane == 0) s_flag[1] = fin;
      }
      __syncthreads();
      lap(PH_EX2_POST);
      if (s_flag[1]) { finished = true; break; }

      // ------------------------------ conditional update of eta and e
      const double applied = s_bc[0];
      if (applied != 0.0) {
        if (LAYOUT == 0) {
          const int a = P.woff[(size_t)j * nw1 + c * WPC];
          const int b = P.woff[(size_t)j * nw1 + (c + 1) * WPC];
          if constexpr (sizeof(T) == 4) {
            // loads batched 8 deep: the row indices, then eta, then the stores
            const ff delta = {s_delta[0], s_delta[1]};
            float2* etap = reinterpret_cast<float2*>(P.eta);
            float* ep = reinterpret_cast<float*>(P.e);
            for (int i0 = a; i0 < b; i0 += 8 * NT) {
              int rr[8];
              float xx[8];
              float2 qq[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * NT + tid;
                rr[u] = i < b ? ri[i] : -1;
                xx[u] = i < b ? (vals ? (float)vals[i] : 1.f) : 0.f;
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) qq[u] = rr[u] >= 0 ? etap[rr[u]] : make_float2(0.f, 0.f);
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                if (rr[u] < 0) continue;
                const ff v = ff_add({qq[u].x, qq[u].y}, ff_mul_f(delta, xx[u]));
                etap[rr[u]] = make_float2(v.hi, v.lo);
                const float ev = expf(v.hi);
                ep[rr[u]] = fmaf(ev, v.lo, ev);
              }
            }
          } else {
            for (int i = a + tid; i < b; i += NT)
              eta_axpy(reinterpret_cast<double*>(P.eta), reinterpret_cast<double*>(P.e), ri[i],
                       vals ? (double)vals[i] : 1.0, applied);
          }
        } else {
          const T* xcol = reinterpret_cast<const T*>(P.X) + (size_t)j * P.ld;
          if constexpr (sizeof(T) == 4) {
            const ff delta = {s_delta[0], s_delta[1]};
            for (int64_t i = cta_row_lo + tid; i < cta_row_hi; i += NT)
              eta_axpy(reinterpret_cast<float2*>(P.eta), reinterpret_cast<float*>(P.e), i, (float)xcol[i], delta);
          } else {
            for (int64_t i = cta_row_lo + tid; i < cta_row_hi; i += NT)
              eta_axpy(reinterpret_cast<double*>(P.eta), reinterpret_cast<double*>(P.e), i, (double)xcol[i], applied);
          }
        }
      }
      __syncthreads();
      lap(PH_UPDATE);
    }
    if (finished) break;
    ++sweep;
  }

  if (tid == 0 && P.timing) {
    atomicMax(P.timing + PH_PASS_MAX, ph[PH_PASS]);
    atomicMin(P.timing + PH_PASS_MIN, ph[PH_PASS]);
    atomicAdd(P.timing + PH_PASS_SUM, ph[PH_PASS]);
    if (c == 0)
      for (int i = 0; i < 9; ++i) P.timing[i] = ph[i];
  }
  if (c == 0 && tid == 0) {
    P.out[OUT_SWEEPS] = (double)sweep;
    P.out[OUT_CONVERGED] = (double)converged;
    P.out[OUT_ETA_UPDATES] = (double)eta_updates;
    P.out[OUT_PASSES] = (double)passes;
    P.out[OUT_EPOCH_END] = (double)passes;
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
