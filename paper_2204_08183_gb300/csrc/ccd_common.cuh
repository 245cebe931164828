// Device pieces shared by the two CCD schedules (the persistent kernel and
// the per-coordinate kernel pair): vector loads, the eta / e update, the
// exchange payload format, accumulator helpers, the Newton step of
// Section 2.4 and the row pass of step 2.
#pragma once
#include <cfloat>
#include <climits>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace survgpu {
namespace ccdk {

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
// (a subject held out of a cross-validation fit keeps e = 0)
__device__ __forceinline__ void eta_axpy(float2* eta, float* e, int64_t i, float x, ff delta, bool held = false) {
  float2 q = eta[i];
  ff v = ff_add({q.x, q.y}, ff_mul_f(delta, x));
  eta[i] = make_float2(v.hi, v.lo);
  float ev = expf(v.hi);
  e[i] = held ? 0.f : fmaf(ev, v.lo, ev);  // exp(hi + lo) to first order in lo
}
__device__ __forceinline__ void eta_axpy(double* eta, double* e, int64_t i, double x, double delta,
                                         bool held = false) {
  double v = eta[i] + x * delta;
  eta[i] = v;
  e[i] = held ? 0.0 : exp(v);
}

// 8-byte exchange payload words: float-float as (hi, lo), double as its bits
__device__ __forceinline__ uint64_t pack8(ff a) {
  return (uint64_t)__float_as_uint(a.hi) | ((uint64_t)__float_as_uint(a.lo) << 32);
}
__device__ __forceinline__ uint64_t pack8(double a) { return (uint64_t)__double_as_longlong(a); }
template <typename A> __device__ __forceinline__ A unpack8(uint64_t w);
template <> __device__ __forceinline__ ff unpack8<ff>(uint64_t w) {
  return {__uint_as_float((unsigned)(w & 0xffffffffull)), __uint_as_float((unsigned)(w >> 32))};
}
template <> __device__ __forceinline__ double unpack8<double>(uint64_t w) { return __longlong_as_double((long long)w); }

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

// Newton step on g = l + pi for one coordinate (Section 2.4); grad, hess are
// the log-likelihood derivatives.  Mirrors the CPU reading exactly.
__device__ __forceinline__ double newton_step(double b, double grad, double hess, int penalty, double lam) {
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
  static constexpr int U = LAYOUT == 0 ? 8 : 4;
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


// Data a warp's pass reads that does not depend on e: the positions of
// the group ends in its rows (lane i holds gend[k_lo + i]) and the first
// SR rounds of 32 nonzeros of column j in its rows (row index and value).
// A kernel loads them before it waits for anything.
template <typename T, int SR_>
struct PassPrefetch {
  static constexpr int SR = SR_;
  int k_lo = 0, k_hi = 0;
  int kreg = INT_MAX;
  int sa = 0, sb = 0;
  const int32_t* ri = nullptr;
  const T* vals = nullptr;
  int prow[SR];
  T pval[SR];
};

template <int LAYOUT, typename T, int SR>
__device__ __forceinline__ void pass_prefetch(const CcdParams& P, int j, int gw, PassPrefetch<T, SR>& pf) {
  const int lane = threadIdx.x & 31;
  pf.k_lo = P.wk0[gw];
  pf.k_hi = P.wk0[gw + 1];
  pf.kreg = pf.k_lo + lane < pf.k_hi ? P.gend[pf.k_lo + lane] : INT_MAX;
  if (LAYOUT != 0) return;
  const int nw1 = P.nwarps + 1;
  const int64_t cb = P.col_ptr[j];
  pf.ri = P.row_idx + cb;
  pf.vals = P.values ? reinterpret_cast<const T*>(P.values) + cb : nullptr;
  pf.sa = P.woff[(size_t)j * nw1 + gw];
  pf.sb = P.woff[(size_t)j * nw1 + gw + 1];
  const uint64_t strm = l2_stream();
#pragma unroll
  for (int r = 0; r < SR; ++r) {
    const int i = pf.sa + 32 * r + lane;
    const bool valid = i < pf.sb;
    pf.prow[r] = valid ? ld_hint(pf.ri + i, strm) : INT_MAX;
    pf.pval[r] = valid ? (pf.vals ? ld_stream(pf.vals + i, strm) : T(1)) : T(0);
  }
}

// Walks the group ends of a warp in order; positions come from the lane
// registers of the prefetch, 32 at a time (kn is the same in every lane).
struct EndCursor {
  int kn, k_hi, base, reg;
  __device__ __forceinline__ int64_t pos(const int32_t* gend) {
    if (kn >= k_hi) return LLONG_MAX;
    if (kn - base >= 32) {
      base = kn;
      const int i = base + (int)(threadIdx.x & 31);
      reg = i < k_hi ? gend[i] : INT_MAX;
    }
    return (int64_t)__shfl_sync(0xffffffffu, reg, kn - base);
  }
  // after pos(): is the end after the current one also before `limit`?
  // (true when it lies outside the loaded window: the caller then takes its
  // general path, which is correct for any number of ends)
  __device__ __forceinline__ bool second_before(int64_t limit) const {
    const int k2 = kn + 1;
    if (k2 >= k_hi) return false;
    if (k2 - base >= 32) return true;
    return (int64_t)__shfl_sync(0xffffffffu, reg, k2 - base) < limit;
  }
};

// Step 2 for one warp: the tuple sums over rows [row_lo, row_hi) of column j.
// At every group end k of the warp the warp-relative prefix (rows of the
// warp up to and including the end) is stored in rec[k * M + m]; tot[] gets
// the warp totals (every lane holds them).  The dense components stream e
// (and X, W) in tiles of 32 * U * VEC rows; the CSC components walk the
// column's nonzeros in the warp's rows (woff holds the per-warp offsets).
template <int MODEL, int LAYOUT, typename T, int U_, int SR, bool MULTI = false>
// dense = false (CSC only): e has not changed since the previous pass of the
// fit, so the dense components (e, and for Fine-Gray W e), their records at
// the group ends and their totals are the stored ones; they are neither
// recomputed nor written (tot gets zeros for them).
// xq (dense X, FP32 only): the pending step delta of the column xq is applied
// in the same sweep over the warp's rows: each tile loads eta and x_q
// instead of e, writes eta + delta x_q and its e (the arithmetic of
// warp_update, element for element) and passes the new e on; null: e is read.
__device__ __forceinline__ void warp_pass(const CcdParams& P, int j, int64_t row_lo, int64_t row_hi,
                                          typename AccOf<T>::type* rec,
                                          typename AccOf<T>::type (&tot)[Cfg<MODEL, LAYOUT, T>::M],
                                          const PassPrefetch<T, SR>& pf, bool dense = true,
                                          const T* xq = nullptr, ff delta = ff{0.f, 0.f}) {
  using A = typename AccOf<T>::type;
  using C = Cfg<MODEL, LAYOUT, T>;
  constexpr int M = C::M;
  constexpr int VEC = C::VEC;
  constexpr int U = U_;
  constexpr int TILE = 32 * U * VEC;
  constexpr int ND = C::ND;
  constexpr int NS = C::NS;
  const int lane = threadIdx.x & 31;
  const T* e = reinterpret_cast<const T*>(P.e);
  const T* w2 = reinterpret_cast<const T*>(P.w2);
  const uint64_t keep = l2_keep(), strm = l2_stream();
#pragma unroll
  for (int m = 0; m < M; ++m) acc_zero(tot[m]);
  if (LAYOUT == 1 || dense) {
    A acc[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) acc_zero(acc[d]);
    EndCursor ec{pf.k_lo, pf.k_hi, pf.k_lo, pf.kreg};
    int64_t next_end = ec.pos(P.gend);
    const T* xcol = LAYOUT == 1 ? reinterpret_cast<const T*>(P.X) + (size_t)j * P.ld : nullptr;

    // loads of one tile from global memory (16-byte loads; the last partial
    // tile element by element)
    auto load_tile = [&](int64_t t0, T (&ev)[U][VEC], T (&xv)[U][VEC], T (&wv)[U][VEC]) {
      if constexpr (LAYOUT == 1 && sizeof(T) == 4) {
        if (xq) {
          // fused update of the pending step (FP32 mode: eta float-float)
          float2* etap = reinterpret_cast<float2*>(P.eta);
          float* ep = reinterpret_cast<float*>(P.e);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int64_t r = t0 + (int64_t)(lane + 32 * u) * VEC;
            float xx[VEC];
            float2 qq[VEC];
            if (r + VEC <= row_hi) {
              ld4_hint(reinterpret_cast<const float*>(xq) + r, strm, xx);
              const float4 a = *reinterpret_cast<const float4*>(etap + r);
              const float4 b = *reinterpret_cast<const float4*>(etap + r + 2);
              qq[0] = make_float2(a.x, a.y);
              qq[1] = make_float2(a.z, a.w);
              qq[2] = make_float2(b.x, b.y);
              qq[3] = make_float2(b.z, b.w);
              ld4_hint(xcol + r, strm, xv[u]);
              if (MODEL == 1) ld4_hint(w2 + r, keep, wv[u]);
            } else {
#pragma unroll
              for (int q = 0; q < VEC; ++q) {
                const bool in = r + q < row_hi;
                xx[q] = in ? reinterpret_cast<const float*>(xq)[r + q] : 0.f;
                qq[q] = in ? etap[r + q] : make_float2(0.f, 0.f);
                xv[u][q] = in ? xcol[r + q] : T(0);
                wv[u][q] = (MODEL == 1 && in) ? w2[r + q] : T(0);
              }
            }
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
              const ff v = ff_add({qq[q].x, qq[q].y}, ff_mul_f(delta, xx[q]));
              qq[q] = make_float2(v.hi, v.lo);
              const float ex = expf(v.hi);
              // rows past the warp's range take no part (e = 0), as in the plain loads
              const bool in = r + q < row_hi;
              const bool held = in && P.fold_id && P.fold_id[r + q] == P.fold;
              ev[u][q] = (!in || held) ? 0.f : fmaf(ex, v.lo, ex);
            }
            if (r + VEC <= row_hi) {
              *reinterpret_cast<float4*>(etap + r) = make_float4(qq[0].x, qq[0].y, qq[1].x, qq[1].y);
              *reinterpret_cast<float4*>(etap + r + 2) = make_float4(qq[2].x, qq[2].y, qq[3].x, qq[3].y);
              *reinterpret_cast<float4*>(ep + r) = make_float4(ev[u][0], ev[u][1], ev[u][2], ev[u][3]);
            } else {
#pragma unroll
              for (int q = 0; q < VEC; ++q)
                if (r + q < row_hi) {
                  etap[r + q] = qq[q];
                  ep[r + q] = ev[u][q];
                }
            }
          }
          return;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t r = t0 + (int64_t)(lane + 32 * u) * VEC;
        if (r + VEC <= row_hi) {
          ld4_hint(e + r, keep, ev[u]);
          if (LAYOUT == 1) ld4_hint(xcol + r, strm, xv[u]);
          if (MODEL == 1) ld4_hint(w2 + r, keep, wv[u]);
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
    };
    // One tile.  Lane l holds chunks c = 32 u + l of VEC consecutive rows
    // (rows t0 + VEC c .. + VEC - 1); chunk sums are pairwise within the
    // lane and feed the running sums.
    //   One dense component (CSC layouts of Cox): the lane's share of the
    //   rows up to an end in chunk c* is its chunks before c* plus chunk c*
    //   up to the end.  A tile with one end reduces (running sum + share)
    //   in one float-float tree; a tile with several reduces the running
    //   sums once and each end's shares in an FP32 tree.
    //   Several components (register pressure): every end reduces the
    //   running sums plus the tile's rows up to the end in one tree.
    auto chunk_sum = [&](int d, const T (&ev)[U][VEC], const T (&xv)[U][VEC], const T (&wv)[U][VEC], int u) {
      const T a0 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][0], xv[u][0], wv[u][0]);
      const T a1 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][1], xv[u][1], wv[u][1]);
      if (VEC == 4) {
        const T a2 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][VEC > 2 ? 2 : 0], xv[u][VEC > 2 ? 2 : 0],
                                                  wv[u][VEC > 2 ? 2 : 0]);
        const T a3 = dense_comp<MODEL, LAYOUT, T>(d, ev[u][VEC > 3 ? 3 : 0], xv[u][VEC > 3 ? 3 : 0],
                                                  wv[u][VEC > 3 ? 3 : 0]);
        return (a0 + a1) + (a2 + a3);
      }
      return a0 + a1;
    };
    auto tile = [&](int64_t t0, const T (&ev)[U][VEC], const T (&xv)[U][VEC], const T (&wv)[U][VEC]) {
      const int64_t t_end = min(t0 + (int64_t)TILE, row_hi);
      if constexpr (ND == 1 && MULTI) {
        // acc[0] is the warp-uniform sum of the rows before the tile.  One
        // FP32 lane scan per chunk row u gives every chunk's tile-relative
        // exclusive prefix; the lane that owns an end's chunk adds the rows
        // of the chunk up to the end and writes the record.
        T su[U], ex[U], tu[U];
#pragma unroll
        for (int u = 0; u < U; ++u) su[u] = chunk_sum(0, ev, xv, wv, u);
#pragma unroll
        for (int u = 0; u < U; ++u) ex[u] = su[u];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1)
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const T t = __shfl_up_sync(0xffffffffu, ex[u], d);
            if (lane >= d) ex[u] += t;
          }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          tu[u] = __shfl_sync(0xffffffffu, ex[u], 31);  // chunk row total
          const T t = __shfl_up_sync(0xffffffffu, ex[u], 1);
          ex[u] = lane == 0 ? T(0) : t;                  // lanes before, same u
        }
        while (next_end < t_end) {
          const int off = (int)(next_end - t0);
          const int cstar = off / VEC, qstar = off - cstar * VEC;
          if ((cstar & 31) == lane) {
            const int ustar = cstar >> 5;
            T pre = T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              if (u < ustar) pre += tu[u];
              if (u == ustar) {
                T in = ex[u];
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                  if (q <= qstar) in += dense_comp<MODEL, LAYOUT, T>(0, ev[u][q], xv[u][q], wv[u][q]);
                pre += in;
              }
            }
            rec[(size_t)ec.kn * M + C::dmap(0)] = acc_add_v(acc[0], pre);
          }
          ++ec.kn;
          next_end = ec.pos(P.gend);
        }
        T tt = tu[0];
#pragma unroll
        for (int u = 1; u < U; ++u) tt += tu[u];
        acc[0] = acc_add_v(acc[0], tt);
      } else {
        while (next_end < t_end) {
          A pref[ND];
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
            pref[d] = acc_add_v(acc[d], part);
          }
          warp_sum_some<ND>(pref);
          if (lane == 0)
#pragma unroll
            for (int d = 0; d < ND; ++d) rec[(size_t)ec.kn * M + C::dmap(d)] = pref[d];
          ++ec.kn;
          next_end = ec.pos(P.gend);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          T su[U];
#pragma unroll
          for (int u = 0; u < U; ++u) su[u] = chunk_sum(d, ev, xv, wv, u);
#pragma unroll
          for (int s = 1; s < U; s <<= 1)
#pragma unroll
            for (int u = 0; u + s < U; u += 2 * s) su[u] += su[u + s];
          acc[d] = acc_add_v(acc[d], su[0]);
        }
      }
    };

    for (int64_t t0 = row_lo; t0 < row_hi; t0 += TILE) {
      T ev[U][VEC], xv[U][VEC], wv[U][VEC];
      load_tile(t0, ev, xv, wv);
      tile(t0, ev, xv, wv);
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) tot[C::dmap(d)] = acc[d];  // lane partials (MULTI, ND = 1: the warp sum)
  }
  if (LAYOUT == 0 && NS > 0) {
    // sparse part: the nonzeros of column j inside the warp's rows
    if constexpr (MULTI) {
      const int sa = pf.sa, sb = pf.sb;
      const int32_t* ri = pf.ri;
      const T* vals = pf.vals;
      // Two running sums: sacc holds lane partials (plain adds), run the
      // warp-uniform sum folded in from sacc by rounds with several ends.  A
      // round with one end reduces sacc plus the round's nonzeros up to the
      // end in one tree.  A round with several ends folds sacc into run, takes
      // one inclusive lane scan, and each end reads the scan at the last
      // nonzero at or before it (row indices increase with the lane, so a
      // ballot counts them).
      constexpr int NSX = NS > 0 ? NS : 1;
      A sacc[NSX], run[NSX];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        acc_zero(sacc[s]);
        acc_zero(run[s]);
      }
      bool sacc_dirty = false;
      EndCursor ec{pf.k_lo, pf.k_hi, pf.k_lo, pf.kreg};
      int64_t next_end = ec.pos(P.gend);
      auto round = [&](int row, T x, T ev, T wv, int nvalid) {
        T sv[NSX];
        sv[0] = ev * x;
        if (NS > 1) sv[NS > 1 ? 1 : 0] = sv[0] * x;
        if (NS > 2) {
          sv[NS > 2 ? 2 : 0] = wv * sv[0];
          sv[NS > 3 ? 3 : 0] = wv * sv[NS > 1 ? 1 : 0];
        }
        const int last_row = __shfl_sync(0xffffffffu, row, nvalid - 1);
        if (next_end < (int64_t)last_row && !ec.second_before(last_row)) {
          // one end in the round: one tree of the lane partials and the
          // round's nonzeros up to the end
          A pref[NSX];
#pragma unroll
          for (int s = 0; s < NS; ++s) pref[s] = acc_add_v(sacc[s], (int64_t)row <= next_end ? sv[s] : T(0));
          warp_sum_some<NSX>(pref);
          if (lane == 0)
#pragma unroll
            for (int s = 0; s < NS; ++s) rec[(size_t)ec.kn * M + C::smap(s)] = acc_add(run[s], pref[s]);
          ++ec.kn;
          next_end = ec.pos(P.gend);
#pragma unroll
          for (int s = 0; s < NS; ++s) sacc[s] = acc_add_v(sacc[s], sv[s]);
          sacc_dirty = true;
        } else if (next_end < (int64_t)last_row) {
          if (sacc_dirty) {
            warp_sum_some<NSX>(sacc);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              run[s] = acc_add(run[s], sacc[s]);
              acc_zero(sacc[s]);
            }
            sacc_dirty = false;
          }
          A sc[NSX];
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            acc_zero(sc[s]);
            sc[s] = acc_add_v(sc[s], sv[s]);
          }
          warp_scan_n<NSX>(sc, lane);
          while (next_end < (int64_t)last_row) {
            const int cnt = __popc(__ballot_sync(0xffffffffu, (int64_t)row <= next_end));
            A pref[NSX];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              const A v = shfl_idx(sc[s], cnt > 0 ? cnt - 1 : 0);
              pref[s] = cnt > 0 ? acc_add(run[s], v) : run[s];
            }
            if (lane == 0)
#pragma unroll
              for (int s = 0; s < NS; ++s) rec[(size_t)ec.kn * M + C::smap(s)] = pref[s];
            ++ec.kn;
            next_end = ec.pos(P.gend);
          }
#pragma unroll
          for (int s = 0; s < NS; ++s) run[s] = acc_add(run[s], shfl_idx(sc[s], 31));
        } else {
#pragma unroll
          for (int s = 0; s < NS; ++s) sacc[s] = acc_add_v(sacc[s], sv[s]);
          sacc_dirty = true;
        }
      };
      // e (and W) at the prefetched rows
      T pe[SR], pw[SR];
#pragma unroll
      for (int r = 0; r < SR; ++r) {
        const int row = pf.prow[r];
        pe[r] = row == INT_MAX ? T(0) : ld_hint(e + row, keep);
        pw[r] = (MODEL == 1 && row != INT_MAX) ? ld_hint(w2 + row, keep) : T(0);
      }
      // one call site of round() (it is large): the first SR rounds take the
      // prefetched values through a select chain, later rounds load theirs
      int r = 0;
      for (int base = sa; base < sb; base += 32, ++r) {
        int row;
        T x, ev, wv;
        if (r < SR) {
          row = pf.prow[0];
          x = pf.pval[0];
          ev = pe[0];
          wv = pw[0];
#pragma unroll
          for (int q = 1; q < SR; ++q)
            if (r == q) {
              row = pf.prow[q];
              x = pf.pval[q];
              ev = pe[q];
              wv = pw[q];
            }
        } else {
          const int i = base + lane;
          const bool valid = i < sb;
          row = valid ? ld_hint(ri + i, strm) : INT_MAX;
          x = valid ? (vals ? ld_stream(vals + i, strm) : T(1)) : T(0);
          ev = valid ? ld_hint(e + row, keep) : T(0);
          wv = (MODEL == 1 && valid) ? ld_hint(w2 + row, keep) : T(0);
        }
        round(row, x, ev, wv, min(32, sb - base));
      }
      // lane partials of the rounds without ends are reduced; run and the
      // dense sum (both warp-uniform) are added after the reduction
#pragma unroll
      for (int s = 0; s < NS; ++s) tot[C::smap(s)] = sacc[s];
      const A dense_run = tot[C::dmap(0)];
      acc_zero(tot[C::dmap(0)]);
      warp_sum_some<M>(tot);
      tot[C::dmap(0)] = dense_run;
#pragma unroll
      for (int s = 0; s < NS; ++s) tot[C::smap(s)] = acc_add(run[s], tot[C::smap(s)]);
      // the ends after the last nonzero of the range see the warp totals
      for (; ec.kn < pf.k_hi; ++ec.kn)
        if (lane == 0)
#pragma unroll
          for (int s = 0; s < NS; ++s) rec[(size_t)ec.kn * M + C::smap(s)] = tot[C::smap(s)];
    } else {
      const int sa = pf.sa, sb = pf.sb;
      const int32_t* ri = pf.ri;
      const T* vals = pf.vals;
      A sacc[NS > 0 ? NS : 1];
#pragma unroll
      for (int s = 0; s < NS; ++s) acc_zero(sacc[s]);
      EndCursor ec{pf.k_lo, pf.k_hi, pf.k_lo, pf.kreg};
      int64_t next_end = ec.pos(P.gend);
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
          A pref[NS > 0 ? NS : 1];
#pragma unroll
          for (int s = 0; s < NS; ++s) pref[s] = acc_add_v(sacc[s], (int64_t)row <= next_end ? sv[s] : T(0));
          warp_sum_some<(NS > 0 ? NS : 1)>(pref);
          if (lane == 0)
#pragma unroll
            for (int s = 0; s < NS; ++s) rec[(size_t)ec.kn * M + C::smap(s)] = pref[s];
          ++ec.kn;
          next_end = ec.pos(P.gend);
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) sacc[s] = acc_add_v(sacc[s], sv[s]);
      };
      // e (and W) at the prefetched rows
      T pe[SR], pw[SR];
#pragma unroll
      for (int r = 0; r < SR; ++r) {
        const int row = pf.prow[r];
        pe[r] = row == INT_MAX ? T(0) : ld_hint(e + row, keep);
        pw[r] = (MODEL == 1 && row != INT_MAX) ? ld_hint(w2 + row, keep) : T(0);
      }
#pragma unroll
      for (int r = 0; r < SR; ++r)
        if (sa + 32 * r < sb) round(pf.prow[r], pf.pval[r], pe[r], pw[r], min(32, sb - sa - 32 * r));
      for (int base = sa + 32 * SR; base < sb; base += 32) {
        const int i = base + lane;
        const bool valid = i < sb;
        const int row = valid ? ld_hint(ri + i, strm) : INT_MAX;
        const T x = valid ? (vals ? ld_stream(vals + i, strm) : T(1)) : T(0);
        const T ev = valid ? ld_hint(e + row, keep) : T(0);
        const T wv = (MODEL == 1 && valid) ? ld_hint(w2 + row, keep) : T(0);
        round(row, x, ev, wv, min(32, sb - base));
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) tot[C::smap(s)] = sacc[s];  // lane partials, reduced below
      // warp totals, then the ends after the last nonzero of the range see them
      warp_sum_some<M>(tot);
      for (; ec.kn < pf.k_hi; ++ec.kn)
        if (lane == 0)
#pragma unroll
          for (int s = 0; s < NS; ++s) rec[(size_t)ec.kn * M + C::smap(s)] = tot[C::smap(s)];
    }
  } else {
    warp_sum_some<M>(tot);
  }
}

// Conditional update (Section 2.4) of eta += x_j * applied and e = exp(eta)
// on the rows of warps [w_lo, w_hi): the CSC nonzeros of column j in those
// warps' rows, or the dense row range [r_lo, r_hi).  delta is applied as
// float-float in the FP32 mode.  Every thread of the block takes part.
template <int LAYOUT, typename T>
__device__ __forceinline__ void cta_update(const CcdParams& P, int j, int w_lo, int w_hi, int64_t r_lo,
                                           int64_t r_hi, double applied, ff delta) {
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  if (LAYOUT == 0) {
    const int nw1 = P.nwarps + 1;
    const int64_t cb = P.col_ptr[j];
    const int32_t* ri = P.row_idx + cb;
    const T* vals = P.values ? reinterpret_cast<const T*>(P.values) + cb : nullptr;
    const int a = P.woff[(size_t)j * nw1 + w_lo];
    const int b = P.woff[(size_t)j * nw1 + w_hi];
    if constexpr (sizeof(T) == 4) {
      // loads batched 8 deep: the row indices, then eta, then the stores
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
      for (int64_t i = r_lo + tid; i < r_hi; i += NT)
        eta_axpy(reinterpret_cast<float2*>(P.eta), reinterpret_cast<float*>(P.e), i, (float)xcol[i], delta);
    } else {
      for (int64_t i = r_lo + tid; i < r_hi; i += NT)
        eta_axpy(reinterpret_cast<double*>(P.eta), reinterpret_cast<double*>(P.e), i, (double)xcol[i], applied);
    }
  }
}

// The same update restricted to the rows of one warp (CSC: the nonzeros of
// column j between the warp's offsets; dense: rows [r_lo, r_hi)).  Only the
// calling warp's lanes take part; a __syncwarp after it makes the new e
// visible to the warp's own pass.  In a batched cross-validation fit the
// subjects of the fit's fold keep e = 0 (their eta is still updated: it is
// x_i^T beta for the held-out score).
template <int LAYOUT, typename T>
__device__ __forceinline__ void warp_update(const CcdParams& P, int j, int gw, int64_t r_lo, int64_t r_hi,
                                            double applied, ff delta) {
  const int lane = threadIdx.x & 31;
  if (LAYOUT == 0) {
    const int nw1 = P.nwarps + 1;
    const int64_t cb = P.col_ptr[j];
    const int32_t* ri = P.row_idx + cb;
    const T* vals = P.values ? reinterpret_cast<const T*>(P.values) + cb : nullptr;
    const int a = P.woff[(size_t)j * nw1 + gw];
    const int b = P.woff[(size_t)j * nw1 + gw + 1];
    if constexpr (sizeof(T) == 4) {
      float2* etap = reinterpret_cast<float2*>(P.eta);
      float* ep = reinterpret_cast<float*>(P.e);
      for (int i0 = a; i0 < b; i0 += 4 * 32) {
        int rr[4];
        float xx[4];
        float2 qq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * 32 + lane;
          rr[u] = i < b ? ri[i] : -1;
          xx[u] = i < b ? (vals ? (float)vals[i] : 1.f) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) qq[u] = rr[u] >= 0 ? etap[rr[u]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (rr[u] < 0) continue;
          const ff v = ff_add({qq[u].x, qq[u].y}, ff_mul_f(delta, xx[u]));
          etap[rr[u]] = make_float2(v.hi, v.lo);
          const float ev = expf(v.hi);
          // subjects held out of a cross-validation fit stay out of every risk set
          ep[rr[u]] = (P.fold_id && P.fold_id[rr[u]] == P.fold) ? 0.f : fmaf(ev, v.lo, ev);
        }
      }
    } else {
      for (int i = a + lane; i < b; i += 32) {
        const int r = ri[i];
        eta_axpy(reinterpret_cast<double*>(P.eta), reinterpret_cast<double*>(P.e), r,
                 vals ? (double)vals[i] : 1.0, applied, P.fold_id && P.fold_id[r] == P.fold);
      }
    }
  } else {
    const T* xcol = reinterpret_cast<const T*>(P.X) + (size_t)j * P.ld;
    if constexpr (sizeof(T) == 4) {
      // loads batched 4 deep (x, then eta), then the stores: the element
      // arithmetic is eta_axpy's, only more loads are in flight
      float2* etap = reinterpret_cast<float2*>(P.eta);
      float* ep = reinterpret_cast<float*>(P.e);
      for (int64_t i0 = r_lo + lane; i0 < r_hi; i0 += 4 * 32) {
        float xx[4];
        float2 qq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xx[u] = i0 + 32 * u < r_hi ? (float)xcol[i0 + 32 * u] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) qq[u] = i0 + 32 * u < r_hi ? etap[i0 + 32 * u] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + 32 * u;
          if (i >= r_hi) continue;
          const ff v = ff_add({qq[u].x, qq[u].y}, ff_mul_f(delta, xx[u]));
          etap[i] = make_float2(v.hi, v.lo);
          const float ev = expf(v.hi);
          ep[i] = (P.fold_id && P.fold_id[i] == P.fold) ? 0.f : fmaf(ev, v.lo, ev);
        }
      }
    } else {
      for (int64_t i = r_lo + lane; i < r_hi; i += 32)
        eta_axpy(reinterpret_cast<double*>(P.eta), reinterpret_cast<double*>(P.e), i, (double)xcol[i], applied,
                 P.fold_id && P.fold_id[i] == P.fold);
    }
  }
  __syncwarp();
}

// Pieces of the objective at the current beta (Section 2.4): lin =
// sum_j beta_j delta^T X_j (= delta^T eta) and pen = -penalty(beta), summed
// by one warp in a fixed order.  Coordinate oq (if >= 0) is taken as ob
// instead of its stored value.
__device__ __forceinline__ void warp_lin_pen(const CcdParams& P, int oq, double ob, double& lin, double& pen) {
  const int lane = threadIdx.x & 31;
  lin = 0.0;
  pen = 0.0;
  for (int q0 = 0; q0 < P.p; q0 += 32 * 4) {
    double bq[4], dq[4], fq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + 32 * u + lane;
      bq[u] = q < P.p ? (q == oq ? ob : __ldcg(P.beta + q)) : 0.0;
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

// Fixed-order sums by one warp of NV payload vectors laid out [NV][G]
// (every lane gets the totals).
template <typename A, int NV>
__device__ __forceinline__ void warp_fold_slots(const uint64_t* soa, int G, A (&out)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < NV; ++m) acc_zero(out[m]);
  for (int q0 = 0; q0 < G; q0 += 32 * 5) {
    uint64_t v[NV][5];
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      const int q = q0 + 32 * u + lane;
#pragma unroll
      for (int m = 0; m < NV; ++m) v[m][u] = q < G ? __ldcg(soa + (size_t)m * G + q) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 5; ++u)
#pragma unroll
      for (int m = 0; m < NV; ++m) out[m] = acc_add(out[m], unpack8<A>(v[m][u]));
  }
  warp_sum_n<NV>(out);
}

// Steps 3-4 for the group ends [kc_lo, kc_hi) of one CTA range: the risk-set
// sums at end k are s_base[w][.] + rec[k][.] (w = warp holding the end,
// relative to wbase), plus for Fine-Gray the suffix of the censoring-weighted
// sums times G(t_k) (Eqs. fg_g, fg_h).  Each warp leaves its sums of
// d_k G_k, d_k (H_k - G_k^2) and (if eval) d_k log den_k in s_red[w]; returns
// the number of warps that wrote.  Few ends: one end per thread in FP64
// (latency-bound); many ends: float-float (FP64 throughput on GB300 is ~1/70
// of FP32).  The caller synchronises the block before reading s_red.
template <int MODEL, typename A>
__device__ __forceinline__ int cta_transform(const CcdParams& P, bool eval, int kc_lo, int kc_hi, int wbase,
                                             const A (*s_base)[MODEL == 0 ? 3 : 6], const A* s_tot, const A* rec,
                                             A (*s_red)[3]) {
  constexpr int M = MODEL == 0 ? 3 : 6;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int NT = blockDim.x;
  const int nends = kc_hi - kc_lo;
  double pg1 = 0.0, pg2 = 0.0, pl = 0.0;
  int nw_red;
  if (nends <= NT) {
    nw_red = (nends + 31) >> 5;
    if (tid < nends) {
      const int k = kc_lo + tid;
      const int d = P.dk[k];
      if (d != 0) {
        const int wl = (int)((P.gend[k] >> 5) / P.wpw) - wbase;
        double Pm[M];
#pragma unroll
        for (int m = 0; m < M; ++m) Pm[m] = acc_to_d(acc_add(s_base[wl][m], rec[(size_t)k * M + m]));
        double den = Pm[0], num1 = Pm[1], num2 = Pm[2];
        if (MODEL == 1) {
          const double g = P.Gk[k];
          den += g * (acc_to_d(s_tot[3]) - Pm[3]);
          num1 += g * (acc_to_d(s_tot[4]) - Pm[4]);
          num2 += g * (acc_to_d(s_tot[5]) - Pm[5]);
        }
        const double inv = 1.0 / den;
        const double Gr = num1 * inv, H = num2 * inv;
        pg1 = d * Gr;
        pg2 = d * (H - Gr * Gr);
        if (eval) pl = d * log(den);
      }
    }
    if (w < nw_red) {
      const A f1 = warp_sum(acc_from_d(pg1, (A*)nullptr)), f2 = warp_sum(acc_from_d(pg2, (A*)nullptr));
      const A fl = warp_sum(acc_from_d(pl, (A*)nullptr));
      if (lane == 0) { s_red[w][0] = f1; s_red[w][1] = f2; s_red[w][2] = fl; }
    }
  } else {
    nw_red = NT >> 5;
    A fg1, fg2;
    acc_zero(fg1);
    acc_zero(fg2);
    for (int k = kc_lo + tid; k < kc_hi; k += NT) {
      const int d = P.dk[k];
      if (d == 0) continue;
      const int wl = (int)((P.gend[k] >> 5) / P.wpw) - wbase;
      A Pm[M];
#pragma unroll
      for (int m = 0; m < M; ++m) Pm[m] = acc_add(s_base[wl][m], rec[(size_t)k * M + m]);
      A den = Pm[0], num1 = Pm[1], num2 = Pm[2];
      if (MODEL == 1) {
        const float2 gf = P.Gkff[k];
        const A g = acc_base<A>(P.Gk[k], ff{gf.x, gf.y});
        den = acc_add(den, acc_mul(g, acc_add(s_tot[3], acc_neg(Pm[3]))));
        num1 = acc_add(num1, acc_mul(g, acc_add(s_tot[4], acc_neg(Pm[4]))));
        num2 = acc_add(num2, acc_mul(g, acc_add(s_tot[5], acc_neg(Pm[5]))));
      }
      const A inv = acc_recip(den);
      const A Gr = acc_mul(num1, inv);
      const A H = acc_mul(num2, inv);
      fg1 = acc_add(fg1, acc_scale(Gr, d));
      fg2 = acc_add(fg2, acc_scale(acc_add(H, acc_neg(acc_mul(Gr, Gr))), d));
      if (eval) pl += (double)d * log(acc_to_d(den));
    }
    const A f1 = warp_sum(fg1), f2 = warp_sum(fg2);
    const A fl = warp_sum(acc_from_d(pl, (A*)nullptr));
    if (lane == 0) { s_red[w][0] = f1; s_red[w][1] = f2; s_red[w][2] = fl; }
  }
  return nw_red;
}

}  // namespace ccdk
}  // namespace survgpu
