// Device helpers shared by the survgpu kernels (sm_103a).
//
// * float-float ("ff") arithmetic: an unevaluated sum hi + lo of two floats,
//   built from Knuth's TwoSum and the FMA form of Dekker's TwoProd.  It gives
//   about 44-48 significant bits with FP32 instructions only; GB300's FP64
//   pipe is far too slow for per-element or per-group use.  The __f*_rn
//   intrinsics keep the compiler from contracting the error terms into FMAs.
// * acquire/release flag access and a bounded wait used by the grid-wide
//   exchange of the persistent CCD kernel.  Every wait gives up after a
//   wall-clock limit read from %globaltimer and raises an error word instead
//   of spinning forever.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace survgpu {

// ------------------------------------------------------------------ ff type
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_zero() { return {0.f, 0.f}; }

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float err = __fsub_rn(b, __fsub_rn(s, a));
  return {s, err};
}

// accurate ff + ff (two TwoSums, renormalised)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  ff t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// ff + float
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

// ff * float (exact product of the leading parts via FMA)
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a / b with two correction steps (long division on the leading parts)
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  ff r = ff_sub(a, ff_mul_f(b, q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = ff_sub(r, ff_mul_f(b, q2));
  float q3 = __fdiv_rn(r.hi, b.hi);
  ff q = fast_two_sum(q1, q2);
  return ff_add_f(q, q3);
}

__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff d_to_ff(double d) {
  float hi = (float)d;
  float lo = (float)(d - (double)hi);
  return {hi, lo};
}

// ------------------------------------------------------------ accumulators
// Acc<float> is ff, Acc<double> is double: one code path for both precision
// modes of the kernels.
template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = ff; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ void acc_zero(ff& a) { a = ff_zero(); }
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ ff acc_add(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_add_v(ff a, float v) { return ff_add_f(a, v); }
__device__ __forceinline__ double acc_add_v(double a, double v) { return a + v; }
__device__ __forceinline__ double acc_to_d(ff a) { return ff_to_d(a); }
__device__ __forceinline__ double acc_to_d(double a) { return a; }
__device__ __forceinline__ ff acc_to_ff(ff a) { return a; }
__device__ __forceinline__ ff acc_to_ff(double a) { return d_to_ff(a); }
__device__ __forceinline__ ff acc_neg(ff a) { return ff_neg(a); }
__device__ __forceinline__ double acc_neg(double a) { return -a; }

__device__ __forceinline__ ff shfl_down(ff a, int d) {
  return {__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ double shfl_down(double a, int d) { return __shfl_down_sync(0xffffffffu, a, d); }
__device__ __forceinline__ ff shfl_up(ff a, int d) {
  return {__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ double shfl_up(double a, int d) { return __shfl_up_sync(0xffffffffu, a, d); }
__device__ __forceinline__ ff shfl_idx(ff a, int s) {
  return {__shfl_sync(0xffffffffu, a.hi, s), __shfl_sync(0xffffffffu, a.lo, s)};
}
__device__ __forceinline__ double shfl_idx(double a, int s) { return __shfl_sync(0xffffffffu, a, s); }

// Fixed-shape tree reduction over the 32 lanes (result broadcast to all
// lanes).  The order of additions does not depend on timing.  The bodies are
// out of line: the kernels call them from dozens of sites, and inlining every
// copy made the once-per-coordinate code outgrow the SM's instruction cache.
static __device__ __noinline__ ff warp_sum_ff(ff v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = ff_add(v, shfl_down(v, d));
  return shfl_idx(v, 0);
}
static __device__ __noinline__ double warp_sum_dd(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return __shfl_sync(0xffffffffu, v, 0);
}
// Plain FP32 / FP64 sum over the lanes, same tree shape (result in every lane).
__device__ __forceinline__ float warp_sum_t(float v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ double warp_sum_t(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ ff warp_sum(ff v) { return warp_sum_ff(v); }
__device__ __forceinline__ double warp_sum(double v) { return warp_sum_dd(v); }

// N independent sums with the same tree shape as warp_sum, interleaved
// level by level so that their shuffles and adds overlap (inline; for the
// latency-bound once-per-coordinate code).  Results broadcast to all lanes.
template <int N>
__device__ __forceinline__ void warp_sum_n(ff (&v)[N]) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    ff u[N];
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = shfl_down(v[i], d);
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = ff_add(v[i], u[i]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = shfl_idx(v[i], 0);
}
template <int N>
__device__ __forceinline__ void warp_sum_n(double (&v)[N]) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    double u[N];
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = __shfl_down_sync(0xffffffffu, v[i], d);
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] += u[i];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = __shfl_sync(0xffffffffu, v[i], 0);
}

// The same sums where register pressure matters: interleaved up to three
// at a time, one out-of-line tree each beyond that (identical results).
template <int N, typename A>
__device__ __forceinline__ void warp_sum_some(A (&v)[N]) {
  if constexpr (N <= 3) {
    warp_sum_n<N>(v);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = warp_sum(v[i]);
  }
}

// Sums of N values over the 32 lanes (N a power of two, 2..32) by recursive
// halving: at distance d = 16, 8, ... each lane keeps half of its values
// and adds the partner's copy of that half, so N values cost N - 1 + 5 -
// log2(N) float-float additions instead of 5 N for N separate trees.  On
// return v[0] holds the total of component warp_rs_component<N>(lane) in
// every lane (lanes that differ only in the low 5 - log2(N) bits hold the
// same component).  Fixed order: the result does not depend on timing.
template <int N>
__device__ __forceinline__ int warp_rs_component(int lane) {
  int c = 0;
#pragma unroll
  for (int d = 16, h = N / 2; h >= 1; d >>= 1, h >>= 1)
    if (lane & d) c += h;
  return c;
}
template <int N>
__device__ __forceinline__ int warp_rs_lane(int comp) {
  int l = 0;
#pragma unroll
  for (int d = 16, h = N / 2; h >= 1; d >>= 1, h >>= 1)
    if (comp & h) l |= d;
  return l;
}
template <int N>
__device__ __forceinline__ void warp_reduce_scatter(ff (&v)[N], int lane) {
  static_assert(N >= 2 && N <= 32 && (N & (N - 1)) == 0, "N: a power of two");
  int d = 16;
#pragma unroll
  for (int h = N / 2; h >= 1; h >>= 1, d >>= 1) {
    const bool up = (lane & d) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const ff keep = up ? v[i + h] : v[i];
      const ff give = up ? v[i] : v[i + h];
      const ff got = {__shfl_xor_sync(0xffffffffu, give.hi, d), __shfl_xor_sync(0xffffffffu, give.lo, d)};
      v[i] = up ? ff_add(got, keep) : ff_add(keep, got);
    }
  }
#pragma unroll
  for (; d >= 1; d >>= 1) {
    const ff got = {__shfl_xor_sync(0xffffffffu, v[0].hi, d), __shfl_xor_sync(0xffffffffu, v[0].lo, d)};
    v[0] = (lane & d) ? ff_add(got, v[0]) : ff_add(v[0], got);
  }
}

// N independent inclusive scans over the lanes (Hillis-Steele, fixed
// shape), interleaved level by level.
template <int N>
__device__ __forceinline__ void warp_scan_n(ff (&v)[N], int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    ff u[N];
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = shfl_up(v[i], d);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (lane >= d) v[i] = ff_add(v[i], u[i]);
  }
}
template <int N>
__device__ __forceinline__ void warp_scan_n(double (&v)[N], int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    double u[N];
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = __shfl_up_sync(0xffffffffu, v[i], d);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (lane >= d) v[i] += u[i];
  }
}

// Inclusive scan over lanes (Hillis-Steele, fixed shape).
static __device__ __noinline__ ff warp_scan_ff(ff v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    ff u = shfl_up(v, d);
    if (lane >= d) v = ff_add(v, u);
  }
  return v;
}
static __device__ __noinline__ double warp_scan_dd(double v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    double u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  return v;
}
__device__ __forceinline__ ff warp_inclusive_scan(ff v, int lane) { return warp_scan_ff(v, lane); }
__device__ __forceinline__ double warp_inclusive_scan(double v, int lane) { return warp_scan_dd(v, lane); }

// ------------------------------------------------------ L2 cache policies
// e (and W) are re-read by every coordinate's pass and should stay in L2;
// column data is read once per sweep and should not push them out.
__device__ __forceinline__ uint64_t l2_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Loads with an L2 policy.  The "memory" clobber keeps loads of data this
// warp has just written (e after the update) behind those writes.
__device__ __forceinline__ void ld4_hint(const float* p, uint64_t pol, float (&v)[4]) {
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
               : "l"(p), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void ld4_hint(const double* p, uint64_t pol, double (&v)[2]) {
  asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v[0]), "=d"(v[1])
               : "l"(p), "l"(pol)
               : "memory");
}
__device__ __forceinline__ float ld_hint(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ double ld_hint(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ int ld_hint(const int* p, uint64_t pol) {
  int v;
  asm("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
// column data (never written while a fit runs): no ordering needed
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

// ---------------------------------------------------------- flags / waits
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// Device error bits (also reported to the host in surv_fit_info).
enum : unsigned {
  DEV_ERR_TIMEOUT = 1u,      // a grid exchange wait gave up
  DEV_ERR_ABORT = 2u,        // a test-only abort request was honoured
};

}  // namespace survgpu
