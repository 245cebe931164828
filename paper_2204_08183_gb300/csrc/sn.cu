// Sparse-numerator form of the Cox CCD (not in the paper; an algebraic
// rearrangement of Eqs. cox_g / cox_h that gives the same l'_j and l''_j).
//
// With subjects in decreasing time, tie groups k (last subject e_k, d_k
// events), Den_k = sum_{r <= e_k} e_r and a_t = x_t e_{i_t} over the
// nonzeros t of column j (rows increasing, group g_t):
//   sum_k d_k N1_k / Den_k     = sum_t a_t Lambda(g_t),
//   sum_k d_k N2_k / Den_k     = sum_t x_t a_t Lambda(g_t),
//   sum_k d_k (N1_k / Den_k)^2 = sum_t C_t^2 [W(g_{t+1}) - W(g_t)],
// Lambda(g) = sum_{k >= g} d_k / Den_k, W(g) = sum_{k < g} d_k / Den_k^2,
// C_t = a_1 + ... + a_t, g_{m+1} = K.  Den, Lambda and W depend on e only,
// so they are rebuilt only after a nonzero step; every coordinate then costs
// O(nnz_j) instead of a pass over all N subjects.
//
// Five kernels per coordinate j, captured once per sweep as a CUDA graph
// with programmatic dependent launch (every kernel reads the control line
// and returns early when it has nothing to do):
//   k_sn_den_a   each warp applies the step of coordinate j - 1 to its rows
//                (eta, e); if the risk sets are stale it runs the row pass
//                for e alone (prefix at the warp's group ends) and the CTA
//                publishes its warp offsets and aggregate
//   k_sn_den_b   (stale only) Den_k at each group end, v1 = d_k / Den_k,
//                v2 = d_k / Den_k^2, per-CTA sums of v1, v2, d_k log Den_k
//   k_sn_lam     (stale only) Lambda (suffix of v1) and W (prefix of v2) as
//                float-float, and sum_k d_k log Den_k
//   k_sn_col_a   column j in chunks: chunk totals of a, and the partial
//                sums S1 = sum a Lambda, S2 = sum x a Lambda
//   k_sn_col_b   chunk prefix, C_t, Q = sum C_t^2 dW; the last CTA takes
//                the Newton step exactly as the row-pass schedule does
// All sums run in a fixed order.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "graph_common.cuh"

namespace survgpu {
namespace {

using namespace ccdk;

constexpr int kSnPassThreads = 512;  // k_sn_den_a: the row-pass shape
constexpr int kSnThreads = 256;      // the other kernels
constexpr int kSnWarps = kSnThreads / 32;

__device__ __forceinline__ double warp_sum_d(double v) { return warp_sum(v); }

// fixed-order block sum of one double (every thread gets it)
__device__ __forceinline__ double block_sum_d(double v, double* s_w) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) s_w[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_w[q];
  return t;
}

// fixed-order block sum of one float-float value (every thread gets it)
__device__ __forceinline__ ff block_sum_ff(ff v, ff* s_w) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) s_w[w] = v;
  __syncthreads();
  ff t = s_w[0];
  for (int q = 1; q < (int)(blockDim.x >> 5); ++q) t = ff_add(t, s_w[q]);
  return t;
}

// Exclusive prefix (thread order) of one value per thread, fixed shape:
// lane scans, then the warp totals in order.  *total gets the block total.
template <typename V>
__device__ __forceinline__ V block_excl_scan(V v, V* s_w, V* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  V incl = warp_inclusive_scan(v, lane);
  V ex = shfl_up(incl, 1);
  if (lane == 0) acc_zero(ex);
  __syncthreads();
  if (lane == 31) s_w[w] = incl;
  __syncthreads();
  V off, tot;
  acc_zero(off);
  acc_zero(tot);
  for (int q = 0; q < nw; ++q) {
    if (q < w) off = acc_add(off, s_w[q]);
    tot = acc_add(tot, s_w[q]);
  }
  *total = tot;
  return acc_add(off, ex);
}

// Exclusive suffix (sum over the threads after this one), fixed shape.
__device__ __forceinline__ double block_excl_suffix_d(double v, double* s_w) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  double incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double u = __shfl_down_sync(0xffffffffu, incl, d);
    if (lane + d < 32) incl += u;
  }
  double ex = __shfl_down_sync(0xffffffffu, incl, 1);
  if (lane == 31) ex = 0.0;
  __syncthreads();
  if (lane == 0) s_w[w] = incl;
  __syncthreads();
  double off = 0.0;
  for (int q = nw - 1; q > w; --q) off += s_w[q];
  return off + ex;
}

__global__ void k_sn_groups(const int32_t* gend, int32_t K, int64_t n, int32_t* grp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (gend[mid] >= i) hi = mid; else lo = mid + 1;
    }
    grp[i] = lo;
  }
}

// ------------------------------------------------------------- k_sn_den_a
template <bool MULTI>
__global__ void __launch_bounds__(kSnPassThreads, 2) k_sn_den_a(const __grid_constant__ CcdParams P, int j) {
  using A = ff;
  constexpr int M = 3;
  __shared__ A s_wtot[kMaxWarpsPerCta][M];
  __shared__ int s_go;
  __shared__ double s_applied;
  __shared__ float s_delta[2];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int WPC = P.wpc, c = blockIdx.x, G = P.G;
  const int64_t n = P.n;
  const int64_t nwords = (n + 31) >> 5;
  const int gw = c * WPC + w;
  const int64_t word_lo = min((int64_t)gw * P.wpw, nwords);
  const int64_t word_hi = min(word_lo + P.wpw, nwords);
  const int64_t row_lo = word_lo * 32, row_hi = min(word_hi * 32, n);
  const int q = j == 0 ? P.p - 1 : j - 1;
  // the warp's group ends (static); no column is walked by this pass
  PassPrefetch<float, 4> pf;
  pf.k_lo = P.wk0[gw];
  pf.k_hi = P.wk0[gw + 1];
  pf.kreg = pf.k_lo + lane < pf.k_hi ? P.gend[pf.k_lo + lane] : INT_MAX;
  pf.sa = pf.sb = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    pf.prow[r] = INT_MAX;
    pf.pval[r] = 0.f;
  }
  pdl_wait();
  if (tid == 0) {
    const CtlLine* L = &P.gctl->line[c % kRep];
    const int stop = __ldcg(&L->stop);
    s_applied = __ldcg(&L->applied);
    s_delta[0] = __ldcg(&L->delta_hi);
    s_delta[1] = __ldcg(&L->delta_lo);
    // 0: stopped; 1: update only; 2: update (if any) and rebuild
    s_go = stop ? 0 : ((__ldcg(&L->dirty) || s_applied != 0.0) ? 2 : 1);
  }
  __syncthreads();
  const int go = s_go;
  if (go == 0) return;
  if (s_applied != 0.0) warp_update<0, float>(P, q, gw, row_lo, row_hi, s_applied, ff{s_delta[0], s_delta[1]});
  if (go == 1) return;
  A* rec = reinterpret_cast<A*>(P.rec);
  A tot[M];
  warp_pass<0, 0, float, 4, 4, MULTI>(P, j, row_lo, row_hi, rec, tot, pf);
  pdl_launch_dependents();
  if (lane == 0) s_wtot[w][0] = tot[0];
  __syncthreads();
  if (w == 0) {
    A v[1];
    acc_zero(v[0]);
    if (lane < WPC) v[0] = s_wtot[lane][0];
    warp_scan_n<1>(v, lane);
    A ex = shfl_up(v[0], 1);
    if (lane == 0) acc_zero(ex);
    if (lane < WPC) P.wt[c * WPC + lane] = pack8(ex);
    const A t = shfl_idx(v[0], WPC - 1);
    if (lane < kRep) P.agg[(size_t)lane * G + c] = pack8(t);
  }
}

// the step in the control line says whether the risk sets were rebuilt
__device__ __forceinline__ bool sn_rebuilt(const CcdParams& P, int c, int* s_flag) {
  if (threadIdx.x == 0) {
    const CtlLine* L = &P.gctl->line[c % kRep];
    const int stop = __ldcg(&L->stop);
    *s_flag = !stop && (__ldcg(&L->dirty) || __ldcg(&L->applied) != 0.0);
  }
  __syncthreads();
  return *s_flag != 0;
}

// ------------------------------------------------------------- k_sn_den_b
__global__ void __launch_bounds__(kSnThreads) k_sn_den_b(const __grid_constant__ CcdParams P,
                                                          const __grid_constant__ SnParams S, int j) {
  __shared__ int s_flag;
  __shared__ double s_w[kSnWarps];
  __shared__ ff s_wf[kSnWarps];
  const int tid = threadIdx.x, c = blockIdx.x, G = P.G, WPC = P.wpc;
  const int kc_lo = P.wk0[c * WPC], kc_hi = P.wk0[(c + 1) * WPC];
  pdl_wait();
  if (!sn_rebuilt(P, c, &s_flag)) return;
  // aggregate of the CTAs before c (replica c mod kRep), fixed order
  const uint64_t* agg = P.agg + (size_t)(c % kRep) * G;
  ff pre = ff_zero();
  for (int qc = tid; qc < c; qc += kSnThreads) pre = ff_add(pre, unpack8<ff>(__ldcg(agg + qc)));
  const ff T_c = block_sum_ff(pre, s_wf);
  const ff* rec = reinterpret_cast<const ff*>(P.rec);
  double a1 = 0.0, a2 = 0.0, al = 0.0;
  for (int k = kc_lo + tid; k < kc_hi; k += kSnThreads) {
    const int wl = (int)((P.gend[k] >> 5) / P.wpw);
    const ff Pm = ff_add(ff_add(T_c, unpack8<ff>(__ldcg(P.wt + wl))), rec[(size_t)k * 3]);
    const double D = ff_to_d(Pm);
    const int d = P.dk[k];
    const double v1 = (double)d / D;
    const double v2 = v1 / D;
    S.den[k] = D;
    S.v1[k] = v1;
    S.v2[k] = v2;
    a1 += v1;
    a2 += v2;
    if (d) al += (double)d * log(D);
  }
  pdl_launch_dependents();
  a1 = block_sum_d(a1, s_w);
  a2 = block_sum_d(a2, s_w);
  al = block_sum_d(al, s_w);
  if (tid == 0) {
    S.part_den[c] = a1;
    S.part_den[G + c] = a2;
    S.part_den[2 * G + c] = al;
  }
}

// --------------------------------------------------------------- k_sn_lam
// CTA c owns the group ends of its rows [kc_lo, kc_hi); each thread takes a
// contiguous run of them.
__global__ void __launch_bounds__(kSnThreads) k_sn_lam(const __grid_constant__ CcdParams P,
                                                        const __grid_constant__ SnParams S, int j) {
  __shared__ int s_flag;
  __shared__ double s_w[kSnWarps];
  const int tid = threadIdx.x, lane = tid & 31, c = blockIdx.x, G = P.G, WPC = P.wpc;
  const int kc_lo = P.wk0[c * WPC], kc_hi = P.wk0[(c + 1) * WPC];
  pdl_wait();
  if (!sn_rebuilt(P, c, &s_flag)) return;
  // sum of v1 over the CTAs after c, of v2 over the CTAs before c
  double suf = 0.0, pre = 0.0;
  for (int qc = tid; qc < G; qc += kSnThreads) {
    if (qc > c) suf += __ldcg(S.part_den + qc);
    if (qc < c) pre += __ldcg(S.part_den + G + qc);
  }
  suf = block_sum_d(suf, s_w);
  pre = block_sum_d(pre, s_w);
  const int ne = kc_hi - kc_lo;
  const int per = (ne + kSnThreads - 1) / kSnThreads;
  const int lo = min(kc_lo + tid * per, kc_hi), hi = min(lo + per, kc_hi);
  double t1 = 0.0, t2 = 0.0;
  for (int k = lo; k < hi; ++k) {
    t1 += __ldcg(S.v1 + k);
    t2 += __ldcg(S.v2 + k);
  }
  // v1 of the runs after this thread's, v2 of the runs before (fixed order)
  const double after = block_excl_suffix_d(t1, s_w);
  double tot2 = 0.0;
  const double before = block_excl_scan(t2, s_w, &tot2);
  double run1 = suf + after;
  for (int k = hi - 1; k >= lo; --k) {
    run1 += __ldcg(S.v1 + k);
    const ff v = d_to_ff(run1);
    S.lam[k] = make_float2(v.hi, v.lo);
  }
  double run2 = pre + before;
  for (int k = lo; k < hi; ++k) {
    const ff v = d_to_ff(run2);
    S.W[k] = make_float2(v.hi, v.lo);
    run2 += __ldcg(S.v2 + k);
  }
  pdl_launch_dependents();
  if (c == G - 1 && tid == 0) {
    // W(K): everything (the last CTA's own total after its prefix)
    const ff v = d_to_ff(pre + tot2);
    S.W[P.K] = make_float2(v.hi, v.lo);
  }
  if (c == 0 && tid < 32) {
    double l = 0.0;
    for (int qc = lane; qc < G; qc += 32) l += __ldcg(S.part_den + 2 * G + qc);
    l = warp_sum_d(l);
    if (lane == 0) *S.ll_den = l;
  }
}

// -------------------------------------------------------------- column j
// Column j in chunks of at most kSnElems * kSnThreads nonzeros (the host
// sizes G2 for the longest column): thread entries and their tie groups do
// not depend on e, so they are loaded before the wait on the previous
// kernel; e, Lambda and W are gathered in one round trip after it.
constexpr int kSnElems = 8;

struct ColChunk {
  int64_t cb;  // first entry of column j
  int m;       // nonzeros of column j
  int lo, hi;  // this CTA's entries [lo, hi) (relative to cb)
};
__device__ __forceinline__ ColChunk col_chunk(const CcdParams& P, int G2, int j) {
  ColChunk r;
  r.cb = P.col_ptr[j];
  r.m = (int)(P.col_ptr[j + 1] - r.cb);
  const int ch = (r.m + G2 - 1) / G2;
  r.lo = min(blockIdx.x * ch, r.m);
  r.hi = min(r.lo + ch, r.m);
  return r;
}

__global__ void __launch_bounds__(kSnThreads) k_sn_col_a(const __grid_constant__ CcdParams P,
                                                          const __grid_constant__ SnParams S, int j) {
  __shared__ ff s_wf[kSnWarps];
  __shared__ int s_stop;
  const int tid = threadIdx.x, c = blockIdx.x, G2 = S.G2;
  const ColChunk ck = col_chunk(P, G2, j);
  const int32_t* ri = P.row_idx + ck.cb;
  const float* vals = P.values ? reinterpret_cast<const float*>(P.values) + ck.cb : nullptr;
  const float* e = reinterpret_cast<const float*>(P.e);
  // strided entries t = lo + tid + u * kSnThreads
  int r[kSnElems], g[kSnElems];
  float x[kSnElems];
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) {
    const int t = ck.lo + tid + u * kSnThreads;
    const bool ok = t < ck.hi;
    r[u] = ok ? ri[t] : -1;
    x[u] = ok ? (vals ? vals[t] : 1.f) : 0.f;
  }
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) g[u] = r[u] >= 0 ? __ldg(S.grp + r[u]) : 0;
  pdl_wait();
  if (tid == 0) s_stop = __ldcg(&P.gctl->line[c % kRep].stop);
  float ev[kSnElems];
  float2 L[kSnElems];
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) {
    ev[u] = r[u] >= 0 ? __ldcg(e + r[u]) : 0.f;
    L[u] = r[u] >= 0 ? __ldcg(S.lam + g[u]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (s_stop) return;
  ff ta = ff_zero(), s1 = ff_zero(), s2 = ff_zero();
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) {
    const float a = x[u] * ev[u];
    const ff aL = ff_mul_f(ff{L[u].x, L[u].y}, a);
    ta = ff_add_f(ta, a);
    s1 = ff_add(s1, aL);
    s2 = ff_add(s2, ff_mul_f(aL, x[u]));
  }
  pdl_launch_dependents();
  ta = block_sum_ff(ta, s_wf);
  s1 = block_sum_ff(s1, s_wf);
  s2 = block_sum_ff(s2, s_wf);
  if (tid == 0) {
    S.part_col[c] = pack8(ta);
    S.part_col[G2 + c] = pack8(s1);
    S.part_col[2 * G2 + c] = pack8(s2);
  }
}

__global__ void __launch_bounds__(kSnThreads) k_sn_col_b(const __grid_constant__ CcdParams P,
                                                          const __grid_constant__ SnParams S, int j) {
  __shared__ ff s_wf[kSnWarps];
  __shared__ ff s_red[3];
  __shared__ int s_last;
  __shared__ double s_lin[2];
  __shared__ double s_next[4];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, c = blockIdx.x, G2 = S.G2;
  const bool eval = j == 0;
  const ColChunk ck = col_chunk(P, G2, j);
  const int32_t* ri = P.row_idx + ck.cb;
  const float* vals = P.values ? reinterpret_cast<const float*>(P.values) + ck.cb : nullptr;
  const float* e = reinterpret_cast<const float*>(P.e);
  GraphCtl* ctl = P.gctl;
  const int K = P.K;
  // each thread a contiguous run of the chunk (at most kSnElems entries);
  // gn is the group of the entry after each one (K after the column's last)
  const int len = ck.hi - ck.lo;
  const int per = (len + kSnThreads - 1) / kSnThreads;
  const int lo = ck.lo + min(tid * per, len), hi = min(lo + per, ck.hi);
  int r[kSnElems], g[kSnElems], gn[kSnElems];
  float x[kSnElems];
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) {
    const int t = lo + u;
    const bool ok = t < hi;
    r[u] = ok ? ri[t] : -1;
    x[u] = ok ? (vals ? vals[t] : 1.f) : 0.f;
  }
  const int r_after = hi < ck.m ? ri[hi] : -1;
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) g[u] = r[u] >= 0 ? __ldg(S.grp + r[u]) : K;
  const int g_after = r_after >= 0 ? __ldg(S.grp + r_after) : K;
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) gn[u] = u + 1 < kSnElems && lo + u + 1 < hi ? g[u + 1] : g_after;
  pdl_wait();
  LineView lv;
  if (tid == 0) {
    lv = load_line(ctl, c);
    s_last = lv.stop;
  }
  float ev[kSnElems];
  float2 w0[kSnElems], w1[kSnElems];
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) {
    const bool ok = r[u] >= 0;
    ev[u] = ok ? __ldcg(e + r[u]) : 0.f;
    const bool step = ok && gn[u] != g[u];
    w0[u] = step ? __ldcg(S.W + g[u]) : make_float2(0.f, 0.f);
    w1[u] = step ? __ldcg(S.W + gn[u]) : make_float2(0.f, 0.f);
  }
  // chunk totals of the CTAs before c (fixed order)
  ff pre = ff_zero();
  for (int qc = tid; qc < c; qc += kSnThreads) pre = ff_add(pre, unpack8<ff>(__ldcg(S.part_col + qc)));
  __syncthreads();
  if (s_last) return;  // the fit has stopped
  const ff base = block_sum_ff(pre, s_wf);
  ff run = ff_zero();
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) run = ff_add_f(run, x[u] * ev[u]);
  ff chunk_tot;
  ff C = ff_add(base, block_excl_scan(run, s_wf, &chunk_tot));
  ff Q = ff_zero();
#pragma unroll
  for (int u = 0; u < kSnElems; ++u) {
    C = ff_add_f(C, x[u] * ev[u]);
    if (r[u] >= 0 && gn[u] != g[u]) {
      const ff dW = ff_sub(ff{w1[u].x, w1[u].y}, ff{w0[u].x, w0[u].y});
      Q = ff_add(Q, ff_mul(ff_mul(C, C), dW));
    }
  }
  Q = block_sum_ff(Q, s_wf);
  if (tid == 0) {
    S.part_col[3 * G2 + c] = pack8(Q);
    unsigned prev;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&ctl->ticket) : "memory");
    s_last = prev == (unsigned)(G2 - 1);
  }
  pdl_launch_dependents();
  __syncthreads();
  if (!s_last) return;
  // ------------------------------- last CTA: the step of coordinate j
  if (w < 3) {
    // warp m sums vector m + 1 (S1, S2, Q) over the CTAs in a fixed order
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    ff acc = ff_zero();
    for (int qc = lane; qc < G2; qc += 32)
      acc = ff_add(acc, unpack8<ff>(__ldcg(S.part_col + (size_t)(w + 1) * G2 + qc)));
    acc = warp_sum(acc);
    if (lane == 0) s_red[w] = acc;
  } else if (w == 3 && eval) {
    double lin, pen;
    warp_lin_pen(P, -1, 0.0, lin, pen);
    if (lane == 0) {
      s_lin[0] = lin;
      s_lin[1] = pen;
    }
  } else if (w == 4 && lane == 0) {
    const int jn = j + 1 < P.p ? j + 1 : 0;
    s_next[0] = __ldcg(P.beta + jn);
    s_next[1] = __ldcg(P.width + jn);
    s_next[2] = P.pen[jn];
    s_next[3] = P.dTx[jn];
  }
  __syncthreads();
  if (w == 0) {
    const double s1 = ff_to_d(s_red[0]), s2 = ff_to_d(s_red[1]), qd = ff_to_d(s_red[2]);
    const double sum_dlog = eval ? __ldcg(S.ll_den) : 0.0;
    publish_step(P, j, lv, lv.dtx - s1, -(s2 - qd), eval, s_lin[0], s_lin[1], sum_dlog, s_next);
  }
}

cudaError_t capture_sn(const CcdParams& P, const SnParams& S, bool pdl, cudaStream_t cs, cudaGraph_t* g) {
  cudaError_t st = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (st != cudaSuccess) return st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cudaLaunchConfig_t ca = {};
  ca.gridDim = dim3(P.G);
  ca.blockDim = dim3(kSnPassThreads);
  ca.stream = cs;
  ca.attrs = attr;
  ca.numAttrs = 1;
  cudaLaunchConfig_t cb = ca;
  cb.blockDim = dim3(kSnThreads);
  cudaLaunchConfig_t cc = cb;
  cc.gridDim = dim3(S.G2);
  auto ka = S.multi ? k_sn_den_a<true> : k_sn_den_a<false>;
  cudaError_t lst = cudaSuccess;
  for (int j = 0; j < P.p && lst == cudaSuccess; ++j) {
    lst = cudaLaunchKernelEx(&ca, ka, P, j);
    if (lst == cudaSuccess) lst = cudaLaunchKernelEx(&cb, k_sn_den_b, P, S, j);
    if (lst == cudaSuccess) lst = cudaLaunchKernelEx(&cb, k_sn_lam, P, S, j);
    if (lst == cudaSuccess) lst = cudaLaunchKernelEx(&cc, k_sn_col_a, P, S, j);
    if (lst == cudaSuccess) lst = cudaLaunchKernelEx(&cc, k_sn_col_b, P, S, j);
  }
  st = cudaStreamEndCapture(cs, g);
  return lst != cudaSuccess ? lst : st;
}

}  // namespace

cudaError_t sn_groups(const int32_t* gend, int32_t K, int64_t n, int32_t* grp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  k_sn_groups<<<(unsigned)g, 256, 0, s>>>(gend, K, n, grp);
  return cudaGetLastError();
}

cudaError_t run_sn_graph(const CcdParams& P, const SnParams& S, cudaStream_t s, GraphCache* gc, cudaEvent_t t0,
                         int* replays, int* launches) {
  static_assert(sizeof(SnParams) <= sizeof(GraphCache::key2), "graph cache key too small");
  *replays = 0;
  *launches = 0;
  GraphCache local;
  struct LocalGuard {
    GraphCache* g;
    ~LocalGuard() { graph_cache_free(g); }
  } guard{gc ? nullptr : &local};
  if (!gc) gc = &local;
  cudaError_t st;
  if ((st = graph_cache_prepare(gc)) != cudaSuccess) return st;
  const bool pdl = !P.no_pdl;
  const int mlp = 1000 + (pdl ? 1 : 0);
  unsigned char key2[sizeof(GraphCache::key2)] = {};
  std::memcpy(key2, &S, sizeof(S));
  if (!gc->exec || gc->mlp != mlp || std::memcmp(&gc->key, &P, sizeof(P)) != 0 ||
      std::memcmp(gc->key2, key2, sizeof(key2)) != 0) {
    if (gc->exec) {
      cudaGraphExecDestroy(gc->exec);
      gc->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    st = capture_sn(P, S, pdl, gc->cs, &g);
    if (st == cudaSuccess) st = cudaGraphInstantiate(&gc->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != cudaSuccess) {
      gc->exec = nullptr;
      return st;
    }
    gc->key = P;
    std::memcpy(gc->key2, key2, sizeof(key2));
    gc->mlp = mlp;
  }
  return replay_until_stop(P, s, gc, t0, 5 * P.p, replays, launches);
}

}  // namespace survgpu
