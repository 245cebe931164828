// Per-coordinate CCD schedule (Sections 2.4 and 2.7): two kernels per
// coordinate, one sweep of them captured once as a CUDA graph and replayed
// until the device reports that the fit has stopped.
//
//   k_pass(j)   CTA c reads the step of coordinate q = j - 1 (line c % kRep),
//               each warp applies eta += x_q * step and e = exp(eta) to its
//               own rows, then runs the row pass (step 2) of coordinate j
//               over those rows and the CTA publishes its warp totals and its
//               aggregate (the latter in kRep replicas).
//   k_trans(j)  every CTA sums the aggregates of the CTAs before it (its
//               exclusive prefix) in a fixed order, transforms its group ends
//               (steps 3-4) and publishes three partial sums.  The last CTA
//               to finish (atomic ticket; nobody waits for it) sums the
//               partials in a fixed order, takes the FP64 Newton step of
//               Section 2.4, stores beta_j and its trust-region width, on
//               j = 0 evaluates the objective and the stopping rule, and
//               publishes the step for k_pass(j + 1).
//
// Kernel boundaries order every producer before its consumers: no kernel
// waits on another CTA.  A warp only reads and writes eta / e on its own
// rows, so the update of q needs no barrier before the pass.  Launches use
// programmatic dependent launch: loads of static tables are issued before
// griddepcontrol.wait, which hides most of the launch gap.
//
// Batched fits (cross-validation x lambda path, Section 2.8): the same two
// kernels run every fit at once, fit f on blockIdx.y with its own
// parameters (CcdParams::fits[f], copied to shared memory at the start of
// each CTA).  Fits stop independently; each one counts itself into a device
// counter when it stops, and the host replays the sweep until all have.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "graph_common.cuh"

namespace survgpu {
namespace {

using namespace ccdk;

// Pass kernel shape: 512 threads, two CTAs per SM (64 registers a thread):
// tiles of 4 16-byte loads per array per lane (2 for Fine-Gray, whose six
// running sums take the registers), 4 rounds of the column's nonzeros
// prefetched.  Measured at N = 10^7 against one CTA of 16 warps per
// SM, and against staging e in shared memory with bulk copies (whole SM or
// per warp), this shape was the fastest.
template <int MODEL, int LAYOUT>
struct GCfg {
  static constexpr int NT = 512;
  static constexpr int MINB = 2;
  static constexpr int U = (MODEL == 1 && LAYOUT == 1) ? 1 : (MODEL == 1 ? 2 : 4);
  static constexpr int SR = 4;
};
constexpr int kTransThreads = 256;
constexpr int kTransWarps = kTransThreads / 32;

// Fill every control line for the first coordinate of a fit (of fit
// blockIdx.y in a batched launch).
__global__ void k_graph_init(const __grid_constant__ CcdParams P0) {
  const CcdParams& P = P0.fits ? P0.fits[blockIdx.y] : P0;
  const int r = threadIdx.x;
  if (r >= kRep) return;
  CtlLine* L = &P.gctl->line[r];
  L->stop = 0;
  L->nevals = 0;
  L->applied = 0.0;
  L->delta_hi = 0.f;
  L->delta_lo = 0.f;
  L->beta = P.beta[0];
  L->width = P.width[0];
  L->pen = P.pen[0];
  L->dtx = P.dTx[0];
  L->f_prev = 0.0;
  L->passes = 0;
  L->eta_updates = 0;
  L->dirty = 1;
  L->j0 = 0;
  L->q = -1;
  L->batches = 0;
}

// MULTI selects the group-end handling for warps that hold many ends (see
// warp_pass); the host picks it when the tie groups outnumber the warps.
// TW picks the tile shape: 0 the configured one, 1 half the 16-byte loads of
// e per lane a tile, 2 half the rounds of nonzeros loaded together (twice
// the loads spilled at the 64-register cap).
template <int MODEL, int LAYOUT, typename T, bool BATCH, bool MULTI, int TW = 0>
__global__ void __launch_bounds__(GCfg<MODEL, LAYOUT>::NT, GCfg<MODEL, LAYOUT>::MINB)
    k_pass(const __grid_constant__ CcdParams P0, int j) {
  using A = typename AccOf<T>::type;
  using C = Cfg<MODEL, LAYOUT, T>;
  constexpr int M = C::M;
  __shared__ A s_wtot[kMaxWarpsPerCta][M];
  __shared__ int s_stop, s_dirty;
  __shared__ double s_applied;
  __shared__ float s_delta[2];
  __shared__ CcdParams s_fit;
  if (BATCH) load_fit(s_fit, P0);
  const CcdParams& P = BATCH ? s_fit : P0;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  const int WPC = P.wpc;
  const int c = blockIdx.x;
  const int G = P.G;
  const int64_t n = P.n;
  const int64_t nwords = (n + 31) >> 5;
  const int gw = c * WPC + w;
  const int64_t word_lo = min((int64_t)gw * P.wpw, nwords);
  const int64_t word_hi = min(word_lo + P.wpw, nwords);
  const int64_t row_lo = word_lo * 32;
  const int64_t row_hi = min(word_hi * 32, n);
  const int q = j == 0 ? P.p - 1 : j - 1;  // coordinate whose step is applied here

  // column j's first nonzeros and the warp's group ends do not depend on
  // earlier kernels: load them before waiting for the previous kernel
  using GC = GCfg<MODEL, LAYOUT>;
  constexpr int U = TW == 1 ? (GC::U > 1 ? GC::U / 2 : 1) : GC::U;
  constexpr int SR = TW == 2 ? GC::SR / 2 : GC::SR;
  PassPrefetch<T, SR> pf;
  pass_prefetch<LAYOUT, T, SR>(P, j, gw, pf);
  pdl_wait();

  // the step of q (zero before the first coordinate of a fit), read once
  if (tid == 0) {
    const CtlLine* L = &P.gctl->line[c % kRep];
    s_stop = __ldcg(&L->stop);
    s_applied = __ldcg(&L->applied);
    s_delta[0] = __ldcg(&L->delta_hi);
    s_delta[1] = __ldcg(&L->delta_lo);
    s_dirty = __ldcg(&L->dirty);
  }
  __syncthreads();
  if (s_stop) return;  // the same value in every CTA
  const double applied = s_applied;
  // dense X in the FP32 mode: the update rides along the row pass (one sweep
  // over the warp's rows); otherwise it runs first
  constexpr bool kFuse = LAYOUT == 1 && sizeof(T) == 4;
  if (applied != 0.0 && !kFuse) warp_update<LAYOUT, T>(P, q, gw, row_lo, row_hi, applied, ff{s_delta[0], s_delta[1]});
  // CSC: with a zero pending step e is the e of the previous coordinate's
  // pass (after the fit's first pass), and so are the sums of its dense
  // components, stored by that pass; they are reused bit for bit
  const bool dense = LAYOUT == 1 || applied != 0.0 || s_dirty != 0;
  const T* xq = (kFuse && applied != 0.0) ? reinterpret_cast<const T*>(P.X) + (size_t)q * P.ld : nullptr;

  // ------------------------------------------- step 2 for coordinate j
  A* rec = reinterpret_cast<A*>(P.rec);
  A tot[M];
  warp_pass<MODEL, LAYOUT, T, U, SR, MULTI>(P, j, row_lo, row_hi, rec, tot, pf, dense, xq, ff{s_delta[0], s_delta[1]});
  pdl_launch_dependents();
  if (lane == 0)
#pragma unroll
    for (int m = 0; m < M; ++m) s_wtot[w][m] = tot[m];
  __syncthreads();
  if (w == 0) {
    // warp offsets inside the CTA (exclusive scan of the warp totals) and
    // the CTA aggregate (their total), every lane in the same order
    A v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      acc_zero(v[m]);
      if (lane < WPC) v[m] = s_wtot[lane][m];
    }
    warp_scan_n<M>(v, lane);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      // the stored values of the dense CSC components stay when they were reused
      const bool keep = LAYOUT == 0 && !dense && (m == 0 || m == 3);
      A ex = shfl_up(v[m], 1);
      if (lane == 0) acc_zero(ex);
      if (lane < WPC && !keep) P.wt[(size_t)m * P.nwarps + c * WPC + lane] = pack8(ex);
      v[m] = shfl_idx(v[m], WPC - 1);
    }
    if (lane < kRep)
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (!(LAYOUT == 0 && !dense && (m == 0 || m == 3))) P.agg[((size_t)lane * M + m) * G + c] = pack8(v[m]);
  }
}

// Latency-bound: every load that does not depend on another value of this
// kernel is issued first (CTA aggregates, this CTA's warp totals, its group
// ends), the several sums of each stage share one reduction tree, and the
// common path (at most one group end per thread) has one block barrier
// before the partials.
template <int MODEL, int LAYOUT, typename T, bool BATCH>
__global__ void __launch_bounds__(kTransThreads) k_trans(const __grid_constant__ CcdParams P0, int j) {
  using A = typename AccOf<T>::type;
  constexpr int M = MODEL == 0 ? 3 : 6;
  // prefix sums of the M components (+ for Fine-Gray the grand totals of
  // the three suffix components 3..5, which the transform subtracts from)
  constexpr int NA = MODEL == 0 ? M : M + 3;
  constexpr int NT = kTransThreads;
  __shared__ A s_wp[kTransWarps][NA];
  __shared__ A s_tc[NA];
  __shared__ A s_base[kMaxWarpsPerCta][M];
  __shared__ A s_red[kTransWarps][3];
  __shared__ int s_last;
  __shared__ int s_stopped;
  __shared__ double s_lin[2];
  __shared__ double s_next[4];
  __shared__ CcdParams s_fit;
  if (BATCH) load_fit(s_fit, P0);
  const CcdParams& P = BATCH ? s_fit : P0;

  GraphCtl* ctl = P.gctl;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  const int WPC = P.wpc;
  const int c = blockIdx.x;
  const int G = P.G;
  const bool eval = j == 0;
  const int kc_lo = P.wk0[c * WPC], kc_hi = P.wk0[(c + 1) * WPC];
  const int nends = kc_hi - kc_lo;
  const bool one_end = nends <= NT;

  // ---------------------------------------------- static loads
  int kd = 0, kge = 0;
  double kg = 0.0;
  float2 kgf = make_float2(0.f, 0.f);
  if (one_end && tid < nends) {
    const int k = kc_lo + tid;
    kd = P.dk[k];
    kge = P.gend[k];
    if (MODEL == 1) {
      kg = P.Gk[k];
      kgf = P.Gkff[k];
    }
  }
  pdl_wait();

  // ------------------ every load of this kernel's inputs, in one round trip
  // (thread 0 also reads the control line: stop flag and the scalars of j)
  LineView lv;
  if (tid == 0) {
    lv = load_line(ctl, c);
    s_stopped = lv.stop;
  }
  const uint64_t* agg = P.agg + (size_t)(c % kRep) * M * G;
  // warp of this thread's group end (relative to the CTA); the pass kernel
  // stored each warp's offset inside the CTA in wt
  const int wl = (one_end && tid < nends) ? (int)((kge >> 5) / P.wpw) - c * WPC : (tid < WPC ? tid : 0);
  uint64_t v0[M], v1[M], wbv[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    v0[m] = tid < G ? __ldcg(agg + (size_t)m * G + tid) : 0ull;
    v1[m] = tid + NT < G ? __ldcg(agg + (size_t)m * G + tid + NT) : 0ull;
    wbv[m] = ((one_end && tid < nends) || (!one_end && tid < WPC))
                 ? __ldcg(P.wt + (size_t)m * P.nwarps + c * WPC + wl)
                 : 0ull;
  }
  const A* rec = reinterpret_cast<const A*>(P.rec);
  A kr[M];
  if (one_end && tid < nends)
#pragma unroll
    for (int m = 0; m < M; ++m) kr[m] = rec[(size_t)(kc_lo + tid) * M + m];

  // ------------------- per-warp sums of the aggregates of CTAs before c
  {
    A r[NA];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const A x0 = unpack8<A>(v0[m]), x1 = unpack8<A>(v1[m]);
      acc_zero(r[m]);
      if (tid < c) r[m] = x0;
      if (tid + NT < c) r[m] = acc_add(r[m], x1);
      if (MODEL == 1 && m >= 3) r[M + m - 3] = acc_add(x0, x1);
    }
    for (int qc = tid + 2 * NT; qc < G; qc += NT)  // grids above 512 CTAs
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const A x = unpack8<A>(__ldcg(agg + (size_t)m * G + qc));
        if (qc < c) r[m] = acc_add(r[m], x);
        if (MODEL == 1 && m >= 3) r[M + m - 3] = acc_add(r[M + m - 3], x);
      }
    warp_sum_n<NA>(r);
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < NA; ++i) s_wp[w][i] = r[i];
  }
  __syncthreads();
  if (BATCH && s_stopped) return;  // this fit has stopped (the others go on)
  // prefix before CTA c and (Fine-Gray) grand totals: thread i sums value i
  // over the warps in a fixed order, once for the CTA
  if (tid < NA) {
    A t = s_wp[0][tid];
#pragma unroll 1
    for (int qw = 1; qw < kTransWarps; ++qw) t = acc_add(t, s_wp[qw][tid]);
    s_tc[tid] = t;
  }
  __syncthreads();
  A T_c[M], tot[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    T_c[m] = s_tc[m];
    if (MODEL == 1 && m >= 3) tot[m] = s_tc[M + m - 3];
    else acc_zero(tot[m]);
  }

  // ---------------------------------------------- steps 3-4
  A fg1, fg2;
  acc_zero(fg1);
  acc_zero(fg2);
  double pl = 0.0;
  auto end_terms = [&](int d, const A (&Pm)[M], double g, float2 gf) {
    A den = Pm[0], num1 = Pm[1], num2 = Pm[2];
    if (MODEL == 1) {
      const A gg = acc_base<A>(g, ff{gf.x, gf.y});
      den = acc_add(den, acc_mul(gg, acc_add(tot[3 % M], acc_neg(Pm[3 % M]))));
      num1 = acc_add(num1, acc_mul(gg, acc_add(tot[4 % M], acc_neg(Pm[4 % M]))));
      num2 = acc_add(num2, acc_mul(gg, acc_add(tot[5 % M], acc_neg(Pm[5 % M]))));
    }
    const A inv = acc_recip(den);
    const A Gr = acc_mul(num1, inv);
    const A H = acc_mul(num2, inv);
    fg1 = acc_add(fg1, acc_scale(Gr, d));
    fg2 = acc_add(fg2, acc_scale(acc_add(H, acc_neg(acc_mul(Gr, Gr))), d));
    if (eval) pl += (double)d * log(acc_to_d(den));
  };
  if (one_end) {
    if (kd != 0) {
      // prefix at the end: CTAs before, the CTA's warps before, the warp's rows
      A Pm[M];
#pragma unroll
      for (int m = 0; m < M; ++m) Pm[m] = acc_add(acc_add(T_c[m], unpack8<A>(wbv[m])), kr[m]);
      end_terms(kd, Pm, kg, kgf);
    }
  } else {
    if (tid < WPC)
#pragma unroll
      for (int m = 0; m < M; ++m) s_base[tid][m] = acc_add(T_c[m], unpack8<A>(wbv[m]));
    __syncthreads();
    for (int k = kc_lo + tid; k < kc_hi; k += NT) {
      const int d = P.dk[k];
      if (d == 0) continue;
      const int wl = (int)((P.gend[k] >> 5) / P.wpw) - c * WPC;
      A Pm[M];
#pragma unroll
      for (int m = 0; m < M; ++m) Pm[m] = acc_add(s_base[wl][m], rec[(size_t)k * M + m]);
      end_terms(d, Pm, MODEL == 1 ? P.Gk[k] : 0.0, MODEL == 1 ? P.Gkff[k] : make_float2(0.f, 0.f));
    }
  }

  // ------------------------------------------- CTA partials, fixed order
  {
    A r[3] = {fg1, fg2, eval ? acc_from_d(pl, (A*)nullptr) : A{}};
    warp_sum_n<3>(r);
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < 3; ++i) s_red[w][i] = r[i];
  }
  __syncthreads();
  uint64_t* part = reinterpret_cast<uint64_t*>(P.slot_part);
  if (tid == 0) {
    A a[3] = {s_red[0][0], s_red[0][1], s_red[0][2]};
#pragma unroll 1
    for (int qw = 1; qw < kTransWarps; ++qw)
#pragma unroll
      for (int i = 0; i < 3; ++i) a[i] = acc_add(a[i], s_red[qw][i]);
    if (lv.stop) {
      s_last = 0;  // the fit has stopped: nothing to publish
    } else {
      part[c] = pack8(a[0]);
      part[G + c] = pack8(a[1]);
      part[2 * G + c] = pack8(a[2]);
      // release: the partials above are visible to whoever sees the count
      unsigned prev;
      asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&ctl->ticket) : "memory");
      s_last = prev == (unsigned)(G - 1);
    }
  }
  pdl_launch_dependents();
  __syncthreads();
  if (!s_last) return;

  // ------------------------------- last CTA: the step of coordinate j
  if (w < 3) {
    // warp m sums partial vector m over the CTAs in a fixed order (acquire:
    // every other CTA released its partials before its count)
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    A acc;
    acc_zero(acc);
    for (int q0 = 0; q0 < G; q0 += 32 * 10) {
      uint64_t v[10];
#pragma unroll
      for (int u = 0; u < 10; ++u) {
        const int qc = q0 + 32 * u + lane;
        v[u] = qc < G ? __ldcg(part + (size_t)w * G + qc) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 10; ++u) acc = acc_add(acc, unpack8<A>(v[u]));
    }
    A r[1] = {acc};
    warp_sum_n<1>(r);
    if (lane == 0) s_red[0][w] = r[0];
  } else if (w == 3 && eval) {
    // objective pieces at the current beta (every earlier step is stored)
    double lin, pen;
    warp_lin_pen(P, -1, 0.0, lin, pen);
    if (lane == 0) {
      s_lin[0] = lin;
      s_lin[1] = pen;
    }
  } else if (w == 4 && lane == 0) {
    // scalars of the next coordinate, for the control line
    const int jn = j + 1 < P.p ? j + 1 : 0;
    s_next[0] = __ldcg(P.beta + jn);
    s_next[1] = __ldcg(P.width + jn);
    s_next[2] = P.pen[jn];
    s_next[3] = P.dTx[jn];
  }
  __syncthreads();
  if (w == 0)
    publish_step(P, j, lv, lv.dtx - acc_to_d(s_red[0][0]), -acc_to_d(s_red[0][1]), eval, s_lin[0],
                 s_lin[1], acc_to_d(s_red[0][2]), s_next);
}

// Transform of single fits with the work spread evenly: every CTA scans the
// pass CTAs' aggregates (one per thread, two-level warp scans in shared
// memory; Fine-Gray also takes the grand totals of the suffix components)
// and takes an even share of the group ends, about one a thread.  The
// per-CTA range split of k_trans gave the CTAs holding the first rows (many
// small tie groups) most of the work.  It reads the control line and its
// first end's group table entries before the wait: the line was written by
// the previous coordinate's transform, which finished before this
// coordinate's pass kernel passed its own wait.
constexpr int kBtNT = 512;
constexpr int kBtWarps = kBtNT / 32;

template <int MODEL, int LAYOUT, typename T>
__global__ void __launch_bounds__(kBtNT, 1) k_btrans(const __grid_constant__ CcdParams P, int j) {
  using A = typename AccOf<T>::type;
  constexpr int M = MODEL == 0 ? 3 : 6;
  __shared__ A s_T[kBtNT][M];
  __shared__ A s_w[kBtWarps][M];
  __shared__ A s_tot3[3];
  __shared__ A s_red[kBtWarps][3];
  __shared__ int s_last, s_stop;
  __shared__ double s_lin[2];
  __shared__ double s_next[4];
  GraphCtl* ctl = P.gctl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int WPC = P.wpc, G = P.G, G2 = gridDim.x, c2 = blockIdx.x;
  const bool eval = j == 0;
  LineView lv;
  if (tid == 0) {
    lv = load_line(ctl, c2);
    s_stop = lv.stop;
  }
  const int stride = G2 * kBtNT;
  const int k0 = c2 * kBtNT + tid;
  int d1 = 0, gw1 = 0;
  double g1 = 0.0;
  float2 gf1 = make_float2(0.f, 0.f);
  if (k0 < P.K) {
    d1 = P.dk[k0];
    gw1 = (int)((P.gend[k0] >> 5) / P.wpw);
    if (MODEL == 1) {
      g1 = P.Gk[k0];
      gf1 = P.Gkff[k0];
    }
  }
  __syncthreads();
  if (s_stop) {  // the same value in every CTA
    pdl_wait();
    return;
  }
  pdl_wait();

  // exclusive prefix over the pass CTAs of their aggregates, fixed order
  {
    const uint64_t* agg = P.agg + (size_t)(c2 % kRep) * M * G;
    A v[M], incl[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      acc_zero(v[m]);
      if (tid < G) v[m] = unpack8<A>(__ldcg(agg + (size_t)m * G + tid));
      incl[m] = v[m];
    }
    warp_scan_n<M>(incl, lane);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const A ex = shfl_up(incl[m], 1);
      if (lane == 0) acc_zero(v[m]);
      else v[m] = ex;
    }
    if (lane == 31)
#pragma unroll
      for (int m = 0; m < M; ++m) s_w[w][m] = incl[m];
    __syncthreads();
    if (w == 0) {
      A t[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        acc_zero(t[m]);
        if (lane < kBtWarps) t[m] = s_w[lane][m];
      }
      warp_scan_n<M>(t, lane);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const A ex = shfl_up(t[m], 1);
        const A all = shfl_idx(t[m], kBtWarps - 1);
        if (lane < kBtWarps) {
          if (lane == 0) acc_zero(s_w[lane][m]);
          else s_w[lane][m] = ex;
        }
        if (MODEL == 1 && m >= 3 && lane == 0) s_tot3[m % 3] = all;
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < M; ++m) s_T[tid][m] = acc_add(s_w[w][m], v[m]);
  }
  __syncthreads();

  // steps 3-4 at the group ends
  A fg1, fg2;
  acc_zero(fg1);
  acc_zero(fg2);
  double pl = 0.0;
  A tot3[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc_zero(tot3[i]);
    if (MODEL == 1) tot3[i] = s_tot3[i];
  }
  const A* rec = reinterpret_cast<const A*>(P.rec);
  for (int k = k0; k < P.K; k += stride) {
    int d, gwk;
    double g;
    float2 gf;
    if (k == k0) {
      d = d1, gwk = gw1, g = g1, gf = gf1;
    } else {
      d = P.dk[k];
      gwk = (int)((P.gend[k] >> 5) / P.wpw);
      g = MODEL == 1 ? P.Gk[k] : 0.0;
      gf = MODEL == 1 ? P.Gkff[k] : make_float2(0.f, 0.f);
    }
    if (d == 0) continue;
    const int f = gwk / WPC;
    A Pm[M];
#pragma unroll
    for (int m = 0; m < M; ++m)
      Pm[m] = acc_add(acc_add(s_T[f][m], unpack8<A>(__ldcg(P.wt + (size_t)m * P.nwarps + gwk))),
                      rec[(size_t)k * M + m]);
    A den = Pm[0], num1 = Pm[1], num2 = Pm[2];
    if (MODEL == 1) {
      // the competing-event suffix strictly after the end, weighted by G(t_k)
      const A gg = acc_base<A>(g, ff{gf.x, gf.y});
      den = acc_add(den, acc_mul(gg, acc_add(tot3[0], acc_neg(Pm[3 % M]))));
      num1 = acc_add(num1, acc_mul(gg, acc_add(tot3[1], acc_neg(Pm[4 % M]))));
      num2 = acc_add(num2, acc_mul(gg, acc_add(tot3[2], acc_neg(Pm[5 % M]))));
    }
    const A inv = acc_recip(den);
    const A Gr = acc_mul(num1, inv);
    const A H = acc_mul(num2, inv);
    fg1 = acc_add(fg1, acc_scale(Gr, d));
    fg2 = acc_add(fg2, acc_scale(acc_add(H, acc_neg(acc_mul(Gr, Gr))), d));
    if (eval) pl += (double)d * log(acc_to_d(den));
  }

  // CTA partials, fixed order
  {
    A r[3] = {fg1, fg2, eval ? acc_from_d(pl, (A*)nullptr) : A{}};
    warp_sum_n<3>(r);
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < 3; ++i) s_red[w][i] = r[i];
  }
  __syncthreads();
  uint64_t* part = reinterpret_cast<uint64_t*>(P.slot_part);
  if (tid < 3) {
    A a = s_red[0][tid];
#pragma unroll 1
    for (int qw = 1; qw < kBtWarps; ++qw) a = acc_add(a, s_red[qw][tid]);
    part[(size_t)tid * G2 + c2] = pack8(a);
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    unsigned prev;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&ctl->ticket) : "memory");
    s_last = prev == (unsigned)(G2 - 1);
  }
  pdl_launch_dependents();
  __syncthreads();
  if (!s_last) return;

  // ------------------------------- last CTA: the step of coordinate j
  if (w < 3) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    A acc;
    acc_zero(acc);
    for (int qc = lane; qc < G2; qc += 32) acc = acc_add(acc, unpack8<A>(__ldcg(part + (size_t)w * G2 + qc)));
    A r[1] = {acc};
    warp_sum_n<1>(r);
    if (lane == 0) s_red[0][w] = r[0];
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
  if (w == 0)
    publish_step(P, j, lv, lv.dtx - acc_to_d(s_red[0][0]), -acc_to_d(s_red[0][1]), eval, s_lin[0], s_lin[1],
                 acc_to_d(s_red[0][2]), s_next);
}

// CTAs of the balanced transform: about one group end a thread, 4 to 152.
inline int btrans_ctas(int K) { return std::max(4, std::min(152, (K + kBtNT - 1) / kBtNT)); }

// Grid of the pass kernel: as many CTAs per SM (up to MINB) as fit.
template <int MODEL, int LAYOUT, typename T>
cudaError_t grid_graph(int* G, int* wpc) {
  using GC = GCfg<MODEL, LAYOUT>;
  int dev = 0, sms = 0, occ = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st != cudaSuccess) return st;
  if ((st = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return st;
  if ((st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pass<MODEL, LAYOUT, T, false, false>, GC::NT, 0)) !=
      cudaSuccess)
    return st;
  if (occ < 1) return cudaErrorLaunchOutOfResources;
  *G = sms * std::min(occ, GC::MINB);
  *wpc = GC::NT / 32;
  return cudaSuccess;
}

template <int MODEL, int LAYOUT, typename T>
cudaError_t capture_sweep(const CcdParams& P, bool pdl, cudaStream_t cs, cudaGraph_t* g) {
  using GC = GCfg<MODEL, LAYOUT>;
  cudaError_t st = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (st != cudaSuccess) return st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cudaLaunchConfig_t cp = {};
  cp.gridDim = dim3(P.G, P.nfit > 0 ? P.nfit : 1);
  cp.blockDim = dim3(GC::NT);
  cp.stream = cs;
  cp.attrs = attr;
  cp.numAttrs = 1;
  cudaLaunchConfig_t ct = cp;
  ct.blockDim = dim3(kTransThreads);
  // batched fits: Cox only (the censoring weights of Fine-Gray would have
  // to be re-estimated on each training set)
  // Cox passes whose warps hold two group ends or more on average take the
  // many-ends form of the row pass
  auto kp = k_pass<MODEL, LAYOUT, T, false, false>;
  auto kt = k_trans<MODEL, LAYOUT, T, false>;
  if constexpr (MODEL == 0) {
    const bool multi = P.pass_form == 2 || (P.pass_form == 0 && (int64_t)P.K >= 2 * (int64_t)P.nwarps);
    if (P.nfit > 0) {
      kp = multi ? k_pass<MODEL, LAYOUT, T, true, true> : k_pass<MODEL, LAYOUT, T, true, false>;
      if constexpr (LAYOUT == 0 && sizeof(T) == 4) {
        // tile shapes the cross-validation tuner may pick
        if (P.tile_form == 1)
          kp = multi ? k_pass<MODEL, LAYOUT, T, true, true, 1> : k_pass<MODEL, LAYOUT, T, true, false, 1>;
        if (P.tile_form == 2)
          kp = multi ? k_pass<MODEL, LAYOUT, T, true, true, 2> : k_pass<MODEL, LAYOUT, T, true, false, 2>;
      }
      kt = k_trans<MODEL, LAYOUT, T, true>;
    } else if (multi) {
      kp = k_pass<MODEL, LAYOUT, T, false, true>;
    }
  } else {
    if (P.nfit > 0) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(cs, &junk);
      if (junk) cudaGraphDestroy(junk);
      return cudaErrorInvalidValue;
    }
  }
  // single fits: the balanced transform (one pass-CTA aggregate per thread
  // in its scan, so up to kBtNT pass CTAs)
  if (P.nfit == 0 && P.G <= kBtNT) {
    kt = k_btrans<MODEL, LAYOUT, T>;
    ct.gridDim = dim3(btrans_ctas(P.K));
    ct.blockDim = dim3(kBtNT);
  }
  cudaError_t lst = cudaSuccess;
  for (int j = 0; j < P.p && lst == cudaSuccess; ++j) {
    lst = cudaLaunchKernelEx(&cp, kp, P, j);
    if (lst == cudaSuccess) lst = cudaLaunchKernelEx(&ct, kt, P, j);
  }
  st = cudaStreamEndCapture(cs, g);
  return lst != cudaSuccess ? lst : st;
}

}  // namespace

#define SURV_DISPATCH_G(FN, ...)                                             \
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

namespace {
cudaError_t capture_any(int model, int layout, int prec, const CcdParams& P, bool pdl, cudaStream_t cs,
                        cudaGraph_t* g) {
  SURV_DISPATCH_G(capture_sweep, P, pdl, cs, g);
}
}  // namespace

cudaError_t graph_grid_size(int model, int layout, int prec, int* G, int* wpc) {
  SURV_DISPATCH_G(grid_graph, G, wpc);
}

cudaError_t graph_init(const CcdParams& P, cudaStream_t s) {
  k_graph_init<<<dim3(1, P.nfit > 0 ? P.nfit : 1), 32, 0, s>>>(P);
  return cudaGetLastError();
}

void graph_cache_free(GraphCache* gc) {
  if (!gc) return;
  if (gc->exec) cudaGraphExecDestroy(gc->exec);
  for (auto& e : gc->ev)
    if (e) cudaEventDestroy(e);
  if (gc->flag) cudaFreeHost(gc->flag);
  if (gc->cs) cudaStreamDestroy(gc->cs);
  *gc = GraphCache();
}

cudaError_t time_one_sweep(int model, int layout, int prec, const CcdParams& P, cudaStream_t s, float* ms) {
  *ms = 0.f;
  GraphCache gc;
  struct Guard {
    GraphCache* g;
    cudaGraph_t graph = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ~Guard() {
      if (graph) cudaGraphDestroy(graph);
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      graph_cache_free(g);
    }
  } guard{&gc};
  cudaError_t st;
  if ((st = cudaStreamCreateWithFlags(&gc.cs, cudaStreamNonBlocking)) != cudaSuccess) return st;
  const bool pdl = !P.no_pdl;
  if ((st = capture_any(model, layout, prec, P, pdl, gc.cs, &guard.graph)) != cudaSuccess) return st;
  if ((st = cudaGraphInstantiate(&gc.exec, guard.graph, 0)) != cudaSuccess) return st;
  if ((st = cudaEventCreate(&guard.a)) != cudaSuccess) return st;
  if ((st = cudaEventCreate(&guard.b)) != cudaSuccess) return st;
  if ((st = cudaEventRecord(guard.a, s)) != cudaSuccess) return st;
  if ((st = cudaGraphLaunch(gc.exec, s)) != cudaSuccess) return st;
  if ((st = cudaEventRecord(guard.b, s)) != cudaSuccess) return st;
  if ((st = cudaEventSynchronize(guard.b)) != cudaSuccess) return st;
  return cudaEventElapsedTime(ms, guard.a, guard.b);
}

cudaError_t graph_cache_prepare(GraphCache* gc) {
  if (gc->cs) return cudaSuccess;
  cudaError_t st;
  if ((st = cudaStreamCreateWithFlags(&gc->cs, cudaStreamNonBlocking)) != cudaSuccess) return st;
  for (auto& e : gc->ev)
    if ((st = cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) != cudaSuccess) return st;
  return cudaMallocHost(&gc->flag, 2 * sizeof(int));
}

cudaError_t replay_until_stop(const CcdParams& P, cudaStream_t s, GraphCache* gc, cudaEvent_t t0,
                              int launches_per_replay, int* replays, int* launches, int max_replays_in) {
  cudaError_t st;
  gc->flag[0] = gc->flag[1] = 0;
  if (t0 && (st = cudaEventRecord(t0, s)) != cudaSuccess) return st;
  // One replay per sweep.  The stop flag of replay i is read while replay
  // i + 1 runs; kernels of a replay after the stop return at once.  The
  // device stops at the evaluation of sweep max_sweeps at the latest, which
  // falls in replay max_sweeps.  A batched launch ends when every fit has
  // counted itself as stopped.
  const int max_replays = max_replays_in > 0 ? max_replays_in : P.max_sweeps + 2;
  const int target = P.nfit > 0 ? P.nfit : 1;
  const void* stop_src =
      P.nfit > 0 ? static_cast<const void*>(P.done_count) : static_cast<const void*>(&P.gctl->done);
  int i = 0;
  for (; i < max_replays; ++i) {
    if ((st = cudaGraphLaunch(gc->exec, s)) != cudaSuccess) return st;
    *launches += launches_per_replay;
    if ((st = cudaMemcpyAsync(gc->flag + (i & 1), stop_src, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return st;
    if ((st = cudaEventRecord(gc->ev[i & 1], s)) != cudaSuccess) return st;
    if (i >= 1) {
      if ((st = cudaEventSynchronize(gc->ev[(i - 1) & 1])) != cudaSuccess) return st;
      if (gc->flag[(i - 1) & 1] >= target) {
        ++i;
        break;
      }
    }
  }
  *replays = i;
  // the last replay's flag copy must land before the host buffer is reused
  return cudaEventSynchronize(gc->ev[(i - 1) & 1]);
}

cudaError_t run_ccd_graph(int model, int layout, int prec, const CcdParams& P, cudaStream_t s, GraphCache* gc,
                          cudaEvent_t t0, int* replays, int* launches) {
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
  // programmatic dependent launch between the kernels; SURV_FLAG_NO_PDL
  // turns it off (plain stream order), for comparison
  const bool pdl = !P.no_pdl;
  const int mlp = (model * 4 + layout * 2 + prec) * 2 + (pdl ? 1 : 0);
  if (!gc->exec || gc->mlp != mlp || std::memcmp(&gc->key, &P, sizeof(P)) != 0) {
    if (gc->exec) {
      cudaGraphExecDestroy(gc->exec);
      gc->exec = nullptr;
    }
    // capture on a private stream (the caller's may be the legacy stream)
    cudaGraph_t g = nullptr;
    st = capture_any(model, layout, prec, P, pdl, gc->cs, &g);
    if (st == cudaSuccess) st = cudaGraphInstantiate(&gc->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != cudaSuccess) {
      gc->exec = nullptr;
      return st;
    }
    gc->key = P;
    gc->mlp = mlp;
  }
  return replay_until_stop(P, s, gc, t0, 2 * P.p, replays, launches);
}

}  // namespace survgpu
