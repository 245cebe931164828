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

#include "ccd_common.cuh"

namespace survgpu {
namespace {

using namespace ccdk;


// Grid exchange: every CTA writes its payload slot, then thread 0 fences and
// adds 1 to the exchange counter; lane 0 of the waiting warp polls the counter
// with acquire loads until it reaches `target` (= exchanges so far x G), then
// the warp reads the payloads through L2.  One counter measured faster on
// GB300 than one flag per CTA or counters spread over several lines.  The
// wait is bounded by limit_ns.
__device__ __forceinline__ void exchange_arrive(unsigned* counter) {
  // release reduction: orders this thread's payload stores before the count
  // without a sequentially consistent fence
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(counter), "r"(1u) : "memory");
}

__device__ __forceinline__ bool exchange_wait(const unsigned* counter, unsigned target, unsigned* err,
                                              uint64_t limit_ns) {
  const int lane = threadIdx.x & 31;
  uint64_t t0 = 0;
  bool timed = false;
  for (unsigned spin = 0;; ++spin) {
    unsigned v = 0;
    if (lane == 0) v = ld_acquire(counter);
    v = __shfl_sync(0xffffffffu, v, 0);
    if (v >= target) break;
    // error word and wall clock only every 64 polls: both are slow off-SM reads
    if ((spin & 63u) == 63u) {
      unsigned bad = lane == 0 ? ld_volatile(err) : 0u;
      bad = __shfl_sync(0xffffffffu, bad, 0);
      if (bad) return false;
      if (!timed) { t0 = global_ns(); timed = true; }
      if (global_ns() - t0 > limit_ns) {
        if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
        return false;
      }
    }
  }
  __syncwarp();
  return true;
}

template <int MODEL, int LAYOUT, typename T>
__global__ void __launch_bounds__(Cfg<MODEL, LAYOUT, T>::MAXT, 1) ccd_kernel(const __grid_constant__ CcdParams P) {
  using A = typename AccOf<T>::type;
  using C = Cfg<MODEL, LAYOUT, T>;
  constexpr int M = C::M;

  __shared__ A s_wtot[kMaxWarpsPerCta][M];      // warp totals of the pass
  __shared__ A s_base[kMaxWarpsPerCta][M];      // prefix before each warp: CTAs before + warps before
  __shared__ A s_tot[M];                        // grand totals (Fine-Gray suffix)
  __shared__ A s_red[kMaxWarpsPerCta][3];
  __shared__ double s_bc[8];                     // scalars broadcast by thread 0
  __shared__ float s_delta[2];                   // applied step as float-float
  __shared__ int s_flag[2];

  const int tid = threadIdx.x;
  const int WPC = P.wpc;
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
  const int kc_lo = P.wk0[c * WPC], kc_hi = P.wk0[(c + 1) * WPC];

  A* rec = reinterpret_cast<A*>(P.rec);
  const bool single = P.single_j >= 0;

  // control state, meaningful in thread 0 only (identical in every CTA)
  int sweep = 0, converged = 0;
  double f_prev = 0.0, f_prev2 = 0.0, ll_last = 0.0;
  long long eta_updates = 0;
  unsigned passes = 0;
  bool finished = false;
  // phase timers (thread 0): CTA 0 reports its phases, every CTA its pass time
  unsigned long long ph[16] = {0};
  uint64_t tmark = 0;
  // phase timers use the SM cycle counter (cheap); converted to ns at the end
  // with the ratio of %globaltimer to clock64 over the whole launch
  const uint64_t g_start = tid == 0 ? global_ns() : 0;
  const long long c_start = tid == 0 ? clock64() : 0;
  auto lap = [&](int i) {
    if (tid == 0) {
      const uint64_t t = (uint64_t)clock64();
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
        tmark = (uint64_t)clock64();
      }

      // ------------------------------------------------ step 2: warp pass
      A tot[M];
      PassPrefetch<T, 4> pf;
      pass_prefetch<LAYOUT, T, 4>(P, j, gw, pf);
      warp_pass<MODEL, LAYOUT, T, C::U, 4>(P, j, row_lo, row_hi, rec, tot, pf);
      if (lane == 0)
#pragma unroll
        for (int m = 0; m < M; ++m) s_wtot[w][m] = tot[m];
      __syncthreads();
      lap(PH_PASS);

      // ------------------------------ CTA combine and grid exchange #1
      // Payloads are float-float pairs laid out [parity][component][CTA] so
      // that one warp reads every CTA's value with coalesced loads.  All of
      // the combine arithmetic is float-float on the FP32 pipe: GB300's FP64
      // pipe makes even short double-precision warp reductions slow.
      if (w == 0) {
        uint64_t* agg_soa = reinterpret_cast<uint64_t*>(P.slot_agg) + (size_t)par * 6 * G;
        A wv[M], excl[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          acc_zero(wv[m]);
          if (lane < WPC) wv[m] = s_wtot[lane][m];
        }
        A asum[M];
#pragma unroll
        for (int m = 0; m < M; ++m) asum[m] = warp_sum(wv[m]);
        lap(PH_EX1_SUMS);
        if (lane == 0)
#pragma unroll
          for (int m = 0; m < M; ++m) agg_soa[(size_t)m * G + c] = pack8(asum[m]);
        lap(PH_EX1_STORE);
        if (lane == 0 && c != P.withhold_cta) exchange_arrive(P.counters + 0);
        lap(PH_EX1_PRE);
        // CTA-local work while the other CTAs arrive: warp offsets, and the
        // loads of beta / dTx / penalty factors for the objective
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const A incl = warp_inclusive_scan(wv[m], lane);
          const A ex = shfl_up(incl, 1);
          excl[m] = ex;
          if (lane == 0) acc_zero(excl[m]);
        }
        double pen = 0.0, lin = 0.0;
        if (eval) warp_lin_pen(P, -1, 0.0, lin, pen);
        bool ok = exchange_wait(P.counters + 0, passes * (unsigned)G, P.err, P.timeout_ns);
        lap(PH_EX1_WAIT);
        if (lane == 0) s_flag[0] = ok ? 0 : 1;
        if (ok) {
          // exclusive prefix over CTAs < c (fixed order) and grand totals
          A pre[M], all[M];
#pragma unroll
          for (int m = 0; m < M; ++m) { acc_zero(pre[m]); acc_zero(all[m]); }
          for (int q0 = 0; q0 < G; q0 += 32 * 5) {
            uint64_t v[M][5];
#pragma unroll
            for (int u = 0; u < 5; ++u) {
              const int q = q0 + 32 * u + lane;
#pragma unroll
              for (int m = 0; m < M; ++m) v[m][u] = q < G ? __ldcg(agg_soa + (size_t)m * G + q) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 5; ++u) {
              const int q = q0 + 32 * u + lane;
#pragma unroll
              for (int m = 0; m < M; ++m) {
                const A x = unpack8<A>(v[m][u]);
                if (q < c) pre[m] = acc_add(pre[m], x);
                if (MODEL == 1) all[m] = acc_add(all[m], x);
              }
            }
          }
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const A T_c = warp_sum(pre[m]);
            if (MODEL == 1) {
              const A a2 = warp_sum(all[m]);
              if (lane == 0) s_tot[m] = a2;
            }
            if (lane < WPC) s_base[lane][m] = acc_add(T_c, excl[m]);
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
      const int nw_red = cta_transform<MODEL, A>(P, eval, kc_lo, kc_hi, c * WPC, s_base, s_tot, rec, s_red);
      __syncthreads();
      lap(PH_TRANSFORM);

      // ------------------------------ grid exchange #2, Newton step
      if (w == 0) {
        uint64_t* part_soa = reinterpret_cast<uint64_t*>(P.slot_part) + (size_t)par * 3 * G;
        A r0, r1, r2;
        acc_zero(r0);
        acc_zero(r1);
        acc_zero(r2);
        if (lane < nw_red) { r0 = s_red[lane][0]; r1 = s_red[lane][1]; r2 = s_red[lane][2]; }
        const A a1 = warp_sum(r0), a2 = warp_sum(r1), al = warp_sum(r2);
        if (lane == 0) {
          part_soa[c] = pack8(a1);
          part_soa[G + c] = pack8(a2);
          part_soa[2 * G + c] = pack8(al);
          if (c != P.withhold_cta) exchange_arrive(P.counters + 1);
        }
        lap(PH_EX2_PRE);
        bool ok = exchange_wait(P.counters + 1, passes * (unsigned)G, P.err, P.timeout_ns);
        lap(PH_EX2_WAIT);
        int fin = ok ? 0 : 2;
        if (ok) {
          A sums[3];
          warp_fold_slots<A, 3>(part_soa, G, sums);
          const A s1 = sums[0], s2 = sums[1], sl = sums[2];
          const double g1 = acc_to_d(s1), g2 = acc_to_d(s2), gl = acc_to_d(sl);
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
      if (applied != 0.0)
        cta_update<LAYOUT, T>(P, j, c * WPC, (c + 1) * WPC, cta_row_lo, cta_row_hi, applied,
                              ff{s_delta[0], s_delta[1]});
      __syncthreads();
      lap(PH_UPDATE);
    }
    if (finished) break;
    ++sweep;
  }

  if (tid == 0 && P.timing) {
    const double ns_per_cycle =
        (double)(global_ns() - g_start) / (double)max(1ll, clock64() - c_start);
    for (int i = 0; i < 16; ++i) ph[i] = (unsigned long long)(ph[i] * ns_per_cycle);
    atomicMax(P.timing + PH_PASS_MAX, ph[PH_PASS]);
    atomicMin(P.timing + PH_PASS_MIN, ph[PH_PASS]);
    atomicAdd(P.timing + PH_PASS_SUM, ph[PH_PASS]);
    if (c == 0) {
      for (int i = 0; i < 9; ++i) P.timing[i] = ph[i];
      P.timing[PH_EX1_SUMS] = ph[PH_EX1_SUMS];
      P.timing[PH_EX1_STORE] = ph[PH_EX1_STORE];
    }
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
