// Device code shared by the per-coordinate graph schedules (ccd_graph.cu:
// the paper's row pass; sn.cu: the sparse-numerator form): programmatic
// dependent launch, the control lines, and the step of one coordinate.
#pragma once

#include "ccd_common.cuh"

namespace survgpu {
namespace ccdk {

// Programmatic dependent launch: everything before pdl_wait() may only read
// data that no earlier kernel of the fit writes.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Scalars of the control line a CTA reads (thread 0 loads them).
struct LineView {
  int stop = 0, nevals = 0;
  double applied = 0.0;
  ff delta = {0.f, 0.f};
  double beta = 0.0, width = 0.0, pen = 0.0, dtx = 0.0, f_prev = 0.0;
  long long passes = 0, eta_updates = 0;
};
__device__ __forceinline__ LineView load_line(const GraphCtl* ctl, int c) {
  const CtlLine* L = &ctl->line[c % kRep];
  LineView v;
  v.stop = __ldcg(&L->stop);
  v.nevals = __ldcg(&L->nevals);
  v.applied = __ldcg(&L->applied);
  v.delta = {__ldcg(&L->delta_hi), __ldcg(&L->delta_lo)};
  v.beta = __ldcg(&L->beta);
  v.width = __ldcg(&L->width);
  v.pen = __ldcg(&L->pen);
  v.dtx = __ldcg(&L->dtx);
  v.f_prev = __ldcg(&L->f_prev);
  v.passes = __ldcg(&L->passes);
  v.eta_updates = __ldcg(&L->eta_updates);
  return v;
}

// Per-fit parameters of a batched launch, read once per CTA into shared
// memory (the table is written before the fit starts: it may be read before
// the wait on the previous kernel).
__device__ __forceinline__ void load_fit(CcdParams& dst, const CcdParams& P0) {
  static_assert(sizeof(CcdParams) % 8 == 0, "CcdParams is copied in 8-byte words");
  constexpr int W = sizeof(CcdParams) / 8;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(P0.fits + blockIdx.y);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
  for (int i = threadIdx.x; i < W; i += blockDim.x) d[i] = __ldg(src + i);
  __syncthreads();
}

// The step of coordinate j, taken by warp 0 of the kernel's last CTA
// (Section 2.4): lane 0 gets l' (grad) and l'' (hess); on an evaluation pass
// (eval, j = 0) the objective f = lin - sum_dlog + pen at the start of the
// sweep and the stopping rule; then the trust-region Newton step, beta_j and
// its width, and every lane writes one replica of the control line for the
// next kernels (next = beta, width, pen, delta^T X of coordinate j + 1).
__device__ __forceinline__ void publish_step(const CcdParams& P, int j, const LineView& lv, double grad,
                                             double hess, bool eval, double lin, double pen, double sum_dlog,
                                             const double (&next)[4]) {
  const int lane = threadIdx.x & 31;
  GraphCtl* ctl = P.gctl;
  {
    LineView out;
    if (lane == 0) {
      out = lv;
      out.passes = lv.passes + 1;
      out.applied = 0.0;
      out.delta = {0.f, 0.f};
      if (eval) {
        // objective at the start of sweep s = nevals and the stopping rule
        const int sidx = lv.nevals;
        const double ll = lin - sum_dlog;
        const double f = ll + pen;
        const double fp = sidx >= 1 ? lv.f_prev : 0.0;
        const bool conv = sidx >= 1 && fabs(f - fp) / fabs(f) < P.tol;
        out.stop = (conv || sidx >= P.max_sweeps) ? 1 : 0;
        out.nevals = sidx + 1;
        out.f_prev = f;
        if (out.stop) {
          P.out[OUT_LOGLIK] = ll;
          P.out[OUT_OBJECTIVE] = f;
          P.out[OUT_OBJECTIVE_PREV] = fp;
          P.out[OUT_SWEEPS] = (double)sidx;
          P.out[OUT_CONVERGED] = conv ? 1.0 : 0.0;
          P.out[OUT_ETA_UPDATES] = (double)lv.eta_updates;
          P.out[OUT_PASSES] = (double)out.passes;
          ctl->done = 1;
          if (P.done_count) atomicAdd(P.done_count, 1u);
        }
      }
      double bnew = lv.beta, wnew = lv.width;
      if (!out.stop) {
        const double step = newton_step(lv.beta, grad, hess, P.penalty, lv.pen);
        if (step != 0.0) out.applied = copysign(fmin(fabs(step), lv.width), step);
        bnew = lv.beta + out.applied;
        wnew = fmax(2.0 * fabs(out.applied), lv.width / 2.0);
        P.beta[j] = bnew;
        P.width[j] = wnew;
        if (out.applied != 0.0) out.eta_updates = lv.eta_updates + 1;
        out.delta = d_to_ff(out.applied);
      }
      if (P.p == 1) {
        out.beta = bnew;
        out.width = wnew;
      } else {
        out.beta = next[0];
        out.width = next[1];
      }
      out.pen = next[2];
      out.dtx = next[3];
      ctl->ticket = 0u;
    }
    // every lane writes one replica of the line
    out.stop = __shfl_sync(0xffffffffu, out.stop, 0);
    out.nevals = __shfl_sync(0xffffffffu, out.nevals, 0);
    out.applied = __shfl_sync(0xffffffffu, out.applied, 0);
    out.delta.hi = __shfl_sync(0xffffffffu, out.delta.hi, 0);
    out.delta.lo = __shfl_sync(0xffffffffu, out.delta.lo, 0);
    out.beta = __shfl_sync(0xffffffffu, out.beta, 0);
    out.width = __shfl_sync(0xffffffffu, out.width, 0);
    out.pen = __shfl_sync(0xffffffffu, out.pen, 0);
    out.dtx = __shfl_sync(0xffffffffu, out.dtx, 0);
    out.f_prev = __shfl_sync(0xffffffffu, out.f_prev, 0);
    out.passes = __shfl_sync(0xffffffffu, out.passes, 0);
    out.eta_updates = __shfl_sync(0xffffffffu, out.eta_updates, 0);
    CtlLine* L = &ctl->line[lane];
    L->stop = out.stop;
    L->nevals = out.nevals;
    L->applied = out.applied;
    L->delta_hi = out.delta.hi;
    L->delta_lo = out.delta.lo;
    L->beta = out.beta;
    L->width = out.width;
    L->pen = out.pen;
    L->dtx = out.dtx;
    L->f_prev = out.f_prev;
    L->passes = out.passes;
    L->eta_updates = out.eta_updates;
    L->dirty = 0;
  }
}


}  // namespace ccdk
}  // namespace survgpu
