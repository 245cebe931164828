// Speculative coordinate batches for the row-pass schedule (Cox, CSC, FP32
// mode).  Cyclic CCD (Section 2.4) takes coordinate j's Newton step at the
// e left by coordinate j - 1; when that step is zero, e is unchanged and
// coordinate j + 1 sees the same risk sets.  So one row pass evaluates the
// tuple sums (Section 2.7, steps 2-4) of B consecutive coordinates
// j0 .. j0 + B - 1 at the current e, and the steps are taken in order up to
// and including the first nonzero one; later coordinates are evaluated again
// by the next pass, after that step is applied.  Every committed step is the
// one the one-coordinate-at-a-time schedule takes, from the same sums.
//
// Two kernels per batch, replayed as a CUDA graph of S batches with
// programmatic dependent launch; the batch start j0 and the pending step
// travel in the control lines.
//   k_spass   each warp applies the pending step to its rows, streams e
//             once (prefix of e at its group ends) and walks the nonzeros of
//             the B columns in its rows (prefixes of e x and e x^2 at its
//             group ends); the CTA publishes warp offsets and its aggregate.
//   k_strans  every CTA: prefix of the aggregates before it, G and H of the
//             B columns at its group ends, partial sums; the last CTA takes
//             the B candidate steps (one lane each), commits them up to the
//             first nonzero one, evaluates the objective when j0 = 0, and
//             publishes the next batch.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "graph_common.cuh"

namespace survgpu {
namespace {

using namespace ccdk;

constexpr int kSpNT = 512;   // pass kernel: two CTAs of 512 threads per SM
constexpr int kSpU = 4;      // 16-byte loads of e per lane per tile
constexpr int kSpSR = 4;     // rounds of 32 nonzeros loaded together
constexpr int kStNT = 256;   // transform kernel
constexpr int kStWarps = kStNT / 32;

template <int B>
struct SpCfg {
  static constexpr int R = 1 + 2 * B;   // record components: e, then (e x, e x^2) per column
  static constexpr int NP = 2 * B + 1;  // partials: sum d G, sum d (H - G^2) per column, sum d log den
};

// Dense walk: the prefix of e over the warp's rows at each of its group ends
// (warp-relative, rec[k * R]); returns the lane's partial total.
__device__ __forceinline__ ff sp_dense(const float* e, const int32_t* gend, int64_t row_lo, int64_t row_hi, ff* rec,
                                       int R, EndCursor ec) {
  constexpr int U = kSpU, VEC = 4, TILE = 32 * U * VEC;
  const int lane = threadIdx.x & 31;
  const uint64_t keep = l2_keep();
  ff acc = ff_zero();
  int64_t next_end = ec.pos(gend);
  for (int64_t t0 = row_lo; t0 < row_hi; t0 += TILE) {
    float ev[U][VEC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = t0 + (int64_t)(lane + 32 * u) * VEC;
      if (r + VEC <= row_hi) {
        ld4_hint(e + r, keep, ev[u]);
      } else {
#pragma unroll
        for (int q = 0; q < VEC; ++q) ev[u][q] = r + q < row_hi ? e[r + q] : 0.f;
      }
    }
    float su[U];
#pragma unroll
    for (int u = 0; u < U; ++u) su[u] = (ev[u][0] + ev[u][1]) + (ev[u][2] + ev[u][3]);
    const int64_t t_end = min(t0 + (int64_t)TILE, row_hi);
    while (next_end < t_end) {
      // the lane's rows up to the end: chunks before the end's chunk, and
      // that chunk up to the end
      const int off = (int)(next_end - t0);
      const int cstar = off / VEC, qstar = off - cstar * VEC;
      float part = 0.f;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = 32 * u + lane;
        if (c < cstar) {
          part += su[u];
        } else if (c == cstar) {
#pragma unroll
          for (int q = 0; q < VEC; ++q)
            if (q <= qstar) part += ev[u][q];
        }
      }
      ff pref[1] = {ff_add_f(acc, part)};
      warp_sum_some<1>(pref);
      if (lane == 0) rec[(size_t)ec.kn * R] = pref[0];
      ++ec.kn;
      next_end = ec.pos(gend);
    }
#pragma unroll
    for (int s = 1; s < U; s <<= 1)
#pragma unroll
      for (int u = 0; u + s < U; u += 2 * s) su[u] += su[u + s];
    acc = ff_add_f(acc, su[0]);
  }
  return acc;
}

// Sparse walk of one column's nonzeros in the warp's rows [sa, sb): the
// prefixes of e x and e x^2 at the group ends before its last nonzero
// (rec[k * R + off], + 1); s0, s1 get the lane partials.  Returns the first
// group end not written (the later ends see the warp totals).
__device__ __forceinline__ int sp_sparse(const float* e, const int32_t* gend, const int32_t* ri, const float* vals,
                                         int sa, int sb, ff* rec, int R, int off, EndCursor ec, ff& s0, ff& s1) {
  constexpr int SR = kSpSR;
  const int lane = threadIdx.x & 31;
  const uint64_t keep = l2_keep(), strm = l2_stream();
  s0 = ff_zero();
  s1 = ff_zero();
  int64_t next_end = ec.pos(gend);
  for (int base = sa; base < sb; base += 32 * SR) {
    int row[SR];
    float x[SR], ev[SR];
#pragma unroll
    for (int r = 0; r < SR; ++r) {
      const int i = base + 32 * r + lane;
      const bool valid = i < sb;
      row[r] = valid ? ld_hint(ri + i, strm) : INT_MAX;
      x[r] = valid ? (vals ? ld_stream(vals + i, strm) : 1.f) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < SR; ++r) ev[r] = row[r] != INT_MAX ? ld_hint(e + row[r], keep) : 0.f;
#pragma unroll
    for (int r = 0; r < SR; ++r) {
      const int rb = base + 32 * r;
      if (rb >= sb) break;
      const int nvalid = min(32, sb - rb);
      const float v0 = ev[r] * x[r];
      const float v1 = v0 * x[r];
      const int last_row = __shfl_sync(0xffffffffu, row[r], nvalid - 1);
      while (next_end < (int64_t)last_row) {
        const bool in = (int64_t)row[r] <= next_end;
        ff pref[2] = {ff_add_f(s0, in ? v0 : 0.f), ff_add_f(s1, in ? v1 : 0.f)};
        warp_sum_some<2>(pref);
        if (lane == 0) {
          rec[(size_t)ec.kn * R + off] = pref[0];
          rec[(size_t)ec.kn * R + off + 1] = pref[1];
        }
        ++ec.kn;
        next_end = ec.pos(gend);
      }
      s0 = ff_add_f(s0, v0);
      s1 = ff_add_f(s1, v1);
    }
  }
  return ec.kn;
}

template <int B>
__global__ void __launch_bounds__(kSpNT, 2) k_spass(const __grid_constant__ CcdParams P, int slot) {
  constexpr int R = SpCfg<B>::R;
  __shared__ ff s_wtot[kMaxWarpsPerCta][R];
  __shared__ int s_stop, s_j0, s_q, s_dirty;
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
  // the warp's group ends do not depend on earlier kernels
  const int k_lo = P.wk0[gw], k_hi = P.wk0[gw + 1];
  const int kreg = k_lo + lane < k_hi ? P.gend[k_lo + lane] : INT_MAX;
  pdl_wait();
  if (tid == 0) {
    const CtlLine* L = &P.gctl->line[c % kRep];
    s_stop = __ldcg(&L->stop);
    s_j0 = __ldcg(&L->j0);
    s_q = __ldcg(&L->q);
    s_applied = __ldcg(&L->applied);
    s_delta[0] = __ldcg(&L->delta_hi);
    s_delta[1] = __ldcg(&L->delta_lo);
    s_dirty = __ldcg(&L->dirty);
  }
  __syncthreads();
  if (s_stop) return;
  const int j0 = s_j0;
  const int nb = min(B, P.p - j0);
  // e unchanged since the previous pass (zero pending step): its stored
  // prefix of e, warp offsets and CTA aggregate of component 0 still hold
  const bool dense = s_applied != 0.0 || s_dirty != 0;
  // the batch's column slices in this warp's rows (their loads overlap the
  // update and the dense walk)
  const int nw1 = P.nwarps + 1;
  int64_t cb[B];
  int sa[B], sb[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = b < nb ? j0 + b : j0;
    cb[b] = P.col_ptr[j];
    sa[b] = P.woff[(size_t)j * nw1 + gw];
    sb[b] = b < nb ? P.woff[(size_t)j * nw1 + gw + 1] : sa[b];
  }
  if (s_applied != 0.0) warp_update<0, float>(P, s_q, gw, row_lo, row_hi, s_applied, ff{s_delta[0], s_delta[1]});
  ff* rec = reinterpret_cast<ff*>(P.rec);
  const float* e = reinterpret_cast<const float*>(P.e);
  if (dense) {
    ff t0[1] = {sp_dense(e, P.gend, row_lo, row_hi, rec, R, EndCursor{k_lo, k_hi, k_lo, kreg})};
    warp_sum_some<1>(t0);
    if (lane == 0) s_wtot[w][0] = t0[0];
  }
  // one column at a time (one copy of the walk's code): its warp totals go
  // to shared memory and to the group ends after its last nonzero
#pragma unroll 1
  for (int b = 0; b < B; ++b) {
    int64_t cbb = cb[0];
    int sab = sa[0], sbb = sb[0];
#pragma unroll
    for (int q = 1; q < B; ++q)
      if (b == q) {
        cbb = cb[q];
        sab = sa[q];
        sbb = sb[q];
      }
    const float* vals = P.values ? reinterpret_cast<const float*>(P.values) + cbb : nullptr;
    ff t[2];
    const int kn = sp_sparse(e, P.gend, P.row_idx + cbb, vals, sab, sbb, rec, R, 1 + 2 * b,
                             EndCursor{k_lo, k_hi, k_lo, kreg}, t[0], t[1]);
    warp_sum_some<2>(t);
    if (lane == 0) {
      for (int k = kn; k < k_hi; ++k) {
        rec[(size_t)k * R + 1 + 2 * b] = t[0];
        rec[(size_t)k * R + 2 + 2 * b] = t[1];
      }
      s_wtot[w][1 + 2 * b] = t[0];
      s_wtot[w][2 + 2 * b] = t[1];
    }
  }
  pdl_launch_dependents();
  __syncthreads();
  // warp w scans component m = w, w + WPC, ... over the CTA's warps
  // (component 0 only after a dense walk)
  for (int m = dense ? w : w + 1; m < R; m += WPC) {
    ff v = ff_zero();
    if (lane < WPC) v = s_wtot[lane][m];
    const ff incl = warp_inclusive_scan(v, lane);
    ff ex = shfl_up(incl, 1);
    if (lane == 0) ex = ff_zero();
    if (lane < WPC) P.wt[(size_t)m * P.nwarps + c * WPC + lane] = pack8(ex);
    const ff t = shfl_idx(incl, WPC - 1);
    if (lane < kRep) P.agg[((size_t)lane * R + m) * G + c] = pack8(t);
  }
}

// CoordIn: lane b's beta, trust-region width, lambda * penalty factor and
// delta^T X of coordinate j0 + b (loaded by the caller, possibly early).
struct CoordIn {
  double beta = 0.0, width = 0.0, pen = 0.0, dtx = 0.0;
};
__device__ __forceinline__ CoordIn load_coord(const CcdParams& P, int j0, int nb) {
  const int lane = threadIdx.x & 31;
  CoordIn c;
  if (lane < nb) {
    const int j = j0 + lane;
    c.beta = __ldcg(P.beta + j);
    c.width = __ldcg(P.width + j);
    c.pen = P.pen[j];
    c.dtx = P.dTx[j];
  }
  return c;
}


// Warp 0 of a batch's last transform CTA: on j0 = 0 the objective at the
// start of the sweep and the stopping rule; then lane b takes the candidate
// step of coordinate j0 + b (Section 2.4) from the batch's sums s_tot
// (sum d G per column, sum d (H - G^2) per column, sum d log den), the steps
// are committed in order up to and including the first nonzero one, and
// every lane writes one replica of the control line for the next batch.
template <int B>
__device__ __forceinline__ void commit_batch(const CcdParams& P, const LineView& lv, long long batches_prev, int j0,
                                             int nb, bool eval, const ff* s_tot, const double* s_lin,
                                             const CoordIn& ci) {
  GraphCtl* ctl = P.gctl;
  const int lane = threadIdx.x & 31;
  // objective at the start of the sweep and the stopping rule (j0 = 0)
  int stop = 0, nevals = 0;
  double f_prev = 0.0;
  if (lane == 0) {
    nevals = lv.nevals;
    f_prev = lv.f_prev;
    if (eval) {
      const int sidx = lv.nevals;
      const double ll = s_lin[0] - ff_to_d(s_tot[2 * B]);
      const double f = ll + s_lin[1];
      const double fp = sidx >= 1 ? lv.f_prev : 0.0;
      const bool conv = sidx >= 1 && fabs(f - fp) / fabs(f) < P.tol;
      stop = (conv || sidx >= P.max_sweeps) ? 1 : 0;
      nevals = sidx + 1;
      f_prev = f;
      if (stop) {
        P.out[OUT_LOGLIK] = ll;
        P.out[OUT_OBJECTIVE] = f;
        P.out[OUT_OBJECTIVE_PREV] = fp;
        P.out[OUT_SWEEPS] = (double)sidx;
        P.out[OUT_CONVERGED] = conv ? 1.0 : 0.0;
        P.out[OUT_ETA_UPDATES] = (double)lv.eta_updates;
        P.out[OUT_PASSES] = (double)(lv.passes + 1);
        P.out[OUT_BATCHES] = (double)(batches_prev + 1);
        ctl->done = 1;
      }
    }
  }
  stop = __shfl_sync(0xffffffffu, stop, 0);
  // lane b: the candidate step of coordinate j0 + b at the current e
  double applied = 0.0, bnew = 0.0, wnew = 0.0;
  const int j = j0 + lane;
  if (!stop && lane < nb) {
    const double beta = ci.beta, width = ci.width;
    const double grad = ci.dtx - ff_to_d(s_tot[lane]);    // l' = delta^T X_j - sum_k d_k G_k
    const double hess = -ff_to_d(s_tot[B + lane]);         // l''
    const double step = newton_step(beta, grad, hess, P.penalty, ci.pen);
    if (step != 0.0) applied = copysign(fmin(fabs(step), width), step);
    bnew = beta + applied;
    wnew = fmax(2.0 * fabs(applied), width / 2.0);
  }
  // commit in order up to and including the first nonzero step
  const unsigned nz = __ballot_sync(0xffffffffu, lane < nb && applied != 0.0);
  const int bstar = nz ? __ffs((int)nz) - 1 : nb - 1;
  if (!stop && lane <= bstar) {
    P.beta[j] = bnew;
    P.width[j] = wnew;
  }
  const double app = nz ? __shfl_sync(0xffffffffu, applied, bstar) : 0.0;
  long long passes = 0, eta_updates = 0, batches = 0;
  if (lane == 0) {
    passes = lv.passes + (stop ? 1 : bstar + 1);
    eta_updates = lv.eta_updates + (nz && !stop ? 1 : 0);
    batches = batches_prev + 1;
  }
  passes = __shfl_sync(0xffffffffu, passes, 0);
  eta_updates = __shfl_sync(0xffffffffu, eta_updates, 0);
  batches = __shfl_sync(0xffffffffu, batches, 0);
  nevals = __shfl_sync(0xffffffffu, nevals, 0);
  f_prev = __shfl_sync(0xffffffffu, f_prev, 0);
  int j0n = j0 + bstar + 1;
  if (j0n >= P.p) j0n = 0;
  const ff delta = d_to_ff(stop ? 0.0 : app);
  CtlLine* L = &ctl->line[lane];
  L->stop = stop;
  L->nevals = nevals;
  L->applied = stop ? 0.0 : app;
  L->delta_hi = delta.hi;
  L->delta_lo = delta.lo;
  L->f_prev = f_prev;
  L->passes = passes;
  L->eta_updates = eta_updates;
  L->j0 = stop ? j0 : j0n;
  L->q = (nz && !stop) ? j0 + bstar : -1;
  L->batches = batches;
  L->dirty = 0;  // the batch's pass stored the sums of e at the current e
  if (lane == 0) ctl->ticket = 0u;
}

template <int B>
__global__ void __launch_bounds__(kStNT) k_strans(const __grid_constant__ CcdParams P, int slot) {
  constexpr int R = SpCfg<B>::R;
  constexpr int NP = SpCfg<B>::NP;
  __shared__ ff s_wp[kStWarps][R];
  __shared__ ff s_T[R];
  __shared__ ff s_red[kStWarps][NP];
  __shared__ ff s_tot[NP];
  __shared__ int s_stop, s_j0, s_last;
  __shared__ double s_lin[2];
  GraphCtl* ctl = P.gctl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int WPC = P.wpc, c = blockIdx.x, G = P.G;
  const int kc_lo = P.wk0[c * WPC], kc_hi = P.wk0[(c + 1) * WPC];
  pdl_wait();
  LineView lv;
  long long batches_prev = 0;
  if (tid == 0) {
    lv = load_line(ctl, c);
    s_stop = lv.stop;
    s_j0 = __ldcg(&ctl->line[c % kRep].j0);
    batches_prev = __ldcg(&ctl->line[c % kRep].batches);
  }
  __syncthreads();
  if (s_stop) return;
  const int j0 = s_j0;
  const int nb = min(B, P.p - j0);
  const bool eval = j0 == 0;

  // prefix of the aggregates of the CTAs before c, fixed order
  {
    const uint64_t* agg = P.agg + (size_t)(c % kRep) * R * G;
    ff t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) t[r] = ff_zero();
    for (int qc = tid; qc < c; qc += kStNT)
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = ff_add(t[r], unpack8<ff>(__ldcg(agg + (size_t)r * G + qc)));
    warp_sum_n<R>(t);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < R; ++r) s_wp[w][r] = t[r];
  }
  __syncthreads();
  if (tid < R) {
    ff a = s_wp[0][tid];
    for (int q = 1; q < kStWarps; ++q) a = ff_add(a, s_wp[q][tid]);
    s_T[tid] = a;
  }
  __syncthreads();

  // G and H of the B columns at the CTA's group ends (steps 3-4): one
  // thread per (group end, column); column b's thread also adds the end's
  // d_k log den_k on evaluation passes when b = 0
  ff f1[B], f2[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    f1[b] = ff_zero();
    f2[b] = ff_zero();
  }
  double pl = 0.0;
  const ff* rec = reinterpret_cast<const ff*>(P.rec);
  const int nwork = (kc_hi - kc_lo) * nb;
  for (int it = tid; it < nwork; it += kStNT) {
    const int k = kc_lo + it / nb, b = it - (it / nb) * nb;
    const int d = P.dk[k];
    if (d == 0) continue;
    const int gwk = (int)((P.gend[k] >> 5) / P.wpw);
    const ff den = ff_add(ff_add(s_T[0], unpack8<ff>(__ldcg(P.wt + gwk))), rec[(size_t)k * R]);
    const ff n1 = ff_add(ff_add(s_T[1 + 2 * b], unpack8<ff>(__ldcg(P.wt + (size_t)(1 + 2 * b) * P.nwarps + gwk))),
                         rec[(size_t)k * R + 1 + 2 * b]);
    const ff n2 = ff_add(ff_add(s_T[2 + 2 * b], unpack8<ff>(__ldcg(P.wt + (size_t)(2 + 2 * b) * P.nwarps + gwk))),
                         rec[(size_t)k * R + 2 + 2 * b]);
    const ff inv = ff_div(ff{1.f, 0.f}, den);
    const ff Gk = ff_mul(n1, inv);
    const ff Hk = ff_mul(n2, inv);
    const ff g1 = ff_mul_f(Gk, (float)d);
    const ff g2 = ff_mul_f(ff_sub(Hk, ff_mul(Gk, Gk)), (float)d);
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (q == b) {
        f1[q] = ff_add(f1[q], g1);
        f2[q] = ff_add(f2[q], g2);
      }
    if (eval && b == 0) pl += (double)d * log(ff_to_d(den));
  }
  // CTA partials, fixed order
  {
    ff v[NP];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      v[b] = f1[b];
      v[B + b] = f2[b];
    }
    v[2 * B] = d_to_ff(pl);
    warp_sum_n<NP>(v);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < NP; ++r) s_red[w][r] = v[r];
  }
  __syncthreads();
  uint64_t* part = reinterpret_cast<uint64_t*>(P.slot_part);
  // thread r sums partial r over the warps (fixed order) and stores it
  if (tid < NP) {
    ff a = s_red[0][tid];
    for (int q = 1; q < kStWarps; ++q) a = ff_add(a, s_red[q][tid]);
    part[(size_t)tid * G + c] = pack8(a);
  }
  __syncthreads();
  if (tid == 0) {
    // the CTA's partials (stored by several threads, ordered before this
    // thread by the barrier) are visible to whoever sees the count
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    unsigned prev;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&ctl->ticket) : "memory");
    s_last = prev == (unsigned)(G - 1);
  }
  pdl_launch_dependents();
  __syncthreads();
  if (!s_last) return;

  // ------------------------------------ last CTA: the steps of the batch
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  for (int r = w; r < NP; r += kStWarps) {
    ff acc = ff_zero();
    for (int qc = lane; qc < G; qc += 32) acc = ff_add(acc, unpack8<ff>(__ldcg(part + (size_t)r * G + qc)));
    acc = warp_sum(acc);
    if (lane == 0) s_tot[r] = acc;
  }
  if (w == kStWarps - 1 && eval) {
    double lin, pen;
    warp_lin_pen(P, -1, 0.0, lin, pen);
    if (lane == 0) {
      s_lin[0] = lin;
      s_lin[1] = pen;
    }
  }
  __syncthreads();
  if (w != 0) return;
  commit_batch<B>(P, lv, batches_prev, j0, nb, eval, s_tot, s_lin, load_coord(P, j0, nb));
}


// ---------------------------------------------------------------------------
// Indicator columns (CSC without values: every nonzero is 1, so x^2 = x and
// e x^2 = e x).  One numerator component per column: R = 1 + B record and
// aggregate components, and H_k = G_k, so H_k - G_k^2 = G_k (1 - G_k).
//   k_ipass   as k_spass, but the B column walks run in lockstep: each round
//             issues the row-index loads of every column, then the gathers
//             of e, so one DRAM and one L2 round trip serve all B columns;
//             the lanes keep float-float partials and one reduce-scatter
//             over the R components gives the warp totals.
//   k_itrans  every CTA scans the pass CTAs' aggregates (one per thread, in
//             shared memory) and takes an even share of the (group end,
//             column) items: G_k of the B columns, partial sums; the last CTA
//             commits the batch.  It reads its control line before waiting:
//             the line was written by the previous batch's transform, which
//             finished before this batch's pass kernel passed its own wait.
template <int B>
struct IpCfg {
  static constexpr int R = 1 + B;
  static constexpr int RP = R <= 2 ? 2 : (R <= 4 ? 4 : (R <= 8 ? 8 : (R <= 16 ? 16 : 32)));
  static constexpr int NP = 2 * B + 1;
  static constexpr int NPP = NP <= 2 ? 2 : (NP <= 4 ? 4 : (NP <= 8 ? 8 : (NP <= 16 ? 16 : 32)));
  // rounds of 32 nonzeros per column in flight: one (two spilled at the
  // 64-register cap of two CTAs per SM and measured 2 % slower)
  static constexpr int SR = 1;
};
constexpr int kItNT = 512;   // transform kernel threads
constexpr int kItWarps = kItNT / 32;

// Position of the warp's group end k (k warp-uniform): lane registers for
// the first 32, a broadcast load beyond.
__device__ __forceinline__ int end_at(const int32_t* gend, int k, int k_lo, int k_hi, int kreg) {
  if (k >= k_hi) return INT_MAX;
  const int i = k - k_lo;
  if (i < 32) return __shfl_sync(0xffffffffu, kreg, i);
  return __ldg(gend + k);
}

// The B columns' nonzeros in the warp's rows: col[b] points at the first,
// len[b] entries.  At each group end before a column's last nonzero the
// warp-relative prefix of e x is stored in rec[k * R + 1 + b]; acc[b] gets
// the lane partials, kn[b] the first end not written.
// The row indices of the first 32 SR nonzeros of each column are loaded by
// ip_first_rows before the dense walk, so their DRAM latency overlaps it.
template <int B, int SR>
__device__ __forceinline__ void ip_first_rows(const int32_t* const (&col)[B], const int (&len)[B],
                                              int (&row0)[B][SR]) {
  const int lane = threadIdx.x & 31;
  const uint64_t strm = l2_stream();
#pragma unroll
  for (int b = 0; b < B; ++b)
#pragma unroll
    for (int r = 0; r < SR; ++r) {
      const int i = 32 * r + lane;
      row0[b][r] = i < len[b] ? ld_hint(col[b] + i, strm) : INT_MAX;
    }
}

template <int B, int SR>
__device__ __forceinline__ void ip_sparse(const float* e, const int32_t* gend, const int32_t* const (&col)[B],
                                          const int (&len)[B], ff* rec, int R, int k_lo, int k_hi, int kreg,
                                          const int (&row0)[B][SR], ff (&acc)[B], int (&kn)[B]) {
  const int lane = threadIdx.x & 31;
  const uint64_t keep = l2_keep(), strm = l2_stream();
  int ne[B];
  int len_max = 0;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    acc[b] = ff_zero();
    kn[b] = k_lo;
    ne[b] = end_at(gend, k_lo, k_lo, k_hi, kreg);
    len_max = max(len_max, len[b]);
  }
  // the row indices of the next rounds are loaded one iteration ahead, so
  // their DRAM latency overlaps this round's gathers of e
  int rown[B][SR];
#pragma unroll
  for (int b = 0; b < B; ++b)
#pragma unroll
    for (int r = 0; r < SR; ++r) rown[b][r] = row0[b][r];
  for (int base = 0; base < len_max; base += 32 * SR) {
    int row[B][SR];
    float ev[B][SR];
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < SR; ++r) {
        row[b][r] = rown[b][r];
        const int i = base + 32 * SR + 32 * r + lane;
        rown[b][r] = i < len[b] ? ld_hint(col[b] + i, strm) : INT_MAX;
      }
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < SR; ++r) ev[b][r] = row[b][r] != INT_MAX ? ld_hint(e + row[b][r], keep) : 0.f;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < SR; ++r) {
        const int rb = base + 32 * r;
        if (rb >= len[b]) continue;
        const int nvalid = min(32, len[b] - rb);
        const int last_row = __shfl_sync(0xffffffffu, row[b][r], nvalid - 1);
        while (ne[b] < last_row) {
          // the warp-relative prefix at the end: the lanes' float-float
          // partials summed as two FP32 trees (high and low words), error at
          // most 5u of this warp's piece of the prefix
          const ff v = ff_add_f(acc[b], row[b][r] <= ne[b] ? ev[b][r] : 0.f);
          float h = v.hi, l = v.lo;
#pragma unroll
          for (int d = 16; d > 0; d >>= 1) {
            h += __shfl_xor_sync(0xffffffffu, h, d);
            l += __shfl_xor_sync(0xffffffffu, l, d);
          }
          if (lane == 0) rec[(size_t)kn[b] * R + 1 + b] = fast_two_sum(h, l);
          ++kn[b];
          ne[b] = end_at(gend, kn[b], k_lo, k_hi, kreg);
        }
        acc[b] = ff_add_f(acc[b], ev[b][r]);
      }
  }
}

template <int B>
__global__ void __launch_bounds__(kSpNT, 2) k_ipass(const __grid_constant__ CcdParams P, int slot) {
  constexpr int R = IpCfg<B>::R, RP = IpCfg<B>::RP, SR = IpCfg<B>::SR;
  __shared__ ff s_wtot[kMaxWarpsPerCta][R];
  __shared__ int s_stop, s_j0, s_q, s_dirty;
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
  const int k_lo = P.wk0[gw], k_hi = P.wk0[gw + 1];
  const int kreg = k_lo + lane < k_hi ? P.gend[k_lo + lane] : INT_MAX;
  pdl_wait();
  if (tid == 0) {
    const CtlLine* L = &P.gctl->line[c % kRep];
    s_stop = __ldcg(&L->stop);
    s_j0 = __ldcg(&L->j0);
    s_q = __ldcg(&L->q);
    s_applied = __ldcg(&L->applied);
    s_delta[0] = __ldcg(&L->delta_hi);
    s_delta[1] = __ldcg(&L->delta_lo);
    s_dirty = __ldcg(&L->dirty);
  }
  __syncthreads();
  if (s_stop) return;
  const int j0 = s_j0;
  const int nb = min(B, P.p - j0);
  // e changes only through a nonzero step: when the pending step is zero
  // (and the fit has passed its first batch) e is the e of the previous
  // pass, and so are the prefix of e at the group ends, the warp offsets and
  // the CTA aggregate of that component, which stay where that pass stored
  // them, bit for bit
  const bool dense = s_applied != 0.0 || s_dirty != 0;
  const int nw1 = P.nwarps + 1;
  const int32_t* col[B];
  int len[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = b < nb ? j0 + b : j0;
    const int a = P.woff[(size_t)j * nw1 + gw];
    const int z = P.woff[(size_t)j * nw1 + gw + 1];
    col[b] = P.row_idx + P.col_ptr[j] + a;
    len[b] = b < nb ? z - a : 0;
  }
  if (s_applied != 0.0) warp_update<0, float>(P, s_q, gw, row_lo, row_hi, s_applied, ff{s_delta[0], s_delta[1]});
  ff* rec = reinterpret_cast<ff*>(P.rec);
  const float* e = reinterpret_cast<const float*>(P.e);
  int row0[B][SR];
  ip_first_rows<B, SR>(col, len, row0);
  ff tot[RP];
  tot[0] = dense ? sp_dense(e, P.gend, row_lo, row_hi, rec, R, EndCursor{k_lo, k_hi, k_lo, kreg}) : ff_zero();
  int kn[B];
  {
    ff acc[B];
    ip_sparse<B, SR>(e, P.gend, col, len, rec, R, k_lo, k_hi, kreg, row0, acc, kn);
#pragma unroll
    for (int b = 0; b < B; ++b) tot[1 + b] = acc[b];
  }
#pragma unroll
  for (int m = R; m < RP; ++m) tot[m] = ff_zero();
  warp_reduce_scatter<RP>(tot, lane);
  const int comp = warp_rs_component<RP>(lane);
  if (comp < R && lane == warp_rs_lane<RP>(comp)) {
    s_wtot[w][comp] = tot[0];  // component 0 is used only when the dense walk ran
    // group ends after the column's last nonzero in the warp's rows see the
    // warp total
    if (comp >= 1) {
      int k0 = k_hi;
#pragma unroll
      for (int b = 0; b < B; ++b)
        if (comp == 1 + b) k0 = kn[b];
      for (int k = k0; k < k_hi; ++k) rec[(size_t)k * R + comp] = tot[0];
    }
  }
  pdl_launch_dependents();
  __syncthreads();
  // warp m scans component m over the CTA's warps (component 0 only after
  // a dense walk)
  for (int m = dense ? w : w + 1; m < R; m += WPC) {
    ff v = ff_zero();
    if (lane < WPC) v = s_wtot[lane][m];
    const ff incl = warp_inclusive_scan(v, lane);
    ff ex = shfl_up(incl, 1);
    if (lane == 0) ex = ff_zero();
    if (lane < WPC) P.wt[(size_t)m * P.nwarps + c * WPC + lane] = pack8(ex);
    const ff t = shfl_idx(incl, WPC - 1);
    if (lane == 0) P.agg[(size_t)m * G + c] = pack8(t);
  }
}

template <int B>
__global__ void __launch_bounds__(kItNT, 1) k_itrans(const __grid_constant__ CcdParams P, int slot) {
  constexpr int R = IpCfg<B>::R, NP = IpCfg<B>::NP, NPP = IpCfg<B>::NPP;
  __shared__ ff s_T[kItNT][R];           // exclusive prefix of the pass CTAs' aggregates (G <= kItNT)
  __shared__ ff s_w[kItWarps][R];        // warp totals of that scan, then their exclusive prefix
  __shared__ ff s_red[kItWarps][NP];
  __shared__ ff s_tot[NP];
  __shared__ int s_stop, s_j0, s_last;
  __shared__ double s_lin[2];
  GraphCtl* ctl = P.gctl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int WPC = P.wpc, G = P.G, G2 = gridDim.x, c2 = blockIdx.x;
  LineView lv;
  long long batches_prev = 0;
  if (tid == 0) {
    lv = load_line(ctl, c2);
    s_stop = lv.stop;
    s_j0 = __ldcg(&ctl->line[c2 % kRep].j0);
    batches_prev = __ldcg(&ctl->line[c2 % kRep].batches);
  }
  __syncthreads();
  if (s_stop) {
    pdl_wait();
    return;
  }
  const int j0 = s_j0;
  const int nb = min(B, P.p - j0);
  const bool eval = j0 == 0;
  // work items (group end k, column b), k = item / nb, spread over all
  // threads of the grid; the first item's group table entries (written by
  // the prep) are loaded before the wait
  const int nwork = P.K * nb;
  const int stride = G2 * kItNT;
  const int it0 = c2 * kItNT + tid;
  int d1 = 0, gw1 = 0;
  if (it0 < nwork) {
    const int k = it0 / nb;
    d1 = P.dk[k];
    gw1 = (int)((P.gend[k] >> 5) / P.wpw);
  }
  // the batch's coordinate scalars for the commit (written by the previous
  // batch's commit, finished before this kernel launched)
  CoordIn ci;
  if (w == 0) ci = load_coord(P, j0, nb);
  pdl_wait();

  // exclusive prefix over the pass CTAs of their aggregates, fixed order
  {
    ff v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = tid < G ? unpack8<ff>(__ldcg(P.agg + (size_t)m * G + tid)) : ff_zero();
    ff incl[R];
#pragma unroll
    for (int m = 0; m < R; ++m) incl[m] = v[m];
    warp_scan_n<R>(incl, lane);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      ff ex = shfl_up(incl[m], 1);
      v[m] = lane == 0 ? ff_zero() : ex;   // exclusive within the warp
    }
    if (lane == 31)
#pragma unroll
      for (int m = 0; m < R; ++m) s_w[w][m] = incl[m];
    __syncthreads();
    if (w == 0) {
      ff t[R];
#pragma unroll
      for (int m = 0; m < R; ++m) t[m] = lane < kItWarps ? s_w[lane][m] : ff_zero();
      warp_scan_n<R>(t, lane);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const ff ex = shfl_up(t[m], 1);
        if (lane < kItWarps) s_w[lane][m] = lane == 0 ? ff_zero() : ex;
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < R; ++m) s_T[tid][m] = ff_add(s_w[w][m], v[m]);
  }
  __syncthreads();

  // G_k of the batch's columns at the group ends (steps 3-4); column 0's
  // item also adds d_k log den_k on evaluation passes
  ff f1[B], f2[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    f1[b] = ff_zero();
    f2[b] = ff_zero();
  }
  double pl = 0.0;
  const ff* rec = reinterpret_cast<const ff*>(P.rec);
  for (int it = it0; it < nwork; it += stride) {
    const int k = it / nb, b = it - k * nb;
    int d, gwk;
    if (it == it0) {
      d = d1, gwk = gw1;
    } else {
      d = P.dk[k];
      gwk = (int)((P.gend[k] >> 5) / P.wpw);
    }
    if (d == 0) continue;
    const int f = gwk / WPC;
    const ff den = ff_add(ff_add(s_T[f][0], unpack8<ff>(__ldcg(P.wt + gwk))), rec[(size_t)k * R]);
    const ff n1 = ff_add(ff_add(s_T[f][1 + b], unpack8<ff>(__ldcg(P.wt + (size_t)(1 + b) * P.nwarps + gwk))),
                         rec[(size_t)k * R + 1 + b]);
    const ff Gk = ff_div(n1, den);
    const ff g1 = ff_mul_f(Gk, (float)d);
    const ff g2 = ff_mul_f(ff_sub(Gk, ff_mul(Gk, Gk)), (float)d);
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (q == b) {
        f1[q] = ff_add(f1[q], g1);
        f2[q] = ff_add(f2[q], g2);
      }
    if (eval && b == 0) pl += (double)d * log(ff_to_d(den));
  }
  // CTA partials, fixed order
  {
    ff v[NPP];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      v[b] = f1[b];
      v[B + b] = f2[b];
    }
    v[2 * B] = d_to_ff(pl);
#pragma unroll
    for (int m = NP; m < NPP; ++m) v[m] = ff_zero();
    warp_reduce_scatter<NPP>(v, lane);
    const int comp = warp_rs_component<NPP>(lane);
    if (comp < NP && lane == warp_rs_lane<NPP>(comp)) s_red[w][comp] = v[0];
  }
  __syncthreads();
  uint64_t* part = reinterpret_cast<uint64_t*>(P.slot_part);
  if (tid < NP) {
    ff a = s_red[0][tid];
    for (int q = 1; q < kItWarps; ++q) a = ff_add(a, s_red[q][tid]);
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

  // ------------------------------------ last CTA: the steps of the batch
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  for (int r = w; r < NP; r += kItWarps) {
    ff acc = ff_zero();
    for (int qc = lane; qc < G2; qc += 32) acc = ff_add(acc, unpack8<ff>(__ldcg(part + (size_t)r * G2 + qc)));
    acc = warp_sum(acc);
    if (lane == 0) s_tot[r] = acc;
  }
  if (w == kItWarps - 1 && eval) {
    double lin, pen;
    warp_lin_pen(P, -1, 0.0, lin, pen);
    if (lane == 0) {
      s_lin[0] = lin;
      s_lin[1] = pen;
    }
  }
  __syncthreads();
  if (w != 0) return;
  commit_batch<B>(P, lv, batches_prev, j0, nb, eval, s_tot, s_lin, ci);
}

// CTAs of the transform kernel for K group ends and B columns: about one
// (end, column) item per thread, at least 8, at most 152.
int itrans_ctas(int K, int B) { return std::max(8, std::min(152, (K * B + kItNT - 1) / kItNT)); }

template <int B>
cudaError_t capture_spec(const CcdParams& P, int S, bool pdl, cudaStream_t cs, cudaGraph_t* g) {
  cudaError_t st = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (st != cudaSuccess) return st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cudaLaunchConfig_t cp = {};
  cp.gridDim = dim3(P.G);
  cp.blockDim = dim3(kSpNT);
  cp.stream = cs;
  cp.attrs = attr;
  cp.numAttrs = 1;
  cudaLaunchConfig_t ct = cp;
  ct.blockDim = dim3(kStNT);
  // indicator columns: the lockstep walks and the ranged transform
  const bool ind = P.values == nullptr;
  if (ind) {
    if (P.G > kItNT) return cudaErrorInvalidValue;   // the transform scans one aggregate per thread
    ct.gridDim = dim3(itrans_ctas(P.K, B));
    ct.blockDim = dim3(kItNT);
  }
  cudaError_t lst = cudaSuccess;
  for (int slot = 0; slot < S && lst == cudaSuccess; ++slot) {
    lst = ind ? cudaLaunchKernelEx(&cp, k_ipass<B>, P, slot) : cudaLaunchKernelEx(&cp, k_spass<B>, P, slot);
    if (lst == cudaSuccess)
      lst = ind ? cudaLaunchKernelEx(&ct, k_itrans<B>, P, slot) : cudaLaunchKernelEx(&ct, k_strans<B>, P, slot);
  }
  st = cudaStreamEndCapture(cs, g);
  return lst != cudaSuccess ? lst : st;
}

// the kernels for B columns a batch (one fit)
cudaError_t capture_any_spec(const CcdParams& P, int B, int S, bool pdl, cudaStream_t cs, cudaGraph_t* g) {
  if (P.nfit > 0) return cudaErrorInvalidValue;
  return B == 4 ? capture_spec<4>(P, S, pdl, cs, g) : capture_spec<8>(P, S, pdl, cs, g);
}

}  // namespace

// Slots (batches) per graph replay for p coordinates and B columns a batch.
// About half a sweep's worth when most steps are zero: the replay in which
// a fit stops, and the one queued behind it, run their remaining batches
// empty, so shorter replays waste less.
int spec_slots(int p, int B) { return std::max(8, ((p + B - 1) / B + 1) / 2 + 2); }

cudaError_t run_spec_graph(const CcdParams& P, int B, cudaStream_t s, GraphCache* gc, cudaEvent_t t0, int* replays,
                           int* launches) {
  *replays = 0;
  *launches = 0;
  if (B != 4 && B != 8) return cudaErrorInvalidValue;
  GraphCache local;
  struct LocalGuard {
    GraphCache* g;
    ~LocalGuard() { graph_cache_free(g); }
  } guard{gc ? nullptr : &local};
  if (!gc) gc = &local;
  cudaError_t st;
  if ((st = graph_cache_prepare(gc)) != cudaSuccess) return st;
  const bool pdl = !P.no_pdl;
  const int S = spec_slots(P.p, B);
  const int mlp = 2000 + B * 2 + (pdl ? 1 : 0);
  if (!gc->exec || gc->mlp != mlp || std::memcmp(&gc->key, &P, sizeof(P)) != 0) {
    if (gc->exec) {
      cudaGraphExecDestroy(gc->exec);
      gc->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    st = capture_any_spec(P, B, S, pdl, gc->cs, &g);
    if (st == cudaSuccess) st = cudaGraphInstantiate(&gc->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != cudaSuccess) {
      gc->exec = nullptr;
      return st;
    }
    gc->key = P;
    gc->mlp = mlp;
  }
  // every batch commits at least one coordinate, so max_sweeps sweeps and
  // the final evaluation take at most max_sweeps * p + 1 batches
  const int64_t max_batches = (int64_t)P.max_sweeps * P.p + 1;
  const int max_replays = (int)std::min<int64_t>((max_batches + S - 1) / S + 2, 1 << 30);
  return replay_until_stop(P, s, gc, t0, 2 * S, replays, launches, max_replays);
}

}  // namespace survgpu
