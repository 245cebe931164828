// Differentiable form (Section 2.9): the Cox negative log partial likelihood
// (Breslow ties) of C linear predictors at once, eta = X B, and its gradient
// with respect to B.
//
//   forward   Bcat^T = [B_hi | B_lo]^T (bf16 split of the FP32 B), the
//             tensor-core product eta = X B_hi + X B_lo (nll_tc.cu: TMA,
//             tcgen05.mma with FP32 accumulators in TMEM), then the risk-set
//             scan: e = exp(eta); every lane of a warp owns two of the C
//             columns and walks the warp's rows in order with float-float
//             running sums, so a group end costs its lanes a store, not a
//             reduction; a per-column kernel adds the prefix of the warps
//             before, takes d_k log den_k in FP64 and returns
//             NLL_b = -sum_i delta_i eta_ib + sum_k d_k log den_kb.
//   backward  Lambda_kb = sum_{k' >= k} d_k' / den_k'b (reverse scan per
//             column), G_ib = g_b (e_ib Lambda_b(group of i) - delta_i) split
//             into bf16 [G_hi | G_lo], the tensor-core product X^T Gcat
//             (nll_tc.cu), its halves and CTA partials summed in FP64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "tc.cuh"
#include "survgpu.h"
#include "workspace.h"

namespace survgpu {
namespace {

constexpr int kNllThreads = 512;   // scan kernels: two CTAs of 16 warps per SM
constexpr int kNllMaxCols = 64;    // two columns per lane

// B (p x C, row-major FP32) -> Bcat^T (2 Cp rows of ld bf16): row c < C holds
// hi(B[:, c]), row Cp + c holds lo(B[:, c]) = bf16(B - hi); every other entry
// (padding rows and columns p..ld-1) is zero.
__global__ void k_split_bt(const float* B, int64_t p, int C, int Cp, int64_t ld, __nv_bfloat16* BcatT) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int NB = 2 * Cp;
  if (i >= (int64_t)NB * ld) return;
  const int r = (int)(i / ld);
  const int64_t j = i - (int64_t)r * ld;
  const int c = r < Cp ? r : r - Cp;
  __nv_bfloat16 v = __float2bfloat16_rn(0.f);
  if (c < C && j < p) {
    const float b = B[j * C + c];
    const __nv_bfloat16 hi = __float2bfloat16_rn(b);
    v = r < Cp ? hi : __float2bfloat16_rn(b - __bfloat162float(hi));
  }
  BcatT[i] = v;
}

// X (n x p) -> Xp (n x ld), zero columns p..ld-1 (TMA needs a row pitch that
// is a multiple of 16 bytes)
__global__ void k_pad_x(const __nv_bfloat16* X, int64_t n, int64_t p, int64_t ld, __nv_bfloat16* Xp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * ld) return;
  const int64_t r = i / ld, j = i - r * ld;
  Xp[i] = j < p ? X[r * p + j] : __float2bfloat16_rn(0.f);
}

// eta of columns c0 = 2 lane and c0 + 1 of row r (8-byte loads when C is
// even, streaming: eta is read once per kernel)
__device__ __forceinline__ void load_pair(const float* y, int C, int c0, bool has0, bool has1, float& v0, float& v1) {
  if (has1 && (C & 1) == 0) {
    const float2 h = __ldcs(reinterpret_cast<const float2*>(y + c0));
    v0 = h.x;
    v1 = h.y;
  } else {
    v0 = has0 ? __ldcs(y + c0) : 0.f;
    v1 = has1 ? __ldcs(y + c0 + 1) : 0.f;
  }
}

// Per-warp staging of eta rows in shared memory by 1-D bulk copies (TMA):
// kStages slots of kStRows rows (8 C floats: a multiple of 16 bytes, and
// every stage starts on a 16-byte boundary because warp row ranges start at
// multiples of 32 rows), one mbarrier each.  Stage s (rows r_lo + 8 s ..)
// goes to slot s % kStages; lane 0 issues the copies, kStages ahead of the
// stage the warp reads, and every lane waits (bounded) on the slot's
// barrier.  Nothing of eta passes through registers before it is used, so
// three stages (6 KB a warp for 64 columns) keep the memory system busy.
constexpr int kStRows = 8;
constexpr int kStages = 3;
constexpr uint64_t kStageWaitNs = 2000000000ull;
struct WarpStage {
  float* buf;          // [kStages][kStRows * C]
  uint64_t* bar;       // [kStages]
  const float* src;    // eta + r_lo * C
  int C;
  __device__ __forceinline__ void issue(int64_t s) const {
    const int slot = (int)(s % kStages);
    const uint32_t bytes = (uint32_t)(kStRows * C * 4);
    tc::mbar_arrive_expect_tx(bar + slot, bytes);
    tc::bulk_load(buf + (size_t)slot * kStRows * C, src + (size_t)s * kStRows * C, bytes, bar + slot);
  }
  __device__ __forceinline__ bool wait(int64_t s) const {
    return tc::mbar_wait(bar + (int)(s % kStages), (uint32_t)((s / kStages) & 1), kStageWaitNs);
  }
  // columns c0, c0 + 1 of row u of stage s
  __device__ __forceinline__ void pair(int64_t s, int u, int c0, bool has0, bool has1, float& v0, float& v1) const {
    const float* r = buf + ((size_t)(s % kStages) * kStRows + u) * C;
    if (has1 && (C & 1) == 0) {
      const float2 h = *reinterpret_cast<const float2*>(r + c0);
      v0 = h.x;
      v1 = h.y;
    } else {
      v0 = has0 ? r[c0] : 0.f;
      v1 = has1 ? r[c0 + 1] : 0.f;
    }
  }
};
// Shared memory of the staged scan kernels: kStages stages of every warp.
size_t stage_smem(int C) { return sizeof(float) * (size_t)(kNllThreads / 32) * kStages * kStRows * C; }

// status of rows r0 .. r0 + 7 packed in two words (one 8-byte broadcast load
// when the rows are whole and the address allows it)
__device__ __forceinline__ uint2 load_status8(const int8_t* status, int64_t r0, int64_t r_hi) {
  if (r0 + 8 <= r_hi && ((reinterpret_cast<uintptr_t>(status + r0)) & 7) == 0)
    return __ldg(reinterpret_cast<const uint2*>(status + r0));
  uint32_t w[2] = {0u, 0u};
#pragma unroll
  for (int b = 0; b < 8; ++b)
    if (r0 + b < r_hi) w[b >> 2] |= (uint32_t)(uint8_t)status[r0 + b] << (8 * (b & 3));
  return make_uint2(w[0], w[1]);
}
__device__ __forceinline__ int status_at(uint2 w, int u) {
  return (int)(int8_t)(((u < 4 ? w.x : w.y) >> (8 * (u & 3))) & 0xFFu);
}

// Waits (bounded) for the copies a warp issued and has not read: before a
// CTA that gave up on one of them exits.
__device__ __forceinline__ void drain_stages(const WarpStage& ws, int64_t s, int64_t nfull) {
  for (int64_t q = s; q < nfull && q < s + kStages; ++q) ws.wait(q);
}

// Forward scan.  Warp gw owns rows [gw * rpw, (gw + 1) * rpw); lane l owns
// the adjacent columns 2l and 2l + 1.  Outputs: rec[k][c] (warp-relative
// prefix of e at group end k, float-float), wt[gw][c] and wd[gw][c] (the
// warp's sums of e and of delta * eta).  Whole stages of 8 rows come through
// shared memory (bulk copies); the last rows of a warp (fewer than 8) are
// loaded directly.  A stage wait that expires sets *err.
__global__ void __launch_bounds__(kNllThreads, 2) k_nll_scan(const float* eta, int64_t n, int C, const int8_t* status,
                                                          const int32_t* gend, const int32_t* wk0, int64_t rpw,
                                                          float2* rec, float2* wt, float2* wd, unsigned* err) {
  extern __shared__ __align__(128) float s_stage[];
  __shared__ __align__(8) uint64_t s_bar[kNllThreads / 32][kStages];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int gw = blockIdx.x * (kNllThreads / 32) + wl;
  const int64_t r_lo = min((int64_t)gw * rpw, n), r_hi = min(r_lo + rpw, n);
  const int c0 = 2 * lane;
  const bool has0 = c0 < C, has1 = c0 + 1 < C;
  ff acc0 = ff_zero(), acc1 = ff_zero(), dl0 = ff_zero(), dl1 = ff_zero();
  int kn = wk0[gw];
  const int k_hi = wk0[gw + 1];
  int64_t next_end = kn < k_hi ? (int64_t)gend[kn] : LLONG_MAX;
  // rows r0 .. r0 + nr - 1 (nr <= 8) with their eta values and status
  auto rows = [&](int64_t r0, int nr, const float (&v0)[kStRows], const float (&v1)[kStRows], uint2 st) {
    float p0 = 0.f, p1 = 0.f, q0 = 0.f, q1 = 0.f;
    if (nr == kStRows && next_end >= r0 + kStRows) {
      // no group end among the rows: sums only
#pragma unroll
      for (int u = 0; u < kStRows; ++u) {
        const float dlt = status_at(st, u) == 1 ? 1.f : 0.f;
        p0 += has0 ? expf(v0[u]) : 0.f;
        p1 += has1 ? expf(v1[u]) : 0.f;
        q0 = fmaf(dlt, v0[u], q0);
        q1 = fmaf(dlt, v1[u], q1);
      }
      nr = 0;
    }
#pragma unroll
    for (int u = 0; u < kStRows; ++u) {
      if (u >= nr) break;
      const int64_t r = r0 + u;
      const float e0 = has0 ? expf(v0[u]) : 0.f, e1 = has1 ? expf(v1[u]) : 0.f;
      p0 += e0;
      p1 += e1;
      if (status_at(st, u) == 1) {
        q0 += v0[u];
        q1 += v1[u];
      }
      if (r == next_end) {  // a group end: the lane's running prefix is the warp's
        const ff a0 = ff_add_f(acc0, p0), a1 = ff_add_f(acc1, p1);
        if (has0) rec[(size_t)kn * C + c0] = make_float2(a0.hi, a0.lo);
        if (has1) rec[(size_t)kn * C + c0 + 1] = make_float2(a1.hi, a1.lo);
        ++kn;
        next_end = kn < k_hi ? (int64_t)gend[kn] : LLONG_MAX;
      }
    }
    acc0 = ff_add_f(acc0, p0);
    acc1 = ff_add_f(acc1, p1);
    dl0 = ff_add_f(dl0, q0);
    dl1 = ff_add_f(dl1, q1);
  };
  const WarpStage ws{s_stage + (size_t)wl * kStages * kStRows * C, s_bar[wl], eta + (size_t)r_lo * C, C};
  const int64_t nfull = (r_hi - r_lo) / kStRows;
  if (lane == 0) {
    for (int q = 0; q < kStages; ++q) tc::mbar_init(&s_bar[wl][q], 1);
    tc::mbar_fence_init();
    for (int64_t q = 0; q < nfull && q < kStages; ++q) ws.issue(q);
  }
  __syncwarp();
  uint2 stq[kStages];  // status of the stages in flight
#pragma unroll
  for (int q = 0; q < kStages; ++q) stq[q] = load_status8(status, r_lo + (int64_t)q * kStRows, r_hi);
  for (int64_t s = 0; s < nfull; ++s) {
    if (!__all_sync(0xffffffffu, ws.wait(s))) {
      if (lane == 0) atomicOr(err, 1u);
      drain_stages(ws, s + 1, nfull);
      return;
    }
    float v0[kStRows], v1[kStRows];
#pragma unroll
    for (int u = 0; u < kStRows; ++u) ws.pair(s, u, c0, has0, has1, v0[u], v1[u]);
    const uint2 st = stq[0];
#pragma unroll
    for (int q = 0; q + 1 < kStages; ++q) stq[q] = stq[q + 1];
    stq[kStages - 1] = load_status8(status, r_lo + (s + kStages) * kStRows, r_hi);
    rows(r_lo + s * kStRows, kStRows, v0, v1, st);
    tc::fence_proxy_async();  // this lane's reads of the slot before the copy that refills it
    __syncwarp();
    if (lane == 0 && s + kStages < nfull) ws.issue(s + kStages);
  }
  const int64_t rt = r_lo + nfull * kStRows;
  if (rt < r_hi) {
    float v0[kStRows], v1[kStRows];
#pragma unroll
    for (int u = 0; u < kStRows; ++u) {
      v0[u] = 0.f;
      v1[u] = 0.f;
      if (rt + u < r_hi) load_pair(eta + (rt + u) * C, C, c0, has0, has1, v0[u], v1[u]);
    }
    rows(rt, (int)(r_hi - rt), v0, v1, load_status8(status, rt, r_hi));
  }
  if (has0) {
    wt[(size_t)gw * C + c0] = make_float2(acc0.hi, acc0.lo);
    wd[(size_t)gw * C + c0] = make_float2(dl0.hi, dl0.lo);
  }
  if (has1) {
    wt[(size_t)gw * C + c0 + 1] = make_float2(acc1.hi, acc1.lo);
    wd[(size_t)gw * C + c0 + 1] = make_float2(dl1.hi, dl1.lo);
  }
}

// Per column c, S CTAs of kFinThreads each (grid C x S): prefix of the warp
// totals in a fixed order (chunk sums, a two-level block scan, the prefix
// inside each chunk; every CTA of the column computes it), den_k = prefix
// before the end's warp + rec[k][c] (kept for the backward) and d_k log den_k
// for the ends k = s kFinThreads + tid (stride S kFinThreads): the FP64 logs
// dominate, so the column's ends are spread over S CTAs.  Each CTA stores its
// sums in part[c][s]; the column's last CTA (ticket cnt[c], reset after use)
// adds them in the order s = 0 .. S-1: NLL_c = -sum delta eta + sum_k d_k
// log den_k.
constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads) k_nll_finish(const float2* rec, const float2* wt, const float2* wd,
                                                          int nwarps, int C, const int32_t* gend, const int32_t* dk,
                                                          int K, int64_t rpw, double* den, double* part,
                                                          unsigned* cnt, double* nll) {
  extern __shared__ float2 s_base[];  // [nwarps] exclusive prefix (float-float)
  __shared__ ff s_ws[32];
  __shared__ double s_red[32][2];
  __shared__ int s_last;
  const int c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ch = (nwarps + kFinThreads - 1) / kFinThreads;
  const int w0 = min(tid * ch, nwarps), w1 = min(w0 + ch, nwarps);
  ff cs = ff_zero();
  for (int q = w0; q < w1; ++q) {
    const float2 v = wt[(size_t)q * C + c];
    cs = ff_add(cs, ff{v.x, v.y});
  }
  const ff incl = warp_inclusive_scan(cs, lane);
  if (lane == 31) s_ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    const ff t = warp_inclusive_scan(s_ws[lane], lane);
    const ff ex = shfl_up(t, 1);
    __syncwarp();
    s_ws[lane] = lane == 0 ? ff_zero() : ex;
  }
  __syncthreads();
  const ff up = shfl_up(incl, 1);  // every lane takes part in the shuffle
  ff pre = ff_add(s_ws[w], lane == 0 ? ff_zero() : up);
  for (int q = w0; q < w1; ++q) {
    s_base[q] = make_float2(pre.hi, pre.lo);
    const float2 v = wt[(size_t)q * C + c];
    pre = ff_add(pre, ff{v.x, v.y});
  }
  __syncthreads();
  // the group ends of this CTA: den in FP64, d log den
  const int S = gridDim.y, sc = blockIdx.y;
  double sl = 0.0, sd = 0.0;
  for (int k = sc * kFinThreads + tid; k < K; k += S * kFinThreads) {
    const int q = (int)(gend[k] / rpw);
    const float2 b = s_base[q];
    const float2 r = rec[(size_t)k * C + c];
    const ff pk = ff_add(ff{b.x, b.y}, ff{r.x, r.y});
    const double d = ff_to_d(pk);
    den[(size_t)k * C + c] = d;
    if (dk[k] != 0) sl += (double)dk[k] * log(d);
  }
  if (sc == 0)
    for (int q = tid; q < nwarps; q += kFinThreads) {
      const float2 v = wd[(size_t)q * C + c];
      sd += (double)v.x + (double)v.y;
    }
  sl = warp_sum(sl);
  sd = warp_sum(sd);
  if (lane == 0) {
    s_red[w][0] = sl;
    s_red[w][1] = sd;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < kFinThreads / 32; ++q) {
      a += s_red[q][0];
      b += s_red[q][1];
    }
    part[((size_t)c * S + sc) * 2] = a;
    part[((size_t)c * S + sc) * 2 + 1] = b;
    __threadfence();
    s_last = atomicAdd(cnt + c, 1u) == (unsigned)(S - 1);
  }
  __syncthreads();
  if (tid == 0 && s_last) {
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int q = 0; q < S; ++q) {
      a += __ldcg(part + ((size_t)c * S + q) * 2);
      b += __ldcg(part + ((size_t)c * S + q) * 2 + 1);
    }
    nll[c] = a - b;
    cnt[c] = 0u;  // ready for the next forward
  }
}

// Backward, per column c (one CTA each): Lambda_k = sum_{k' >= k} d_k' / den_k'
// in float-float (den_k' split once into a float-float pair, the quotients
// and a chunked reverse scan in a fixed order; no FP64 division, which costs
// hundreds of cycles a warp on this GPU), stored as FP32.
__global__ void __launch_bounds__(256) k_nll_lambda(const double* den, const int32_t* dk, int K, int C, float* lam) {
  __shared__ ff s_suf[256];   // sum of the chunks after chunk q
  __shared__ ff s_w[8];
  const int c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ch = (K + 255) / 256;
  const int k0 = min(tid * ch, K), k1 = min(k0 + ch, K);
  auto term = [&](int k) { return ff_div(ff{(float)dk[k], 0.f}, d_to_ff(den[(size_t)k * C + c])); };
  ff cs = ff_zero();
  for (int k = k0; k < k1; ++k) cs = ff_add(cs, term(k));
  s_suf[tid] = cs;
  __syncthreads();
  // inclusive scan in reverse chunk order: thread t takes chunk 255 - t
  const ff v = s_suf[255 - tid];
  const ff incl = warp_inclusive_scan(v, lane);
  if (lane == 31) s_w[w] = incl;
  __syncthreads();
  if (w == 0) {
    const ff t = warp_inclusive_scan(lane < 8 ? s_w[lane] : ff_zero(), lane);
    const ff ex = shfl_up(t, 1);
    if (lane < 8) s_w[lane] = lane == 0 ? ff_zero() : ex;
  }
  __syncthreads();
  const ff up = shfl_up(incl, 1);  // every lane takes part in the shuffle
  s_suf[255 - tid] = ff_add(s_w[w], lane == 0 ? ff_zero() : up);   // chunks after 255 - t
  __syncthreads();
  ff run = s_suf[tid];
  for (int k = k1 - 1; k >= k0; --k) {
    run = ff_add(run, term(k));
    lam[(size_t)k * C + c] = __fadd_rn(run.hi, run.lo);
  }
}

// Backward per row: G_ic = g_c (e_ic Lambda_c(group of i) - delta_i), written
// as bf16 in the layout of Bcat: row i holds 2 Cp values, hi(G_ic) at c,
// lo(G_ic) = bf16(G_ic - hi) at Cp + c, zeros in the padding columns.  eta
// comes through shared memory in stages of 8 rows as in the forward scan.
__global__ void __launch_bounds__(kNllThreads, 2) k_nll_grad(const float* eta, int64_t n, int C, int Cp,
                                                          const int8_t* status, const int32_t* gend,
                                                          const int32_t* wk0, int64_t rpw, const float* lam,
                                                          const double* gout, __nv_bfloat16* Gcat, unsigned* err) {
  extern __shared__ __align__(128) float s_stage[];
  __shared__ __align__(8) uint64_t s_bar[kNllThreads / 32][kStages];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int gw = blockIdx.x * (kNllThreads / 32) + wl;
  const int64_t r_lo = min((int64_t)gw * rpw, n), r_hi = min(r_lo + rpw, n);
  const int NB = 2 * Cp;
  const int c0 = 2 * lane;
  const bool has0 = c0 < C, has1 = c0 + 1 < C;
  const bool pad = c0 < Cp;   // lanes whose column pair lies in [0, Cp): they also write the padding zeros
  const float g0 = has0 ? (float)gout[c0] : 0.f, g1 = has1 ? (float)gout[c0 + 1] : 0.f;
  if (r_lo >= r_hi) return;  // warps past the last row
  int kn = wk0[gw];  // group of the current row: the first end at or after it
  float l0 = 0.f, l1 = 0.f;
  auto load_lam = [&]() {
    l0 = has0 ? lam[(size_t)kn * C + c0] : 0.f;
    l1 = has1 ? lam[(size_t)kn * C + c0 + 1] : 0.f;
  };
  int64_t cur_end = (int64_t)gend[kn];  // every row < n lies in some group (the last row ends one)
  load_lam();
  auto rows = [&](int64_t r0, int nr, const float (&v0)[kStRows], const float (&v1)[kStRows], uint2 st) {
    const bool one_group = r0 + nr - 1 <= cur_end;  // every row in the current group
#pragma unroll
    for (int u = 0; u < kStRows; ++u) {
      if (u >= nr) break;
      const int64_t r = r0 + u;
      if (!one_group && r > cur_end) {  // past the end of the current group
        ++kn;
        cur_end = (int64_t)gend[kn];
        load_lam();
      }
      const float d = status_at(st, u) == 1 ? 1.f : 0.f;
      __nv_bfloat16* g = Gcat + r * NB;
      const float x0 = has0 ? g0 * (expf(v0[u]) * l0 - d) : 0.f;
      const float x1 = has1 ? g1 * (expf(v1[u]) * l1 - d) : 0.f;
      const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
      const __nv_bfloat16 m0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
      const __nv_bfloat16 m1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
      if (pad) {  // Cp is a multiple of 16, so c0 + 1 < Cp too: 4-byte stores
        *reinterpret_cast<__nv_bfloat162*>(g + c0) = __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162*>(g + Cp + c0) = __halves2bfloat162(m0, m1);
      }
    }
  };
  const WarpStage ws{s_stage + (size_t)wl * kStages * kStRows * C, s_bar[wl], eta + (size_t)r_lo * C, C};
  const int64_t nfull = (r_hi - r_lo) / kStRows;
  if (lane == 0) {
    for (int q = 0; q < kStages; ++q) tc::mbar_init(&s_bar[wl][q], 1);
    tc::mbar_fence_init();
    for (int64_t q = 0; q < nfull && q < kStages; ++q) ws.issue(q);
  }
  __syncwarp();
  uint2 stq[kStages];
#pragma unroll
  for (int q = 0; q < kStages; ++q) stq[q] = load_status8(status, r_lo + (int64_t)q * kStRows, r_hi);
  for (int64_t s = 0; s < nfull; ++s) {
    if (!__all_sync(0xffffffffu, ws.wait(s))) {
      if (lane == 0) atomicOr(err, 1u);
      drain_stages(ws, s + 1, nfull);
      return;
    }
    float v0[kStRows], v1[kStRows];
#pragma unroll
    for (int u = 0; u < kStRows; ++u) ws.pair(s, u, c0, has0, has1, v0[u], v1[u]);
    const uint2 st = stq[0];
#pragma unroll
    for (int q = 0; q + 1 < kStages; ++q) stq[q] = stq[q + 1];
    stq[kStages - 1] = load_status8(status, r_lo + (s + kStages) * kStRows, r_hi);
    tc::fence_proxy_async();  // this lane's reads of the slot before the copy that refills it
    __syncwarp();
    if (lane == 0 && s + kStages < nfull) ws.issue(s + kStages);
    rows(r_lo + s * kStRows, kStRows, v0, v1, st);
  }
  const int64_t rt = r_lo + nfull * kStRows;
  if (rt < r_hi) {
    float v0[kStRows], v1[kStRows];
#pragma unroll
    for (int u = 0; u < kStRows; ++u) {
      v0[u] = 0.f;
      v1[u] = 0.f;
      if (rt + u < r_hi) load_pair(eta + (rt + u) * C, C, c0, has0, has1, v0[u], v1[u]);
    }
    rows(rt, (int)(r_hi - rt), v0, v1, load_status8(status, rt, r_hi));
  }
}

int cuda_err(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SURV_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  set_last_error_text(buf);
  return e == cudaErrorMemoryAllocation ? SURV_E_NOMEM : SURV_E_CUDA;
}

// Device memory of the current device, or managed memory.
bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == cur;
}

struct NllCtrl {
  unsigned perr;
  int32_t K;
  int32_t total_events;
  int32_t pad;
};

#define NLL_TRY(expr)        \
  do {                       \
    const int rc_ = (expr);  \
    if (rc_) return rc_;     \
  } while (0)

}  // namespace

}  // namespace survgpu

using survgpu::NllCtrl;

extern "C" {

int cox_nll_forward(const surv_nll_data* d, const float* B, double* nll, void* stream, surv_workspace* ws) {
  using namespace survgpu;
  set_last_error_text("");
  if (!d || !B || !nll || !ws) { set_last_error_text("null argument"); return SURV_E_INVALID; }
  const int64_t n = d->n, p = d->p;
  const int C = d->ncols;
  if (n < 1 || n > 0x7fffffff || p < 1 || p > 0x7fffffff || C < 1 || C > kNllMaxCols) {
    set_last_error_text("bad sizes (need n >= 1, p >= 1, 1 <= ncols <= 64)");
    return SURV_E_INVALID;
  }
  if (!on_device(d->time) || !on_device(d->status) || !on_device(d->X) || !on_device(B) || !on_device(nll)) {
    set_last_error_text("time, status, X, B and nll must be device memory");
    return SURV_E_INVALID;
  }
  if (n > 0x7fffff00 || !nll_tc_fits((int)std::min<int64_t>(p, 1 << 20), C)) {
    set_last_error_text("p too large: X B keeps B in shared memory (p <= 512 for 64 columns)");
    return SURV_E_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  using W = surv_workspace;
  void *ctrl_v, *blk, *gend, *dk, *ck, *wk0, *Y, *Bcat, *rec, *wt, *den;
  NLL_TRY(ws_ensure(ws, W::NLL_CTRL, sizeof(NllCtrl), &ctrl_v));
  NllCtrl* ctrl = static_cast<NllCtrl*>(ctrl_v);
  NLL_TRY(cuda_err(cudaMemsetAsync(ctrl, 0, sizeof(NllCtrl), s), "memset"));
  const int32_t* time = static_cast<const int32_t*>(d->time);
  const int8_t* status = static_cast<const int8_t*>(d->status);
  NLL_TRY(cuda_err(prep_check_times(time, status, n, 0, &ctrl->perr, s), "check times"));
  const int64_t nb = prep_end_blocks(n);
  NLL_TRY(ws_ensure(ws, W::NLL_BLK, 4 * (size_t)nb, &blk));
  NLL_TRY(cuda_err(prep_count_ends(time, n, static_cast<int32_t*>(blk), &ctrl->K, s), "count ends"));
  NllCtrl hc;
  unsigned prev_err = 0;
  NLL_TRY(cuda_err(cudaMemcpyAsync(&hc, ctrl, sizeof(hc), cudaMemcpyDeviceToHost, s), "copy"));
  if (ws->nll_err_init)
    NLL_TRY(cuda_err(cudaMemcpyAsync(&prev_err, ws->bufs[W::NLL_ERR].p, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                     "copy"));
  NLL_TRY(cuda_err(cudaStreamSynchronize(s), "sync"));
  if (prev_err) {
    // a bounded wait of an earlier forward or backward on this workspace
    // expired: its results were not valid
    NLL_TRY(cuda_err(cudaMemsetAsync(ws->bufs[W::NLL_ERR].p, 0, sizeof(unsigned), s), "memset"));
    set_last_error_text("a device-side wait of an earlier cox_nll call on this workspace expired");
    return SURV_E_DEVICE_TIMEOUT;
  }
  if (hc.perr & PREP_UNSORTED) { set_last_error_text("time is not non-increasing"); return SURV_E_UNSORTED; }
  if (hc.perr & PREP_STATUS) { set_last_error_text("status code out of range"); return SURV_E_STATUS; }
  const int K = hc.K;
  NLL_TRY(ws_ensure(ws, W::NLL_GEND, 4 * (size_t)K, &gend));
  NLL_TRY(ws_ensure(ws, W::NLL_DK, 4 * (size_t)K, &dk));
  NLL_TRY(ws_ensure(ws, W::GK, 4 * (size_t)K, &ck));
  NLL_TRY(cuda_err(prep_write_ends(time, n, static_cast<const int32_t*>(blk), static_cast<int32_t*>(gend), s),
                   "write ends"));
  NLL_TRY(cuda_err(prep_group_stats(static_cast<int32_t*>(gend), K, status, n, static_cast<int32_t*>(dk),
                                    static_cast<int32_t*>(ck), &ctrl->total_events, s),
                   "group stats"));
  // row partition of the scan kernels: two CTAs of 16 warps per SM
  int dev = 0, sms = 0;
  NLL_TRY(cuda_err(cudaGetDevice(&dev), "device"));
  NLL_TRY(cuda_err(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"));
  const int G = 2 * sms, wpc = kNllThreads / 32, nwarps = G * wpc;
  const int64_t nwords = (n + 31) / 32;
  const int64_t wpw = (nwords + nwarps - 1) / nwarps;
  const int64_t rpw = wpw * 32;
  NLL_TRY(ws_ensure(ws, W::NLL_WK0, 4 * (size_t)(nwarps + 1), &wk0));
  NLL_TRY(cuda_err(prep_warp_groups(static_cast<int32_t*>(gend), K, n, nwarps, rpw, static_cast<int32_t*>(wk0), s),
                   "warp groups"));
  // eta = X B_hi + X B_lo on the tensor cores (nll_tc.cu).  Bcat^T holds the
  // split in 2 Cp rows, Cp = C rounded up to 16 (at least 32); X and Bcat^T
  // rows have a pitch of ld = p rounded up to 8 elements (16 bytes)
  const int Cp = std::max(32, (C + 15) / 16 * 16);
  const int64_t ld = (p + 7) / 8 * 8;
  const void* Xt = d->X;
  if (ld != p || ((uintptr_t)d->X & 15) != 0) {
    void* xp = nullptr;
    NLL_TRY(ws_ensure(ws, W::NLL_XP, sizeof(__nv_bfloat16) * (size_t)n * ld, &xp));
    const int64_t tot = n * ld;
    k_pad_x<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(d->X), n, p, ld,
                                                        static_cast<__nv_bfloat16*>(xp));
    NLL_TRY(cuda_err(cudaGetLastError(), "pad X"));
    Xt = xp;
  }
  NLL_TRY(ws_ensure(ws, W::NLL_Y, sizeof(float) * (size_t)n * C, &Y));
  NLL_TRY(ws_ensure(ws, W::NLL_BCAT, sizeof(__nv_bfloat16) * (size_t)2 * Cp * ld, &Bcat));
  void* errw = nullptr;
  NLL_TRY(ws_ensure(ws, W::NLL_ERR, sizeof(unsigned), &errw));
  if (!ws->nll_err_init) {
    NLL_TRY(cuda_err(cudaMemsetAsync(errw, 0, sizeof(unsigned), s), "memset"));
    ws->nll_err_init = true;
  }
  const int64_t nbt = (int64_t)2 * Cp * ld;
  k_split_bt<<<(unsigned)((nbt + 255) / 256), 256, 0, s>>>(B, p, C, Cp, ld, static_cast<__nv_bfloat16*>(Bcat));
  NLL_TRY(cuda_err(cudaGetLastError(), "split B"));
  NLL_TRY(cuda_err(nll_xb_tc(Xt, n, (int)p, ld, Bcat, C, Cp, static_cast<float*>(Y), static_cast<unsigned*>(errw), s),
                   "tensor-core X B"));
  NLL_TRY(ws_ensure(ws, W::NLL_REC, sizeof(float2) * (size_t)K * C, &rec));
  NLL_TRY(ws_ensure(ws, W::NLL_WT, 2 * sizeof(float2) * (size_t)nwarps * C, &wt));
  NLL_TRY(ws_ensure(ws, W::NLL_DEN, sizeof(double) * (size_t)K * C, &den));
  float2* wt2 = static_cast<float2*>(wt);
  const size_t ssm = stage_smem(C);
  NLL_TRY(cuda_err(cudaFuncSetAttribute(k_nll_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm), "smem"));
  k_nll_scan<<<G, kNllThreads, ssm, s>>>(static_cast<const float*>(Y), n, C, status, static_cast<int32_t*>(gend),
                                         static_cast<int32_t*>(wk0), rpw, static_cast<float2*>(rec), wt2,
                                         wt2 + (size_t)nwarps * C, static_cast<unsigned*>(errw));
  NLL_TRY(cuda_err(cudaGetLastError(), "scan"));
  const size_t smem = sizeof(float2) * (size_t)nwarps;
  if (smem > 48 * 1024)
    NLL_TRY(cuda_err(cudaFuncSetAttribute(k_nll_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                     "smem"));
  // the logs of each column spread over S CTAs (about two waves of the
  // device's SMs in all), their sums combined by the column's last CTA
  const int S = std::max(1, std::min(8, (2 * sms) / C));
  void* fin = nullptr;
  NLL_TRY(ws_ensure(ws, W::NLL_FIN, sizeof(double) * 2 * (size_t)C * S + sizeof(unsigned) * (size_t)C, &fin));
  double* fin_part = static_cast<double*>(fin);
  unsigned* fin_cnt = reinterpret_cast<unsigned*>(fin_part + 2 * (size_t)C * S);
  NLL_TRY(cuda_err(cudaMemsetAsync(fin_cnt, 0, sizeof(unsigned) * (size_t)C, s), "memset"));
  k_nll_finish<<<dim3(C, S), kFinThreads, smem, s>>>(static_cast<float2*>(rec), wt2, wt2 + (size_t)nwarps * C, nwarps,
                                                     C, static_cast<int32_t*>(gend), static_cast<int32_t*>(dk), K, rpw,
                                                     static_cast<double*>(den), fin_part, fin_cnt, nll);
  NLL_TRY(cuda_err(cudaGetLastError(), "finish"));
  ws->nll_n = n;
  ws->nll_p = (int32_t)p;
  ws->nll_c = C;
  ws->nll_K = K;
  ws->nll_G = G;
  ws->nll_wpc = wpc;
  ws->nll_wpw = (int32_t)wpw;
  ws->nll_x = d->X;
  ws->nll_xt = Xt;
  ws->nll_ld = ld;
  return SURV_OK;
}

int cox_nll_backward(const surv_nll_data* d, const double* grad_nll, float* grad_B, void* stream,
                     surv_workspace* ws) {
  using namespace survgpu;
  set_last_error_text("");
  if (!d || !grad_nll || !grad_B || !ws) { set_last_error_text("null argument"); return SURV_E_INVALID; }
  if (ws->nll_n != d->n || ws->nll_p != d->p || ws->nll_c != d->ncols || ws->nll_x != d->X) {
    set_last_error_text("cox_nll_backward must follow cox_nll_forward on the same data and workspace");
    return SURV_E_INVALID;
  }
  if (!on_device(grad_nll) || !on_device(grad_B)) {
    set_last_error_text("grad_nll and grad_B must be device memory");
    return SURV_E_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  using W = surv_workspace;
  const int64_t n = d->n, p = d->p;
  const int C = d->ncols, K = ws->nll_K, G = ws->nll_G, nwarps = G * ws->nll_wpc;
  const int64_t rpw = (int64_t)ws->nll_wpw * 32;
  void *lam, *G2, *part;
  const int Cp = std::max(32, (C + 15) / 16 * 16);
  const int NB = 2 * Cp;
  int nx = 0;
  const size_t part_floats = nll_xtg_part_floats(n, (int)p, NB, &nx);
  NLL_TRY(ws_ensure(ws, W::NLL_LAM, sizeof(float) * (size_t)K * C, &lam));
  NLL_TRY(ws_ensure(ws, W::NLL_G, sizeof(__nv_bfloat16) * (size_t)n * NB, &G2));
  NLL_TRY(ws_ensure(ws, W::NLL_GB, sizeof(float) * part_floats, &part));
  const double* den = static_cast<const double*>(ws->bufs[W::NLL_DEN].p);
  const int32_t* dk = static_cast<const int32_t*>(ws->bufs[W::NLL_DK].p);
  const int32_t* gend = static_cast<const int32_t*>(ws->bufs[W::NLL_GEND].p);
  const int32_t* wk0 = static_cast<const int32_t*>(ws->bufs[W::NLL_WK0].p);
  k_nll_lambda<<<C, 256, 0, s>>>(den, dk, K, C, static_cast<float*>(lam));
  NLL_TRY(cuda_err(cudaGetLastError(), "lambda"));
  const size_t ssm = stage_smem(C);
  NLL_TRY(cuda_err(cudaFuncSetAttribute(k_nll_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm), "smem"));
  k_nll_grad<<<G, kNllThreads, ssm, s>>>(static_cast<const float*>(ws->bufs[W::NLL_Y].p), n, C, Cp,
                                         static_cast<const int8_t*>(d->status), gend, wk0, rpw,
                                         static_cast<float*>(lam), grad_nll, static_cast<__nv_bfloat16*>(G2),
                                         static_cast<unsigned*>(ws->bufs[W::NLL_ERR].p));
  NLL_TRY(cuda_err(cudaGetLastError(), "grad"));
  (void)nwarps;
  // grad_B = X^T [G_hi | G_lo] on the tensor cores, halves and CTA partials
  // summed in FP64 (nll_tc.cu)
  return cuda_err(nll_xtg_tc(ws->nll_xt, n, (int)p, ws->nll_ld, G2, C, Cp, static_cast<float*>(part), nx, grad_B,
                             static_cast<unsigned*>(ws->bufs[W::NLL_ERR].p), s),
                  "tensor-core X^T G");
}

}  // extern "C"
