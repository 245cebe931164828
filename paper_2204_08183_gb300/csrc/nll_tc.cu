// Tensor-core products of the differentiable form (Section 2.9 with eta =
// X B; X bfloat16 n x p row-major, B split into bfloat16 high and low parts),
// hand-written for sm_103a: TMA tile loads into 128-byte-swizzled shared
// memory, tcgen05.mma issued by one thread with the FP32 accumulators in
// tensor memory, tcgen05.ld read-back in the epilogue.
//
//   k_xb_tc   eta = X B: for every tile of 128 rows, D (128 x NB) = X_tile
//             (128 x p, K-major) times Bcat^T (NB x p, K-major, resident in
//             shared memory), NB = 2 Cp columns: B_hi in [0, C), B_lo in
//             [Cp, Cp + C), zeros elsewhere (Cp = C rounded up to 16).  The
//             epilogue writes eta_c = D_c + D_{Cp + c} as FP32 n x C.
//             Persistent CTAs, a ring of X stages, two TMEM accumulators so
//             the epilogue of one tile overlaps the products of the next.
//   k_xtg_tc  dNLL/dB partials: each CTA takes a contiguous range of rows and
//             accumulates D (p x NB) = X_rows^T (MN-major) G_rows (MN-major)
//             over it, 64 rows a stage, in TMEM (two accumulators of 128 p
//             values); the epilogue writes the CTA's partial sums, and
//             k_xtg_reduce adds the partials in a fixed order in FP64 and the
//             high and low halves.
// Warp roles (192 threads): warp 0 issues the TMA loads, warp 1 allocates
// TMEM and issues the MMAs, warps 2-5 read TMEM (warp w reads lanes
// 32 (w % 4) .. + 31).  Every wait is bounded (err gets 1 and the CTA unwinds).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "tc.cuh"

namespace survgpu {
namespace {

using tc::mbar_wait;

constexpr int kTcThreads = 192;
constexpr int kBoxK = 64;            // bfloat16 elements per 128-byte row
constexpr int kFwdRows = 128;        // rows of a forward tile (MMA M)
constexpr int kFwdStages = 8;
constexpr int kBwdRows = 64;         // rows of a backward stage (MMA K, 4 steps of 16)
constexpr int kBwdStages = 4;
constexpr int kBwdP = 256;           // p values of one backward CTA (two MMA tiles of 128)
constexpr uint32_t kTmemCols = 256;
constexpr uint64_t kWaitNs = 2000000000ull;

struct alignas(8) TcBars {
  uint64_t full[kFwdStages];
  uint64_t empty[kFwdStages];
  uint64_t bfull;
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t done;
  uint32_t tmem_base;
  int32_t abort;
};

__device__ __forceinline__ void raise_abort(TcBars* bars, unsigned* err) {
  atomicOr(err, 1u);
  *reinterpret_cast<volatile int32_t*>(&bars->abort) = 1;
}
__device__ __forceinline__ bool aborted(TcBars* bars) {
  return *reinterpret_cast<volatile int32_t*>(&bars->abort) != 0;
}

// ----------------------------------------------------------------- forward
__global__ void __launch_bounds__(kTcThreads, 1)
    k_xb_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapB, int64_t n, int nkb,
            int C, int Cp, int ns, float* __restrict__ eta, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int NB = 2 * Cp;
  const uint32_t bbox = (uint32_t)NB * 128u;              // bytes of one k-block of Bcat^T
  unsigned char* sB = base;                                // nkb boxes
  unsigned char* sA = base + (size_t)nkb * bbox;           // kFwdStages boxes of 16 KB
  TcBars* bars = reinterpret_cast<TcBars*>(sA + (size_t)ns * 16384);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (n + kFwdRows - 1) / kFwdRows;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFwdStages; ++s) {
      tc::mbar_init(&bars->full[s], 1);
      tc::mbar_init(&bars->empty[s], 1);
    }
    tc::mbar_init(&bars->bfull, 1);
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&bars->tfull[a], 1);
      tc::mbar_init(&bars->tempty[a], 128);
    }
    tc::mbar_init(&bars->done, 1);
    bars->abort = 0;
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(&bars->tmem_base, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    tc::tma_prefetch_map(&mapX);
    tc::tma_prefetch_map(&mapB);
    tc::mbar_arrive_expect_tx(&bars->bfull, bbox * (uint32_t)nkb);
    for (int kb = 0; kb < nkb; ++kb) tc::tma_load_2d(sB + (size_t)kb * bbox, &mapB, &bars->bfull, kb * kBoxK, 0);
    int64_t it = 0;
    int64_t last_use[kFwdStages];
    for (int s = 0; s < kFwdStages; ++s) last_use[s] = -1;
    for (int64_t i = 0; i < my_tiles && !aborted(bars); ++i) {
      const int64_t tile = blockIdx.x + i * gridDim.x;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = (int)(it % ns);
        const int64_t u = it / ns;
        if (u > 0 && !mbar_wait(&bars->empty[s], (uint32_t)((u - 1) & 1), kWaitNs)) {
          raise_abort(bars, err);
          break;
        }
        tc::mbar_arrive_expect_tx(&bars->full[s], 16384u);
        tc::tma_load_2d(sA + (size_t)s * 16384, &mapX, &bars->full[s], kb * kBoxK, (int)(tile * kFwdRows));
        last_use[s] = u;
      }
    }
    // every issued copy has landed before the CTA may exit
    if (!mbar_wait(&bars->bfull, 0, kWaitNs)) raise_abort(bars, err);
    for (int s = 0; s < ns; ++s)
      if (last_use[s] >= 0 && !mbar_wait(&bars->full[s], (uint32_t)(last_use[s] & 1), kWaitNs)) raise_abort(bars, err);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr bool kMN = false;
    const uint32_t idesc = tc::idesc_bf16_f32(kFwdRows, NB, kMN, kMN);
    bool ok = mbar_wait(&bars->bfull, 0, kWaitNs);
    if (!ok) raise_abort(bars, err);
    int64_t it = 0;
    for (int64_t i = 0; ok && i < my_tiles; ++i) {
      const int a = (int)(i & 1);
      const int64_t ua = i >> 1;
      if (ua > 0 && !mbar_wait(&bars->tempty[a], (uint32_t)((ua - 1) & 1), kWaitNs)) {
        raise_abort(bars, err);
        break;
      }
      tc::fence_after_sync();
      const uint32_t d = tmem + (uint32_t)(a * NB);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = (int)(it % ns);
        const int64_t u = it / ns;
        if (!mbar_wait(&bars->full[s], (uint32_t)(u & 1), kWaitNs) || aborted(bars)) {
          raise_abort(bars, err);
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t a_addr = tc::smem_u32(sA + (size_t)s * 16384);
        const uint32_t b_addr = tc::smem_u32(sB + (size_t)kb * bbox);
#pragma unroll
        for (int k = 0; k < kBoxK / 16; ++k) {
          const uint64_t ad = tc::sdesc_sw128(a_addr + 32u * k, 16u, 1024u);
          const uint64_t bd = tc::sdesc_sw128(b_addr + 32u * k, 16u, 1024u);
          tc::mma_bf16(d, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
        }
        tc::mma_commit(&bars->empty[s]);
      }
      if (ok) tc::mma_commit(&bars->tfull[a]);
    }
    // all MMAs issued by this thread have completed
    tc::mma_commit(&bars->done);
    if (!mbar_wait(&bars->done, 0, kWaitNs)) raise_abort(bars, err);
  } else if (warp >= 2) {
    // ---------------- epilogue: eta = D_hi + D_lo
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const bool vec = (C & 3) == 0;
    for (int64_t i = 0; i < my_tiles; ++i) {
      const int a = (int)(i & 1);
      const int64_t ua = i >> 1;
      if (!mbar_wait(&bars->tfull[a], (uint32_t)(ua & 1), kWaitNs) || aborted(bars)) {
        raise_abort(bars, err);
        break;
      }
      tc::fence_after_sync();
      const int64_t tile = blockIdx.x + i * gridDim.x;
      const int64_t row = tile * kFwdRows + 32 * q + lane;
      float* out = eta + row * C;
      for (int c0 = 0; c0 < Cp; c0 += 16) {
        float hi[16], lo[16];
        tc::tmem_ld16(tmem + lane_off + (uint32_t)(a * NB + c0), hi);
        tc::tmem_ld16(tmem + lane_off + (uint32_t)(a * NB + Cp + c0), lo);
        if (row < n) {
          if (vec && c0 + 16 <= C) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
              *reinterpret_cast<float4*>(out + c0 + 4 * v) =
                  make_float4(hi[4 * v] + lo[4 * v], hi[4 * v + 1] + lo[4 * v + 1], hi[4 * v + 2] + lo[4 * v + 2],
                              hi[4 * v + 3] + lo[4 * v + 3]);
          } else {
#pragma unroll
            for (int v = 0; v < 16; ++v)
              if (c0 + v < C) out[c0 + v] = hi[v] + lo[v];
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&bars->tempty[a]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------------------- backward
// Stage layout: X boxes (64 rows x 64 p values, 8 KB each) for the CTA's p
// range, then G boxes (64 rows x 64 columns, 8 KB each).
__global__ void __launch_bounds__(kTcThreads, 1)
    k_xtg_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapG, int64_t n, int p,
             int NB, int64_t rows_per_cta, float* __restrict__ part, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int p0 = blockIdx.y * kBwdP;                        // first p value of this CTA
  const int pv = min(kBwdP, p - p0);                        // p values (1..256)
  const int nxb = (pv + kBoxK - 1) / kBoxK;                 // X boxes a stage (1..4)
  const int nmt = (pv + 127) / 128;                         // MMA tiles of 128 p values (1..2)
  const int ngb = (NB + kBoxK - 1) / kBoxK;                 // G boxes a stage (1..2)
  const uint32_t stage_bytes = (uint32_t)(nxb + ngb) * 8192u;
  TcBars* bars = reinterpret_cast<TcBars*>(base + (size_t)kBwdStages * 6 * 8192);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r_lo = min((int64_t)blockIdx.x * rows_per_cta, n);
  const int64_t r_hi = min(r_lo + rows_per_cta, n);
  const int64_t nst = (r_hi - r_lo + kBwdRows - 1) / kBwdRows;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kBwdStages; ++s) {
      tc::mbar_init(&bars->full[s], 1);
      tc::mbar_init(&bars->empty[s], 1);
    }
    tc::mbar_init(&bars->tfull[0], 1);
    tc::mbar_init(&bars->done, 1);
    bars->abort = 0;
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(&bars->tmem_base, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0 && lane == 0) {
    tc::tma_prefetch_map(&mapX);
    tc::tma_prefetch_map(&mapG);
    int64_t last_use[kBwdStages];
    for (int s = 0; s < kBwdStages; ++s) last_use[s] = -1;
    for (int64_t it = 0; it < nst && !aborted(bars); ++it) {
      const int s = (int)(it % kBwdStages);
      const int64_t u = it / kBwdStages;
      if (u > 0 && !mbar_wait(&bars->empty[s], (uint32_t)((u - 1) & 1), kWaitNs)) {
        raise_abort(bars, err);
        break;
      }
      unsigned char* st = base + (size_t)s * 6 * 8192;
      const int row = (int)(r_lo + it * kBwdRows);
      tc::mbar_arrive_expect_tx(&bars->full[s], stage_bytes);
      for (int b = 0; b < nxb; ++b) tc::tma_load_2d(st + (size_t)b * 8192, &mapX, &bars->full[s], p0 + b * kBoxK, row);
      for (int b = 0; b < ngb; ++b) tc::tma_load_2d(st + (size_t)(4 + b) * 8192, &mapG, &bars->full[s], b * kBoxK, row);
      last_use[s] = u;
    }
    for (int s = 0; s < kBwdStages; ++s)
      if (last_use[s] >= 0 && !mbar_wait(&bars->full[s], (uint32_t)(last_use[s] & 1), kWaitNs)) raise_abort(bars, err);
  } else if (warp == 1 && lane == 0) {
    constexpr bool kMN = true;
    const uint32_t idesc = tc::idesc_bf16_f32(128, NB, kMN, kMN);
    bool ok = true;
    for (int64_t it = 0; it < nst; ++it) {
      const int s = (int)(it % kBwdStages);
      const int64_t u = it / kBwdStages;
      if (!mbar_wait(&bars->full[s], (uint32_t)(u & 1), kWaitNs) || aborted(bars)) {
        raise_abort(bars, err);
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t st = tc::smem_u32(base + (size_t)s * 6 * 8192);
#pragma unroll
      for (int ks = 0; ks < kBwdRows / 16; ++ks) {
        const uint64_t bd = tc::sdesc_sw128(st + 4u * 8192u + 2048u * ks, 8192u, 1024u);
        for (int m = 0; m < nmt; ++m) {
          const uint64_t ad = tc::sdesc_sw128(st + (uint32_t)(2 * m) * 8192u + 2048u * ks, 8192u, 1024u);
          tc::mma_bf16(tmem + (uint32_t)(m * 128), ad, bd, idesc, (it | ks) != 0 ? 1u : 0u);
        }
      }
      tc::mma_commit(&bars->empty[s]);
    }
    if (ok && nst > 0) tc::mma_commit(&bars->tfull[0]);
    tc::mma_commit(&bars->done);
    if (!mbar_wait(&bars->done, 0, kWaitNs)) raise_abort(bars, err);
  } else if (warp >= 2) {
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    bool have = nst > 0;
    if (have && (!mbar_wait(&bars->tfull[0], 0, kWaitNs) || aborted(bars))) {
      raise_abort(bars, err);
      have = false;
    }
    tc::fence_after_sync();
    for (int m = 0; m < nmt; ++m) {
      const int pr = p0 + 128 * m + 32 * q + lane;      // p index of this thread's TMEM lane
      float* out = part + ((size_t)blockIdx.x * p + pr) * NB;
      for (int c0 = 0; c0 < NB; c0 += 16) {
        float v[16];
        if (have) {
          tc::tmem_ld16(tmem + lane_off + (uint32_t)(m * 128 + c0), v);
        } else {
#pragma unroll
          for (int t = 0; t < 16; ++t) v[t] = 0.f;
        }
        if (pr < p && pr < p0 + pv)
#pragma unroll
          for (int t = 0; t < 16; t += 4)
            *reinterpret_cast<float4*>(out + c0 + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// grad_B[j][c] = sum over CTAs x of part[x][j][c] + part[x][j][Cp + c], in
// FP64 and a fixed order: a block of 32 x 8 threads takes 32 consecutive
// outputs (coalesced along c); thread row y sums the CTAs x = y, y + 8, ...
// and row 0 adds the 8 row sums in order.
constexpr int kRedX = 32, kRedY = 8;
__global__ void __launch_bounds__(kRedX * kRedY) k_xtg_reduce(const float* __restrict__ part, int nx, int p, int NB,
                                                              int C, int Cp, float* __restrict__ grad_B) {
  __shared__ double s[kRedY][kRedX];
  const int64_t i = (int64_t)blockIdx.x * kRedX + threadIdx.x;
  const bool in = i < (int64_t)p * C;
  const int j = in ? (int)(i / C) : 0, c = in ? (int)(i - (int64_t)j * C) : 0;
  double a = 0.0;
  if (in)
    for (int x = threadIdx.y; x < nx; x += kRedY) {
      const float* r = part + ((size_t)x * p + j) * NB;
      a += (double)r[c] + (double)r[Cp + c];
    }
  s[threadIdx.y][threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.y == 0 && in) {
    double t = s[0][threadIdx.x];
    for (int y = 1; y < kRedY; ++y) t += s[y][threadIdx.x];
    grad_B[i] = (float)t;
  }
}

// ----------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// bfloat16 row-major rows x cols (row pitch ld elements, ld * 2 a multiple of
// 16 bytes), boxes of 64 columns x box_rows rows, 128-byte swizzle, zero fill
// outside the matrix.
cudaError_t make_map(CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (((uintptr_t)ptr & 15) != 0 || (ld * 2) % 16 != 0) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)kBoxK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  std::memset(m, 0, sizeof(*m));
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

}  // namespace

// Shared memory of the forward kernel with ns X stages (Bcat^T resident).
size_t nll_xb_smem(int p, int Cp, int ns) {
  const int nkb = (p + kBoxK - 1) / kBoxK;
  return 1024 + (size_t)nkb * 2 * Cp * 128 + (size_t)ns * 16384 + sizeof(TcBars);
}

// X stages that fit beside the resident Bcat^T (0: the product does not fit).
int nll_xb_stages(int p, int Cp) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int ns = kFwdStages; ns >= 3; --ns)
    if (nll_xb_smem(p, Cp, ns) <= (size_t)optin) return ns;
  return 0;
}

bool nll_tc_fits(int p, int C) {
  const int Cp = std::max(32, (C + 15) / 16 * 16);
  return nll_xb_stages(p, Cp) >= 3;
}

cudaError_t nll_xb_tc(const void* X, int64_t n, int p, int64_t ldx, const void* BcatT, int C, int Cp, float* eta,
                      unsigned* err, cudaStream_t s) {
  const int NB = 2 * Cp;
  const int nkb = (p + kBoxK - 1) / kBoxK;
  CUtensorMap mx, mb;
  cudaError_t st = make_map(&mx, X, n, p, ldx, kFwdRows);
  if (st == cudaSuccess) st = make_map(&mb, BcatT, NB, p, ldx, NB);
  if (st != cudaSuccess) return st;
  const int ns = nll_xb_stages(p, Cp);
  if (ns < 3) return cudaErrorInvalidValue;
  const size_t smem = nll_xb_smem(p, Cp, ns);
  st = cudaFuncSetAttribute(k_xb_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (st != cudaSuccess) return st;
  const int64_t ntiles = (n + kFwdRows - 1) / kFwdRows;
  const int G = (int)std::min<int64_t>(sm_count(), ntiles);
  if (G < 1) return cudaErrorInvalidValue;
  k_xb_tc<<<G, kTcThreads, smem, s>>>(mx, mb, n, nkb, C, Cp, ns, eta, err);
  return cudaGetLastError();
}

size_t nll_xtg_part_floats(int64_t n, int p, int NB, int* nx) {
  const int gy = (p + kBwdP - 1) / kBwdP;
  const int sms = std::max(1, sm_count());
  int gx = std::max(1, sms / gy);
  const int64_t stages = (n + kBwdRows - 1) / kBwdRows;
  if (gx > stages) gx = (int)std::max<int64_t>(1, stages);
  *nx = gx;
  return (size_t)gx * p * NB;
}

cudaError_t nll_xtg_tc(const void* X, int64_t n, int p, int64_t ldx, const void* Gcat, int C, int Cp, float* part,
                       int nx, float* grad_B, unsigned* err, cudaStream_t s) {
  const int NB = 2 * Cp;
  CUtensorMap mx, mg;
  cudaError_t st = make_map(&mx, X, n, p, ldx, kBwdRows);
  if (st == cudaSuccess) st = make_map(&mg, Gcat, n, NB, NB, kBwdRows);
  if (st != cudaSuccess) return st;
  const size_t smem = 1024 + (size_t)kBwdStages * 6 * 8192 + sizeof(TcBars);
  st = cudaFuncSetAttribute(k_xtg_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (st != cudaSuccess) return st;
  const int gy = (p + kBwdP - 1) / kBwdP;
  const int64_t per = (n + nx - 1) / nx;
  const int64_t rows_per_cta = (per + kBwdRows - 1) / kBwdRows * kBwdRows;
  k_xtg_tc<<<dim3(nx, gy), kTcThreads, smem, s>>>(mx, mg, n, p, NB, rows_per_cta, part, err);
  st = cudaGetLastError();
  if (st != cudaSuccess) return st;
  const int64_t pc = (int64_t)p * C;
  k_xtg_reduce<<<(unsigned)((pc + kRedX - 1) / kRedX), dim3(kRedX, kRedY), 0, s>>>(part, nx, p, NB, C, Cp, grad_B);
  return cudaGetLastError();
}

}  // namespace survgpu
