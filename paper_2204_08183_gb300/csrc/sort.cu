// Stable order of decreasing time (Section 2.7 arranges the subjects by
// decreasing observed time; ties keep their input order).  Least-significant
// digit radix sort, 4 passes of 8 bits over the key ~(t ^ 0x80000000), which
// orders signed times descending; every pass is stable, so equal times keep
// the input order and the permutation is unique.
//
// Per pass: (1) per-tile digit counts, (2) one exclusive scan over the
// digit-major count table, (3) a stable scatter in which each element's rank
// among equal digits of its tile comes from warp match masks plus an
// exclusive scan of per-warp digit counts.
#include <cstdint>

#include "internal.h"

namespace survgpu {
namespace {

constexpr int kTile = 1024;      // elements per tile = threads per block
constexpr int kRadix = 256;

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

__global__ void k_keys(const int32_t* time, int64_t n, uint32_t* keys, int32_t* vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = ~((uint32_t)time[i] ^ 0x80000000u);
    vals[i] = (int32_t)i;
  }
}

__global__ void k_hist(const uint32_t* keys, int64_t n, int shift, int64_t ntiles, uint32_t* counts) {
  __shared__ uint32_t s[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) s[d] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kTile + threadIdx.x;
  if (i < n) atomicAdd(&s[(keys[i] >> shift) & 0xffu], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) counts[(int64_t)d * ntiles + blockIdx.x] = s[d];
}

// single block: exclusive scan of L counts in place
__global__ void k_scan(uint32_t* a, int64_t L) {
  __shared__ uint32_t s[1024];
  const int t = threadIdx.x;
  const int64_t per = (L + blockDim.x - 1) / blockDim.x;
  const int64_t lo = t * per, hi = lo + per < L ? lo + per : L;
  uint32_t sum = 0;
  for (int64_t q = lo; q < hi; ++q) sum += a[q];
  s[t] = sum;
  __syncthreads();
  if (t == 0) {
    uint32_t run = 0;
    for (int q = 0; q < (int)blockDim.x; ++q) {
      const uint32_t v = s[q];
      s[q] = run;
      run += v;
    }
  }
  __syncthreads();
  uint32_t run = s[t];
  for (int64_t q = lo; q < hi; ++q) {
    const uint32_t v = a[q];
    a[q] = run;
    run += v;
  }
}

__global__ void k_scatter(const uint32_t* kin, const int32_t* vin, int64_t n, int shift, int64_t ntiles,
                          const uint32_t* offsets, uint32_t* kout, int32_t* vout) {
  __shared__ uint32_t s_cnt[kTile / 32][kRadix];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < (kTile / 32) * kRadix; q += blockDim.x) (&s_cnt[0][0])[q] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const bool valid = i < n;
  const uint32_t k = valid ? kin[i] : 0u;
  const int32_t v = valid ? vin[i] : 0;
  const unsigned d = valid ? ((k >> shift) & 0xffu) : kRadix;  // sentinel for the tail
  const unsigned peers = __match_any_sync(0xffffffffu, d);
  const unsigned rank_w = __popc(peers & ((1u << lane) - 1u));
  if (valid && (peers & ((1u << lane) - 1u)) == 0u) s_cnt[w][d] = __popc(peers);
  __syncthreads();
  for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
    uint32_t run = 0;
    for (int q = 0; q < kTile / 32; ++q) {
      const uint32_t c = s_cnt[q][dd];
      s_cnt[q][dd] = run;
      run += c;
    }
  }
  __syncthreads();
  if (valid) {
    const uint32_t pos = offsets[(int64_t)d * ntiles + blockIdx.x] + s_cnt[w][d] + rank_w;
    kout[pos] = k;
    vout[pos] = v;
  }
}

}  // namespace

size_t radix_sort_workspace(int64_t n) {
  const int64_t ntiles = (n + kTile - 1) / kTile;
  return align256(4 * (size_t)n) * 3 + align256(4 * (size_t)kRadix * (size_t)ntiles);
}

cudaError_t radix_sort_desc(const int32_t* time, int64_t n, int32_t* perm, void* work, cudaStream_t s,
                            int* launches) {
  if (n <= 0) return cudaSuccess;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  char* wp = static_cast<char*>(work);
  uint32_t* kA = reinterpret_cast<uint32_t*>(wp);
  uint32_t* kB = reinterpret_cast<uint32_t*>(wp + align256(4 * (size_t)n));
  int32_t* vB = reinterpret_cast<int32_t*>(wp + 2 * align256(4 * (size_t)n));
  uint32_t* counts = reinterpret_cast<uint32_t*>(wp + 3 * align256(4 * (size_t)n));
  int32_t* vA = perm;  // four passes end in (kA, vA)
  const unsigned g = (unsigned)((n + 255) / 256 < 65535 * 16 ? (n + 255) / 256 : 65535 * 16);
  k_keys<<<g, 256, 0, s>>>(time, n, kA, vA);
  int nl = 1;
  uint32_t* kin = kA;
  int32_t* vin = vA;
  uint32_t* kout = kB;
  int32_t* vout = vB;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    k_hist<<<(unsigned)ntiles, kTile, 0, s>>>(kin, n, shift, ntiles, counts);
    k_scan<<<1, 1024, 0, s>>>(counts, (int64_t)kRadix * ntiles);
    k_scatter<<<(unsigned)ntiles, kTile, 0, s>>>(kin, vin, n, shift, ntiles, counts, kout, vout);
    nl += 3;
    uint32_t* tk = kin; kin = kout; kout = tk;
    int32_t* tv = vin; vin = vout; vout = tv;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

}  // namespace survgpu
