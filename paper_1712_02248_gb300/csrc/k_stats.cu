// Diagnostics of a computed factor: the Gini coefficient of its entries (Section 5.1, the
// sparsity measure of B in Figures 5.4 and 5.7):
//   G = sum_{i=1..N} (2 i - N - 1) b_(i) / (N sum_i b_(i)),   b_(1) <= ... <= b_(N)  (ascending).
//
// The entries are sorted on the device: each float is mapped to an unsigned key with the same
// order (sign bit flipped for non-negative values, all bits for negative ones), the keys are
// padded with the largest key to a power of two N2 >= 2048 and sorted by a bitonic network
// (stages with a partner distance below 2048 inside shared memory, the rest one launch a stage
// over global memory). The weighted sum and the plain sum are then taken in FP64, a per-block
// partial each, summed in a fixed order by one block. Ties need no care: equal values may take
// their positions in any order without changing the weighted sum.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kLocal = 2048;        // keys a block sorts in shared memory
constexpr int kLocalThreads = 1024;
constexpr int kSumThreads = 256;
constexpr int kSumBlocks = 512;

__device__ __forceinline__ uint32_t float_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void keys_kernel(const float* __restrict__ B, int64_t count, int64_t n2,
                            uint32_t* __restrict__ keys) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n2;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    keys[i] = i < count ? float_key(B[i]) : 0xFFFFFFFFu;
}

// Pair t of a stage with partner distance j: i = the t-th index with bit j clear, partner i + j.
__device__ __forceinline__ int64_t pair_index(int64_t t, int64_t j) { return 2 * t - (t & (j - 1)); }

// INIT: the full network for sizes 2 .. 2048 on this block's keys. Else the stages j = 1024 .. 1
// of merge size k. The direction of a pair is ascending when bit k of its global index is clear.
template <bool INIT>
__global__ void __launch_bounds__(kLocalThreads) bitonic_local_kernel(uint32_t* __restrict__ keys,
                                                                      int64_t kmerge) {
  __shared__ uint32_t s[kLocal];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kLocal;
  const int t = threadIdx.x;
  s[t] = keys[base + t];
  s[t + kLocalThreads] = keys[base + t + kLocalThreads];
  __syncthreads();
  auto step = [&](int64_t k, int j) {
    const int i = static_cast<int>(pair_index(t, j));
    const bool up = ((base + i) & k) == 0;
    const uint32_t a = s[i], b = s[i + j];
    if ((a > b) == up) {
      s[i] = b;
      s[i + j] = a;
    }
    __syncthreads();
  };
  if (INIT) {
    for (int k = 2; k <= kLocal; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) step(k, j);
  } else {
    for (int j = kLocal / 2; j > 0; j >>= 1) step(kmerge, j);
  }
  keys[base + t] = s[t];
  keys[base + t + kLocalThreads] = s[t + kLocalThreads];
}

// One stage (merge size k, partner distance j >= 2048) over global memory.
__global__ void bitonic_global_kernel(uint32_t* __restrict__ keys, int64_t npairs, int64_t k,
                                      int64_t j) {
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < npairs;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = pair_index(t, j);
    const bool up = (i & k) == 0;
    const uint32_t a = keys[i], b = keys[i + j];
    if ((a > b) == up) {
      keys[i] = b;
      keys[i + j] = a;
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per block: sum (2 i - N - 1) b_(i) (i from 1) and sum b_(i) over its stride of sorted keys.
__global__ void __launch_bounds__(kSumThreads) gini_partial_kernel(const uint32_t* __restrict__ keys,
                                                                   int64_t count,
                                                                   double* __restrict__ part) {
  double num = 0.0, tot = 0.0;
  const double nn = static_cast<double>(count) + 1.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double b = key_float(keys[i]);
    num = fma(2.0 * static_cast<double>(i + 1) - nn, b, num);
    tot += b;
  }
  __shared__ double sn[kSumThreads / 32], st[kSumThreads / 32];
  num = warp_sum(num);
  tot = warp_sum(tot);
  if ((threadIdx.x & 31) == 0) {
    sn[threadIdx.x >> 5] = num;
    st[threadIdx.x >> 5] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kSumThreads / 32; ++w) {
      a += sn[w];
      c += st[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = c;
  }
}

// out[0] = weighted sum, out[1] = plain sum: the block partials in block order.
__global__ void gini_final_kernel(const double* __restrict__ part, int nblocks,
                                  double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      a += part[2 * b];
      c += part[2 * b + 1];
    }
    out[0] = a;
    out[1] = c;
  }
}

int64_t padded_count(int64_t count) {
  int64_t n2 = kLocal;
  while (n2 < count) n2 <<= 1;
  return n2;
}

}  // namespace

size_t gini_ws_bytes(int64_t count) {
  return sizeof(uint32_t) * static_cast<size_t>(padded_count(count)) +
         sizeof(double) * 2 * kSumBlocks + 512;
}

cudaError_t launch_gini(const Launcher& L, const float* B, int64_t count, void* ws,
                        size_t ws_bytes, double* out2) {
  if (count < 1 || !B || !out2) return cudaErrorInvalidValue;
  if (ws_bytes < gini_ws_bytes(count)) return cudaErrorInvalidValue;
  const int64_t n2 = padded_count(count);
  uint32_t* keys = static_cast<uint32_t*>(ws);
  uintptr_t q = reinterpret_cast<uintptr_t>(keys + n2);
  q = (q + 255) & ~uintptr_t(255);
  double* part = reinterpret_cast<double*>(q);
  const unsigned gb = static_cast<unsigned>(cdiv(n2, 256) < 8192 ? cdiv(n2, 256) : 8192);
  keys_kernel<<<gb, 256, 0, L.stream>>>(B, count, n2, keys);
  const unsigned nloc = static_cast<unsigned>(n2 / kLocal);
  bitonic_local_kernel<true><<<nloc, kLocalThreads, 0, L.stream>>>(keys, 0);
  int launches = 2;
  for (int64_t k = 2 * kLocal; k <= n2; k <<= 1) {
    for (int64_t j = k >> 1; j >= kLocal; j >>= 1) {
      const int64_t npairs = n2 / 2;
      const unsigned g = static_cast<unsigned>(cdiv(npairs, 256) < 16384 ? cdiv(npairs, 256) : 16384);
      bitonic_global_kernel<<<g, 256, 0, L.stream>>>(keys, npairs, k, j);
      ++launches;
    }
    bitonic_local_kernel<false><<<nloc, kLocalThreads, 0, L.stream>>>(keys, k);
    ++launches;
  }
  const unsigned sb = static_cast<unsigned>(cdiv(count, kSumThreads) < kSumBlocks
                                                ? cdiv(count, kSumThreads)
                                                : kSumBlocks);
  gini_partial_kernel<<<sb, kSumThreads, 0, L.stream>>>(keys, count, part);
  gini_final_kernel<<<1, 32, 0, L.stream>>>(part, static_cast<int>(sb), out2);
  L.count(launches + 2);
  return cudaGetLastError();
}

}  // namespace nmfrp
