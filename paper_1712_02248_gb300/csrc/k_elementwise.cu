// Gaussian test matrix (Section 3: Omega ~ N(0,1)) and the FP32 -> BF16 copy of X.
#include <cuda_fp8.h>

#include "common.cuh"

namespace nmfrp {
namespace {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32->64-bit multiplies
// with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ float to_unit(uint32_t x) {
  // ((x >> 8) + 1/2) * 2^-24, strictly inside (0, 1)
  return (static_cast<float>(x >> 8) + 0.5f) * 5.9604644775390625e-8f;
}

__global__ void gaussian_kernel(int64_t total, uint2 key, uint32_t stream_id, float* out) {
  const int64_t nblk = (total + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
       b += (int64_t)gridDim.x * blockDim.x) {
    const uint4 x = philox4x32_10(
        make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(b >> 32), stream_id, 0u), key);
    float z[4];
    {
      const float rad = sqrtf(-2.0f * logf(to_unit(x.x)));
      float s, c;
      sincospif(2.0f * to_unit(x.y), &s, &c);
      z[0] = rad * c;
      z[1] = rad * s;
    }
    {
      const float rad = sqrtf(-2.0f * logf(to_unit(x.z)));
      float s, c;
      sincospif(2.0f * to_unit(x.w), &s, &c);
      z[2] = rad * c;
      z[3] = rad * s;
    }
    const int64_t e0 = 4 * b;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (e0 + t < total) out[e0 + t] = z[t];
  }
}

// Y[i][j] = N(0, 1) for every column j whose bit is set in mask[j / 32] (rows x ell, row-major):
// the Philox4x32-10 / Box-Muller draws of the Gaussian kernel, counter (element / 4, stream_id).
__global__ void replace_columns_kernel(float* __restrict__ Y, int64_t rows, int ell, uint4 mask,
                                       uint2 key, uint32_t stream_id) {
  const uint32_t mw[4] = {mask.x, mask.y, mask.z, mask.w};
  const int64_t total = rows * ell, nblk = (total + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
       b += (int64_t)gridDim.x * blockDim.x) {
    const uint4 x = philox4x32_10(
        make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(b >> 32), stream_id, 0u), key);
    const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 4; t += 2) {
      const float rad = sqrtf(-2.0f * logf(to_unit(u[t])));
      float sn, cs;
      sincospif(2.0f * to_unit(u[t + 1]), &sn, &cs);
      const float z[2] = {rad * cs, rad * sn};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int64_t e = 4 * b + t + q;
        if (e >= total) continue;
        const int j = static_cast<int>(e % ell);
        if ((mw[j >> 5] >> (j & 31)) & 1u) Y[e] = z[q];
      }
    }
  }
}

__global__ void quantize_bf16_kernel(const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                                     __nv_bfloat16* __restrict__ Xq, int64_t ldq) {
  const int64_t total = m * ldq;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ldq, j = e - i * ldq;
    Xq[e] = __float2bfloat16_rn(j < n ? X[i * ldx + j] : 0.f);
  }
}

// Vectorised variant: n % 4 == 0, ldx % 4 == 0, X 16-byte aligned, ldq == n.
__global__ void quantize_bf16_vec4_kernel(const float* __restrict__ X, int64_t m, int64_t n,
                                          int64_t ldx, __nv_bfloat16* __restrict__ Xq) {
  const int64_t n4 = n / 4, total = m * n4;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n4, j4 = e - i * n4;
    const float4 v = __ldcs(reinterpret_cast<const float4*>(X + i * ldx) + j4);
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 packed;
    packed.x = *reinterpret_cast<uint32_t*>(&lo);
    packed.y = *reinterpret_cast<uint32_t*>(&hi);
    reinterpret_cast<uint2*>(Xq + i * n)[j4] = packed;
  }
}

// BF16 copy plus the two sums the compressed error monitor needs: ||X||^2 and <X - X_q, X>
// (the rounding of X to BF16 enters the monitor's cross term; this sum removes it). FP32 within
// runs of 64 elements a thread, float-float (FSum) beyond, FP64 only for the block partials,
// summed in a fixed order.
template <bool VEC>
__global__ void __launch_bounds__(256) quantize_bf16_stats_kernel(
    const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx, __nv_bfloat16* __restrict__ Xq,
    int64_t ldq, double* __restrict__ part) {
  __shared__ double red[2][8];
  FSum sx2, scorr;
  float fx2 = 0.f, fcorr = 0.f;
  int run = 0;
  if (VEC) {
    // grid-stride over the float4s of the m x n/4 array; the (row, float4) position advances by
    // a fixed (di, dj) each step (one division a thread), two loads in flight a step
    const int64_t n4 = n / 4;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t di = stride / n4, dj = stride - di * n4;
    const int64_t e0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    int64_t i = e0 / n4, j4 = e0 - i * n4;
    auto advance = [&](int64_t& ii, int64_t& jj) {
      ii += di;
      jj += dj;
      if (jj >= n4) {
        jj -= n4;
        ++ii;
      }
    };
    auto consume = [&](const float4 v, int64_t ii, int64_t jj) {
      __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
      __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
      uint2 packed;
      packed.x = *reinterpret_cast<uint32_t*>(&lo);
      packed.y = *reinterpret_cast<uint32_t*>(&hi);
      reinterpret_cast<uint2*>(Xq + ii * ldq)[jj] = packed;
      const float2 ql = __bfloat1622float2(lo), qh = __bfloat1622float2(hi);
      fx2 = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, fx2))));
      fcorr = fmaf(v.x, v.x - ql.x, fmaf(v.y, v.y - ql.y,
                   fmaf(v.z, v.z - qh.x, fmaf(v.w, v.w - qh.y, fcorr))));
      if (++run == 16) {
        sx2.add(fx2);
        scorr.add(fcorr);
        fx2 = fcorr = 0.f;
        run = 0;
      }
    };
    while (i < m) {
      int64_t i2 = i, j2 = j4;
      advance(i2, j2);
      const float4 v = __ldcs(reinterpret_cast<const float4*>(X + i * ldx) + j4);
      const bool two = i2 < m;
      const float4 w = two ? __ldcs(reinterpret_cast<const float4*>(X + i2 * ldx) + j2)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      consume(v, i, j4);
      if (two) consume(w, i2, j2);
      i = i2;
      j4 = j2;
      advance(i, j4);
    }
  } else {
    const int64_t total = m * ldq;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = e / ldq, j = e - i * ldq;
      const float x = j < n ? X[i * ldx + j] : 0.f;
      const __nv_bfloat16 q = __float2bfloat16_rn(x);
      Xq[e] = q;
      fx2 = fmaf(x, x, fx2);
      fcorr = fmaf(x, x - __bfloat162float(q), fcorr);
      if (++run == 64) {
        sx2.add(fx2);
        scorr.add(fcorr);
        fx2 = fcorr = 0.f;
        run = 0;
      }
    }
  }
  sx2.add(fx2);
  scorr.add(fcorr);
  double x2 = sx2.value(), corr = scorr.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    corr += __shfl_xor_sync(0xffffffffu, corr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = x2;
    red[1][threadIdx.x >> 5] = corr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// FP8 copy of X: OCP E4M3 codes at Xq[i * ldq + j] (ldq = n rounded up to 16, pad columns zero)
// and one E8M0 scale byte k + 127 a 32 x 32 tile at S[(i / 32) * tn + j / 32], where 2^k is the
// smallest power of two with amax / 2^k <= 448 over the tile (amax = f 2^e, f in [0.5, 1):
// k = e - 9 if f <= 0.875 else e - 8; k = 0 for an all-zero tile; clamped to [-127, 127]).
// Codes are round-to-nearest-even of x / 2^k, saturating. One warp a tile (lane = column, the
// tile's 32 loads in flight), plus the monitor sums ||X||^2 and <X - X_q, X> in float-float.
__global__ void __launch_bounds__(256) quantize_fp8_stats_kernel(
    const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx, uint8_t* __restrict__ Xq,
    int64_t ldq, uint8_t* __restrict__ S, double* __restrict__ part) {
  __shared__ double red[2][8];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t tn = (n + 31) / 32, tiles = ((m + 31) / 32) * tn;
  FSum sx2, scorr;
  for (int64_t tile = static_cast<int64_t>(blockIdx.x) * 8 + wib; tile < tiles;
       tile += static_cast<int64_t>(gridDim.x) * 8) {
    const int64_t ti = tile / tn, tj = tile - ti * tn;
    const int64_t r0 = ti * 32, c = tj * 32 + lane;
    const int nr = m - r0 < 32 ? static_cast<int>(m - r0) : 32;
    const bool colv = c < n;
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = (i < nr && colv) ? __ldcs(X + (r0 + i) * ldx + c) : 0.f;
    float amax = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) amax = fmaxf(amax, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(full, amax, o));
    int k = 0;
    if (amax > 0.f) {
      int e;
      const float f = frexpf(amax, &e);
      k = f <= 0.875f ? e - 9 : e - 8;
      k = k < -127 ? -127 : (k > 127 ? 127 : k);
    }
    const float sinv = ldexpf(1.f, -k), sc = ldexpf(1.f, k);
    float tx2 = 0.f, tcorr = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(__fmul_rn(x[i], sinv), __NV_SATFINITE,
                                                         __NV_E4M3);
      const float xq = __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))) * sc;
      if (i < nr && c < ldq) Xq[(r0 + i) * ldq + c] = colv ? static_cast<uint8_t>(q) : uint8_t(0);
      tx2 = fmaf(x[i], x[i], tx2);
      tcorr = fmaf(x[i], x[i] - xq, tcorr);
    }
    sx2.add(tx2);
    scorr.add(tcorr);
    if (lane == 0) S[tile] = static_cast<uint8_t>(k + 127);
  }
  double x2 = sx2.value(), corr = scorr.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x2 += __shfl_xor_sync(full, x2, o);
    corr += __shfl_xor_sync(full, corr, o);
  }
  if (lane == 0) {
    red[0][wib] = x2;
    red[1][wib] = corr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void stats_final_kernel(const double* __restrict__ part, int nparts,
                                   double* __restrict__ x2_out, double* __restrict__ corr_out) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (threadIdx.x == 0) {   // either destination may be null (that sum is not wanted)
    if (x2_out) *x2_out = a;
    if (corr_out) *corr_out = b;
  }
}

int grid_for(int64_t work, int threads) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 148;
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  return static_cast<int>(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_gaussian(const Launcher& L, int64_t rows, int64_t cols, uint64_t seed,
                            uint32_t stream_id, float* out) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  gaussian_kernel<<<grid_for((total + 3) / 4, 256), 256, 0, L.stream>>>(total, key, stream_id, out);
  L.count();
  return cudaGetLastError();
}

cudaError_t launch_replace_columns(const Launcher& L, float* Y, int64_t rows, int ell,
                                   const uint32_t* mask, uint64_t seed, uint32_t stream_id) {
  if (rows <= 0 || ell <= 0 || ell > 128) return cudaErrorInvalidValue;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  replace_columns_kernel<<<grid_for((rows * ell + 3) / 4, 256), 256, 0, L.stream>>>(
      Y, rows, ell, make_uint4(mask[0], mask[1], mask[2], mask[3]), key, stream_id);
  L.count();
  return cudaGetLastError();
}

cudaError_t launch_quantize_bf16(const Launcher& L, const float* X, int64_t m, int64_t n,
                                 int64_t ldx, __nv_bfloat16* Xq, int64_t ldq) {
  if (m * n <= 0) return cudaSuccess;
  const bool vec = (n % 4 == 0) && (ldx % 4 == 0) && (ldq == n) &&
                   (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  if (vec)
    quantize_bf16_vec4_kernel<<<grid_for(m * n / 4, 256), 256, 0, L.stream>>>(X, m, n, ldx, Xq);
  else
    quantize_bf16_kernel<<<grid_for(m * ldq, 256), 256, 0, L.stream>>>(X, m, n, ldx, Xq, ldq);
  L.count();
  return cudaGetLastError();
}

size_t fp8_copy_bytes(int64_t m, int64_t n, int64_t* ldq, int64_t* scale_off) {
  const int64_t q = (n + 15) / 16 * 16;
  const int64_t off = (m * q + 255) / 256 * 256;
  if (ldq) *ldq = q;
  if (scale_off) *scale_off = off;
  return static_cast<size_t>(off + ((m + 31) / 32) * ((n + 31) / 32));
}

cudaError_t launch_quantize_fp8_stats(const Launcher& L, const float* X, int64_t m, int64_t n,
                                      int64_t ldx, uint8_t* Xq, double* x2_out, double* corr_out,
                                      void* ws, size_t ws_bytes) {
  if (m <= 0 || n <= 0 || ldx < n) return cudaErrorInvalidValue;
  if (ws_bytes < quantize_stats_ws_bytes() + 64) return cudaErrorInvalidValue;
  int64_t ldq = 0, off = 0;
  fp8_copy_bytes(m, n, &ldq, &off);
  double* part = static_cast<double*>(ws);
  const int64_t tiles = ((m + 31) / 32) * ((n + 31) / 32);
  const int grid = grid_for((tiles + 7) / 8, 1);
  quantize_fp8_stats_kernel<<<grid, 256, 0, L.stream>>>(X, m, n, ldx, Xq, ldq, Xq + off, part);
  // without destinations the sums land in the scratch just past the partials
  double* sink = part + 2 * grid;
  stats_final_kernel<<<1, 32, 0, L.stream>>>(part, grid, x2_out ? x2_out : sink,
                                             corr_out ? corr_out : sink + 1);
  L.count(2);
  return cudaGetLastError();
}

size_t quantize_stats_ws_bytes() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 148;
  return sizeof(double) * 2 * static_cast<size_t>(sms) * 8 + 256;
}

cudaError_t launch_quantize_bf16_stats(const Launcher& L, const float* X, int64_t m, int64_t n,
                                       int64_t ldx, __nv_bfloat16* Xq, int64_t ldq, double* x2_out,
                                       double* corr_out, void* ws, size_t ws_bytes) {
  if (m * n <= 0) return cudaErrorInvalidValue;
  if (ws_bytes < quantize_stats_ws_bytes()) return cudaErrorInvalidValue;
  const bool vec = (n % 4 == 0) && (ldx % 4 == 0) && (ldq % 4 == 0) &&
                   (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  double* part = static_cast<double*>(ws);
  int grid;
  if (vec) {
    grid = grid_for(m * n / 4, 256);
    if (ldq != n) {
      // zero the pad columns first (the vector kernel writes columns [0, n) only)
      cudaError_t e = cudaMemsetAsync(Xq, 0, sizeof(__nv_bfloat16) * m * ldq, L.stream);
      if (e != cudaSuccess) return e;
    }
    quantize_bf16_stats_kernel<true><<<grid, 256, 0, L.stream>>>(X, m, n, ldx, Xq, ldq, part);
  } else {
    grid = grid_for(m * ldq, 256);
    quantize_bf16_stats_kernel<false><<<grid, 256, 0, L.stream>>>(X, m, n, ldx, Xq, ldq, part);
  }
  stats_final_kernel<<<1, 32, 0, L.stream>>>(part, grid, x2_out, corr_out);
  L.count(2);
  return cudaGetLastError();
}

}  // namespace nmfrp
