// Full-size residual of Eq. 2.2: ||X - W H||_F^2 and ||X||_F^2 in one read of X.
// W H is rebuilt per 64 x 128 tile from W rows and H columns staged in shared memory (K = r),
// differences and squares are formed in FP32 per tile and added to per-thread FP64 sums; block
// sums and the final sum are FP64 in a fixed order (deterministic).
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kTR = 64, kTC = 128, kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads) residual_kernel(
    const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx, const float* __restrict__ W,
    const float* __restrict__ H, int r, double* __restrict__ part) {
  extern __shared__ __align__(16) float sh[];
  float* WsT = sh;                 // [r][kTR]
  float* Hs = WsT + r * kTR;       // [r][kTC]
  __shared__ double red[2][kThreads / 32];
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int64_t tiles_r = cdiv(m, kTR), tiles_c = cdiv(n, kTC);
  double e2 = 0.0, x2 = 0.0;
  for (int64_t tile = blockIdx.x; tile < tiles_r * tiles_c; tile += gridDim.x) {
    const int64_t r0 = (tile / tiles_c) * kTR, c0 = (tile % tiles_c) * kTC;
    __syncthreads();
    for (int e = t; e < kTR * r; e += kThreads) {
      const int i = e / r, k = e - i * r;
      WsT[k * kTR + i] = (r0 + i < m) ? W[(r0 + i) * r + k] : 0.f;
    }
    for (int e = t; e < r * kTC; e += kThreads) {
      const int k = e / kTC, c = e - k * kTC;
      Hs[e] = (c0 + c < n) ? H[k * n + c0 + c] : 0.f;
    }
    __syncthreads();
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    for (int k = 0; k < r; ++k) {
      const float4 w = *reinterpret_cast<const float4*>(&WsT[k * kTR + 4 * ty]);
      const float4 h0 = *reinterpret_cast<const float4*>(&Hs[k * kTC + 4 * tx]);
      const float4 h1 = *reinterpret_cast<const float4*>(&Hs[k * kTC + 64 + 4 * tx]);
      const float wv[4] = {w.x, w.y, w.z, w.w};
      const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(wv[a], hv[b], acc[a][b]);
    }
    float te = 0.f, tx2 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t gr = r0 + 4 * ty + a;
      if (gr >= m) continue;
      const float* xr = X + gr * ldx;
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int64_t gc = c0 + 64 * g + 4 * tx;
        float xv[4];
        if (VEC && gc + 3 < n) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(xr + gc));
          xv[0] = v.x; xv[1] = v.y; xv[2] = v.z; xv[3] = v.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) xv[q] = (gc + q < n) ? xr[gc + q] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // out-of-range columns have xv = 0 and acc = 0 (H padded with zeros)
          const float d = xv[q] - acc[a][4 * g + q];
          te = fmaf(d, d, te);
          tx2 = fmaf(xv[q], xv[q], tx2);
        }
      }
    }
    e2 += te;
    x2 += tx2;
  }
  e2 = warp_sum(e2);
  x2 = warp_sum(x2);
  if ((t & 31) == 0) {
    red[0][t >> 5] = e2;
    red[1][t >> 5] = x2;
  }
  __syncthreads();
  if (t < 32) {
    double a = (t < kThreads / 32) ? red[0][t] : 0.0;
    double b = (t < kThreads / 32) ? red[1][t] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (t == 0) {
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = b;
    }
  }
}

__global__ void residual_final_kernel(const double* __restrict__ part, int nparts,
                                      double* __restrict__ out2) {
  const int t = threadIdx.x;  // one warp
  double a = 0.0, b = 0.0;
  for (int i = t; i < nparts; i += 32) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (t == 0) {
    out2[0] = a;
    out2[1] = b;
  }
}

int residual_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (sms > 0 ? sms : 148) * 4;
}

}  // namespace

size_t residual_ws_bytes(int64_t, int64_t) {
  return sizeof(double) * 2 * static_cast<size_t>(residual_grid()) + 256;
}

cudaError_t launch_residual(const Launcher& L, const float* X, int64_t m, int64_t n, int64_t ldx,
                            const float* W, const float* H, int r, double* out2, void* ws,
                            size_t ws_bytes) {
  if (ws_bytes < residual_ws_bytes(m, n)) return cudaErrorInvalidValue;
  const int64_t tiles = cdiv(m, kTR) * cdiv(n, kTC);
  int grid = residual_grid();
  if (tiles < grid) grid = static_cast<int>(tiles);
  double* part = static_cast<double*>(ws);
  const size_t sm = sizeof(float) * (r * kTR + r * kTC);
  const bool vec = (ldx % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  cudaError_t err;
  if (vec) {
    if ((err = cudaFuncSetAttribute(residual_kernel<true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(sm))) != cudaSuccess)
      return err;
    residual_kernel<true><<<grid, kThreads, sm, L.stream>>>(X, m, n, ldx, W, H, r, part);
  } else {
    if ((err = cudaFuncSetAttribute(residual_kernel<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(sm))) != cudaSuccess)
      return err;
    residual_kernel<false><<<grid, kThreads, sm, L.stream>>>(X, m, n, ldx, W, H, r, part);
  }
  residual_final_kernel<<<1, 32, 0, L.stream>>>(part, grid, out2);
  L.count(2);
  return cudaGetLastError();
}

}  // namespace nmfrp
