// Fused dual pass over X on the FP32 SIMT pipes: Y = X V (m x l) and Z = X^T U (n x l) from one
// read of X. Every sketch pass (Section 3, Eq. 3.5: one application of X for the left chain and
// one of X^T for the right chain) and the compression (Section 4: X_chk = X Q_R, X_hat = Q_L^T X)
// is one such pass.
//
// Work split: a CTA owns a rectangle of RH = 32*RC rows x CW = 128*CC columns. It walks the
// rectangle in 32 x 128 chunks staged in shared memory. Z for the current 128 columns is carried
// in registers across the CTA's rows; Y for the CTA's rows is carried in shared memory across its
// columns. Partial sums go to per-rectangle slots and a second kernel adds them in a fixed order
// (deterministic results, no atomics).
#include <cuda_fp8.h>

#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kThreads = 256;
constexpr int kChunkRows = 32;
constexpr int kChunkCols = 128;
constexpr int kXsStride = kChunkCols + 4;

// X element (gr, gc): FP32, BF16, or an FP8 copy (E4M3 code times the E8M0 scale 2^(S - 127) of
// its 32 x 32 tile, S row-major over tiles with tn tiles a row)
__device__ __forceinline__ float load_x(const float* X, int64_t gr, int64_t gc, int64_t ldx,
                                        const uint8_t*, int64_t) {
  return __ldcs(X + gr * ldx + gc);
}
__device__ __forceinline__ float load_x(const __nv_bfloat16* X, int64_t gr, int64_t gc,
                                        int64_t ldx, const uint8_t*, int64_t) {
  return __bfloat162float(X[gr * ldx + gc]);
}
__device__ __forceinline__ float load_x(const uint8_t* X, int64_t gr, int64_t gc, int64_t ldx,
                                        const uint8_t* S, int64_t tn) {
  const __nv_fp8_storage_t q = X[gr * ldx + gc];
  const int k = static_cast<int>(S[(gr >> 5) * tn + (gc >> 5)]) - 127;
  return ldexpf(__half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))), k);
}

template <int LP, typename XT>
__global__ void __launch_bounds__(kThreads) dual_pass_simt_kernel(
    const XT* __restrict__ X, int64_t m, int64_t n, int64_t ldx, int ell,
    const float* __restrict__ V, const float* __restrict__ U, float* __restrict__ Ypart,
    float* __restrict__ Zpart, int RC, int CC, const uint8_t* __restrict__ S, int64_t tn) {
  constexpr int KZ = LP / 4;   // Z accumulators per column per thread
  constexpr int KY = LP / 8;   // Y outputs per thread per chunk
  extern __shared__ __align__(16) float smem[];
  float* Xs = smem;                                  // [32][kXsStride]
  float* Us = Xs + kChunkRows * kXsStride;           // [32][LP]
  float* Vs = Us + kChunkRows * LP;                  // [128][LP]
  float* Ys = Vs + kChunkCols * LP;                  // [RH][LP]

  const int t = threadIdx.x;
  const int RH = kChunkRows * RC;
  const int CW = kChunkCols * CC;
  const int64_t row0 = static_cast<int64_t>(blockIdx.y) * RH;
  const int64_t col0 = static_cast<int64_t>(blockIdx.x) * CW;
  const bool doY = (V != nullptr), doZ = (U != nullptr);

  for (int e = t; e < RH * LP; e += kThreads) Ys[e] = 0.f;

  // Z mapping: column pair cp (2 columns), k-group kg (KZ values of k)
  const int cp = t & 63, kg = t >> 6;
  // Y mapping: row yi in the chunk, k = yk + 8 j
  const int yi = t >> 3, yk = t & 7;

  for (int cc = 0; cc < CC; ++cc) {
    const int64_t cbase = col0 + static_cast<int64_t>(cc) * kChunkCols;
    if (cbase >= n) break;
    __syncthreads();
    for (int e = t; e < kChunkCols * LP; e += kThreads) {
      const int c = e / LP, k = e - c * LP;
      Vs[e] = (doY && cbase + c < n && k < ell) ? V[(cbase + c) * ell + k] : 0.f;
    }
    float acc[2][KZ];
#pragma unroll
    for (int q = 0; q < KZ; ++q) acc[0][q] = acc[1][q] = 0.f;

    for (int rc = 0; rc < RC; ++rc) {
      const int64_t rbase = row0 + static_cast<int64_t>(rc) * kChunkRows;
      if (rbase >= m) break;
      __syncthreads();
      for (int e = t; e < kChunkRows * kChunkCols; e += kThreads) {
        const int i = e >> 7, c = e & 127;
        const int64_t gr = rbase + i, gc = cbase + c;
        Xs[i * kXsStride + c] = (gr < m && gc < n) ? load_x(X, gr, gc, ldx, S, tn) : 0.f;
      }
      for (int e = t; e < kChunkRows * LP; e += kThreads) {
        const int i = e / LP, k = e - i * LP;
        const int64_t gr = rbase + i;
        Us[e] = (doZ && gr < m && k < ell) ? U[gr * ell + k] : 0.f;
      }
      __syncthreads();
      if (doZ) {
#pragma unroll 4
        for (int i = 0; i < kChunkRows; ++i) {
          const float2 x = *reinterpret_cast<const float2*>(&Xs[i * kXsStride + 2 * cp]);
          const float* u = &Us[i * LP + kg * KZ];
#pragma unroll
          for (int q = 0; q < KZ; ++q) {
            acc[0][q] = fmaf(x.x, u[q], acc[0][q]);
            acc[1][q] = fmaf(x.y, u[q], acc[1][q]);
          }
        }
      }
      if (doY) {
        float s[KY];
#pragma unroll
        for (int j = 0; j < KY; ++j) s[j] = 0.f;
        const float* xr = &Xs[yi * kXsStride];
#pragma unroll 4
        for (int c = 0; c < kChunkCols; ++c) {
          const float xv = xr[c];
#pragma unroll
          for (int j = 0; j < KY; ++j) s[j] = fmaf(xv, Vs[c * LP + yk + 8 * j], s[j]);
        }
        float* yrow = &Ys[(rc * kChunkRows + yi) * LP];
#pragma unroll
        for (int j = 0; j < KY; ++j) yrow[yk + 8 * j] += s[j];
      }
    }
    if (doZ) {
#pragma unroll
      for (int q = 0; q < KZ; ++q) {
        const int k = kg * KZ + q;
        if (k < ell) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int64_t gc = cbase + 2 * cp + h;
            if (gc < n) Zpart[(static_cast<int64_t>(blockIdx.y) * n + gc) * ell + k] = acc[h][q];
          }
        }
      }
    }
  }
  __syncthreads();
  if (doY) {
    for (int e = t; e < RH * LP; e += kThreads) {
      const int i = e / LP, k = e - i * LP;
      const int64_t gr = row0 + i;
      if (gr < m && k < ell) Ypart[(static_cast<int64_t>(blockIdx.x) * m + gr) * ell + k] = Ys[e];
    }
  }
}

// out[e] = sum_{s < slots} part[s * total + e], fixed order.
__global__ void reduce_slots_kernel(const float* __restrict__ part, int slots, int64_t total,
                                    float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < slots; ++k) s += part[k * total + e];
    out[e] = s;
  }
}

struct Split {
  int RC, CC;
  int64_t na, nb;
};

Split choose_split(int64_t m, int64_t n, int LP) {
  Split s;
  s.RC = LP > 64 ? 4 : 8;
  // wider column blocks when n is large relative to m keeps the Y partials small
  s.CC = 4;
  s.na = cdiv(m, kChunkRows * s.RC);
  s.nb = cdiv(n, kChunkCols * s.CC);
  return s;
}

int lp_for(int ell) {
  if (ell <= 16) return 16;
  if (ell <= 32) return 32;
  if (ell <= 48) return 48;
  if (ell <= 64) return 64;
  if (ell <= 96) return 96;
  return 128;
}

size_t smem_bytes(int LP, int RC) {
  return sizeof(float) * (kChunkRows * kXsStride + kChunkRows * LP + kChunkCols * LP +
                          kChunkRows * RC * LP);
}

template <int LP, typename XT>
cudaError_t run(const Launcher& L, const XT* X, int64_t m, int64_t n, int64_t ldx, int ell,
                const float* V, const float* U, float* Y, float* Z, float* ws,
                const uint8_t* S, int64_t tn) {
  const Split s = choose_split(m, n, LP);
  float* Ypart = ws;
  float* Zpart = ws + s.nb * m * ell;
  const size_t sm = smem_bytes(LP, s.RC);
  cudaError_t err = cudaFuncSetAttribute(dual_pass_simt_kernel<LP, XT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
  if (err != cudaSuccess) return err;
  dim3 grid(static_cast<unsigned>(s.nb), static_cast<unsigned>(s.na));
  dual_pass_simt_kernel<LP, XT><<<grid, kThreads, sm, L.stream>>>(
      X, m, n, ldx, ell, V, U, V ? Ypart : nullptr, U ? Zpart : nullptr, s.RC, s.CC, S, tn);
  L.count();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (V) {
    const int64_t tot = m * ell;
    reduce_slots_kernel<<<static_cast<unsigned>(cdiv(tot, 256) < 4096 ? cdiv(tot, 256) : 4096), 256,
                          0, L.stream>>>(Ypart, static_cast<int>(s.nb), tot, Y);
    L.count();
  }
  if (U) {
    const int64_t tot = n * ell;
    reduce_slots_kernel<<<static_cast<unsigned>(cdiv(tot, 256) < 4096 ? cdiv(tot, 256) : 4096), 256,
                          0, L.stream>>>(Zpart, static_cast<int>(s.na), tot, Z);
    L.count();
  }
  return cudaGetLastError();
}

template <typename XT>
cudaError_t dispatch(const Launcher& L, const XT* X, int64_t m, int64_t n, int64_t ldx, int ell,
                     const float* V, const float* U, float* Y, float* Z, float* ws,
                     const uint8_t* S = nullptr, int64_t tn = 0) {
  switch (lp_for(ell)) {
    case 16: return run<16>(L, X, m, n, ldx, ell, V, U, Y, Z, ws, S, tn);
    case 32: return run<32>(L, X, m, n, ldx, ell, V, U, Y, Z, ws, S, tn);
    case 48: return run<48>(L, X, m, n, ldx, ell, V, U, Y, Z, ws, S, tn);
    case 64: return run<64>(L, X, m, n, ldx, ell, V, U, Y, Z, ws, S, tn);
    case 96: return run<96>(L, X, m, n, ldx, ell, V, U, Y, Z, ws, S, tn);
    default: return run<128>(L, X, m, n, ldx, ell, V, U, Y, Z, ws, S, tn);
  }
}

}  // namespace

size_t dual_pass_ws_bytes(int64_t m, int64_t n, int ell) {
  const Split s = choose_split(m, n, lp_for(ell));
  const size_t simt = sizeof(float) * static_cast<size_t>(s.nb * m * ell + s.na * n * ell);
  const size_t tc = dual_pass_tc_ws_bytes(m, n, ell);
  return simt > tc ? simt : tc;
}

bool dual_pass_uses_tc(const void* X, int x_type, int64_t m, int64_t n, int64_t ldx, int ell,
                       bool both, bool force_simt) {
  if (!both || force_simt) return false;
  if (x_type == kXFp8) return dual_pass_tc_fp8_supported(m, n, ell, X);
  if (x_type == kXFp32) return dual_pass_tc_f32_supported(m, n, ldx, ell, X);
  return x_type == kXBf16 && dual_pass_tc_supported(m, n, ldx, ell, X);
}

cudaError_t launch_dual_pass(const Launcher& L, const void* X, int x_type, int64_t m, int64_t n,
                             int64_t ldx, int ell, const float* V, const float* U, float* Y,
                             float* Z, void* ws, size_t ws_bytes, int* status, bool force_simt,
                             bool split, bool z_kmajor) {
  if (ws_bytes < dual_pass_ws_bytes(m, n, ell)) return cudaErrorInvalidValue;
  const bool tc = dual_pass_uses_tc(X, x_type, m, n, ldx, ell, V && U, force_simt);
  if (z_kmajor && !tc) return cudaErrorInvalidValue;
  if (x_type == kXFp8) {
    if (tc)
      return launch_dual_pass_tc_fp8(L, static_cast<const uint8_t*>(X), m, n, ell, V, U, Y, Z, ws,
                                     ws_bytes, status, z_kmajor);
    // the FP8 copy: codes with row pitch ldq, then the tile scales (fp8_copy_bytes)
    int64_t ldq = 0, off = 0;
    fp8_copy_bytes(m, n, &ldq, &off);
    const uint8_t* q = static_cast<const uint8_t*>(X);
    return dispatch(L, q, m, n, ldq, ell, V, U, Y, Z, static_cast<float*>(ws), q + off,
                    (n + 31) / 32);
  }
  const bool x_bf16 = x_type == kXBf16;
  if (tc && x_type == kXFp32)
    return launch_dual_pass_tc_f32(L, static_cast<const float*>(X), m, n, ldx, ell, V, U, Y, Z,
                                   ws, ws_bytes, status, z_kmajor);
  if (tc)
    return launch_dual_pass_tc(L, static_cast<const __nv_bfloat16*>(X), m, n, ldx, ell, V, U, Y,
                               Z, ws, ws_bytes, status, split, z_kmajor);
  if (x_bf16)
    return dispatch(L, static_cast<const __nv_bfloat16*>(X), m, n, ldx, ell, V, U, Y, Z,
                    static_cast<float*>(ws));
  return dispatch(L, static_cast<const float*>(X), m, n, ldx, ell, V, U, Y, Z,
                  static_cast<float*>(ws));
}

}  // namespace nmfrp
