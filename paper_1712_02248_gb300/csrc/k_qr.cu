// Thin QR of a tall FP32 matrix (Section 3, Eq. 3.4-3.5: Q from the QR decomposition of the
// sketch) by CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa & Yamamoto 2014): twice
//   G = Y^T Y (FP64 sums of exact FP32 products), G = R^T R (FP64 Cholesky), Y <- Y R^{-1}.
// R^{-1} is formed in FP64. The first sweep applies it with FP64 accumulation (its entries are
// as large as cond(Y), and products of that size cancel); the second sweep's factor is close to
// the identity and is applied in FP32. The result is the Q of the QR factorisation whose R has a
// positive diagonal, rounded to FP32.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kGramRows = 128;   // rows per Gram block
constexpr int kGramThreads = 256;

// Partial Gram of a 128-row slab: Gp[blk][p][q] for p <= q (2x2 register tiles, FP64 FMA).
template <int LP>
__global__ void __launch_bounds__(kGramThreads) gram_partial_kernel(
    const float* __restrict__ Y, int64_t rows, int ell, double* __restrict__ Gp) {
  extern __shared__ __align__(16) float Ysm[];   // [kGramRows][LP]
  auto Ys = reinterpret_cast<float(*)[LP]>(Ysm);
  const int t = threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kGramRows;
  for (int e = t; e < kGramRows * LP; e += kGramThreads) {
    const int i = e / LP, k = e - i * LP;
    const int64_t gr = r0 + i;
    Ys[i][k] = (gr < rows && k < ell) ? Y[gr * ell + k] : 0.f;
  }
  __syncthreads();
  constexpr int T2 = LP / 2;
  double* out = Gp + static_cast<int64_t>(blockIdx.x) * LP * LP;
  for (int tile = t; tile < T2 * T2; tile += kGramThreads) {
    const int P = tile / T2, Qi = tile - P * T2;
    if (P > Qi) continue;
    double a00 = 0, a01 = 0, a10 = 0, a11 = 0;
#pragma unroll 4
    for (int i = 0; i < kGramRows; ++i) {
      const float2 a = *reinterpret_cast<const float2*>(&Ys[i][2 * P]);
      const float2 b = *reinterpret_cast<const float2*>(&Ys[i][2 * Qi]);
      const double a0 = a.x, a1 = a.y, b0 = b.x, b1 = b.y;
      a00 = fma(a0, b0, a00);
      a01 = fma(a0, b1, a01);
      a10 = fma(a1, b0, a10);
      a11 = fma(a1, b1, a11);
    }
    out[(2 * P) * LP + 2 * Qi] = a00;
    out[(2 * P) * LP + 2 * Qi + 1] = a01;
    out[(2 * P + 1) * LP + 2 * Qi] = a10;
    out[(2 * P + 1) * LP + 2 * Qi + 1] = a11;
  }
}

// G[e] = sum_b Gp[b][e] for every entry e < LP*LP: one warp per entry, lanes stride the parts,
// then a fixed shuffle tree (deterministic).
__global__ void sum_parts_kernel(const double* __restrict__ Gp, int nparts, int entries,
                                 double* __restrict__ G) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= entries) return;
  double s = 0.0;
  for (int b = lane; b < nparts; b += 32) s += Gp[static_cast<int64_t>(b) * entries + warp];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) G[warp] = s;
}

// One CTA: Cholesky G = R^T R (in place on the upper triangle), T = R^{-1}. T's strictly upper
// part is kept transposed in the lower triangle of the same array and its diagonal separately.
// Writes T (ell x ell, row-major, FP32) for the application kernel.
template <int LP>
__global__ void __launch_bounds__(1024) chol_inv_kernel(const double* __restrict__ Gin, int ell,
                                                        float* __restrict__ Tout,
                                                        double* __restrict__ Tout64, int* status) {
  constexpr int S = LP + 1;
  extern __shared__ __align__(16) double sh[];
  double* A = sh;          // [LP][S]
  double* dT = A + LP * S; // [LP]
  __shared__ int bad;
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) bad = 0;
  for (int e = t; e < LP * LP; e += nt) {
    const int p = e / LP, q = e - p * LP;
    A[p * S + q] = (p <= q && q < ell) ? Gin[p * LP + q] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < ell; ++j) {
    if (t == 0) {
      double d = A[j * S + j];
      // a non-positive pivot: the sketch is numerically rank deficient
      if (!(d > 0.0)) {
        bad = 1;
        d = 1e-300;
      }
      A[j * S + j] = sqrt(d);
    }
    __syncthreads();
    const double rjj = A[j * S + j];
    for (int q = j + 1 + t; q < ell; q += nt) A[j * S + q] /= rjj;
    __syncthreads();
    const int w = ell - j - 1;
    for (int e = t; e < w * w; e += nt) {
      const int p = j + 1 + e / w, q = j + 1 + e % w;
      if (p <= q) A[p * S + q] -= A[j * S + p] * A[j * S + q];
    }
    __syncthreads();
  }
  // T = R^{-1}, column c by back substitution (one warp per column):
  //   T[c][c] = 1 / R[c][c];  T[i][c] = -(sum_{k=i+1..c} R[i][k] T[k][c]) / R[i][i]
  // T[k][c] (k < c) lives at A[c][k].
  const int warp = t >> 5, lane = t & 31, nw = nt >> 5;
  for (int c = warp; c < ell; c += nw) {
    const double tcc = 1.0 / A[c * S + c];
    if (lane == 0) dT[c] = tcc;
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1 + lane; k <= c; k += 32) {
        const double tkc = (k == c) ? tcc : A[c * S + k];
        s += A[i * S + k] * tkc;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) A[c * S + i] = -s / A[i * S + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = t; e < ell * ell; e += nt) {
    const int p = e / ell, q = e - p * ell;
    double v = 0.0;
    if (p == q) v = dT[p];
    else if (p < q) v = A[q * S + p];
    Tout[e] = static_cast<float>(v);
    Tout64[e] = v;
  }
  if (t == 0 && bad) latch(status, kStQrBreakdown);
}

// Q = Y T (T upper triangular ell x ell), accumulated in ACC (float or double), stored FP32.
// One thread per (row, block of 8 columns).
template <int LP, typename ACC>
__global__ void __launch_bounds__(256) apply_tri_kernel(const float* __restrict__ Y, int64_t rows,
                                                        int ell, const ACC* __restrict__ T,
                                                        float* __restrict__ Q) {
  extern __shared__ __align__(16) unsigned char tsm[];
  ACC* Ts = reinterpret_cast<ACC*>(tsm);   // [LP][LP]
  for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
    const int p = e / LP, q = e - p * LP;
    Ts[e] = (p < ell && q < ell) ? T[p * ell + q] : ACC(0);
  }
  __syncthreads();
  constexpr int CB = 8, NCB = LP / CB;
  const int64_t total = rows * NCB;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / NCB;
    const int cb = static_cast<int>(e - i * NCB);
    ACC acc[CB];
#pragma unroll
    for (int q = 0; q < CB; ++q) acc[q] = ACC(0);
    const float* yr = Y + i * ell;
    const int kmax = min(ell, (cb + 1) * CB);
    for (int k = 0; k < kmax; ++k) {
      const ACC y = static_cast<ACC>(yr[k]);
#pragma unroll
      for (int q = 0; q < CB; ++q) acc[q] = fma(y, Ts[k * LP + cb * CB + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const int c = cb * CB + q;
      if (c < ell) Q[i * ell + c] = static_cast<float>(acc[q]);
    }
  }
}

int lp_for(int ell) {
  if (ell <= 16) return 16;
  if (ell <= 32) return 32;
  if (ell <= 48) return 48;
  if (ell <= 64) return 64;
  if (ell <= 96) return 96;
  return 128;
}

struct QrWs {
  double* Gp;   // nparts x LP x LP
  double* G;    // LP x LP
  double* T64;  // LP x LP
  float* T;     // LP x LP
  float* Q1;    // rows x ell
};

QrWs carve(char* ws, int64_t rows, int ell, int LP) {
  const int64_t nparts = cdiv(rows, kGramRows);
  QrWs w;
  w.Gp = reinterpret_cast<double*>(ws);
  w.G = w.Gp + nparts * LP * LP;
  w.T64 = w.G + LP * LP;
  w.T = reinterpret_cast<float*>(w.T64 + LP * LP);
  w.Q1 = w.T + LP * LP;
  return w;
}

template <int LP>
cudaError_t run(const Launcher& L, const float* Y, int64_t rows, int ell, float* Q, char* ws,
                int* status) {
  const int64_t nparts = cdiv(rows, kGramRows);
  const QrWs w = carve(ws, rows, ell, LP);
  const size_t chol_smem = sizeof(double) * (LP * (LP + 1) + LP);
  const size_t gram_smem = sizeof(float) * kGramRows * LP;
  const size_t apply_smem64 = sizeof(double) * LP * LP;
  const size_t apply_smem32 = sizeof(float) * LP * LP;
  cudaError_t err;
  if ((err = cudaFuncSetAttribute(chol_inv_kernel<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(chol_smem))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(gram_partial_kernel<LP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(gram_smem))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(apply_tri_kernel<LP, double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(apply_smem64))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(apply_tri_kernel<LP, float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(apply_smem32))) != cudaSuccess)
    return err;
  const int chol_threads = LP >= 64 ? 1024 : 512;
  const int64_t apply_work = rows * (LP / 8);
  const unsigned apply_grid =
      static_cast<unsigned>(cdiv(apply_work, 256) < 4096 ? cdiv(apply_work, 256) : 4096);
  const unsigned sum_grid = static_cast<unsigned>(cdiv(static_cast<int64_t>(LP) * LP * 32, 256));
  // Q may alias Y: sweep 0 reads Y and writes the scratch Q1; sweep 1 reads Q1 and writes Q.
  const float* src = Y;
  for (int sweep = 0; sweep < 2; ++sweep) {
    gram_partial_kernel<LP><<<static_cast<unsigned>(nparts), kGramThreads, gram_smem, L.stream>>>(
        src, rows, ell, w.Gp);
    sum_parts_kernel<<<sum_grid, 256, 0, L.stream>>>(w.Gp, static_cast<int>(nparts), LP * LP,
                                                     w.G);
    chol_inv_kernel<LP><<<1, chol_threads, chol_smem, L.stream>>>(w.G, ell, w.T, w.T64, status);
    if (sweep == 0)
      apply_tri_kernel<LP, double><<<apply_grid, 256, apply_smem64, L.stream>>>(src, rows, ell,
                                                                               w.T64, w.Q1);
    else
      apply_tri_kernel<LP, float><<<apply_grid, 256, apply_smem32, L.stream>>>(src, rows, ell,
                                                                              w.T, Q);
    L.count(4);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    src = w.Q1;
  }
  return cudaSuccess;
}

}  // namespace

size_t qr_ws_bytes(int64_t rows, int ell) {
  const int LP = lp_for(ell);
  const int64_t nparts = cdiv(rows, kGramRows);
  return sizeof(double) * (nparts + 2) * LP * LP + sizeof(float) * (LP * LP + rows * ell) + 256;
}

cudaError_t launch_qr(const Launcher& L, const float* Y, int64_t rows, int ell, float* Q,
                      void* ws, size_t ws_bytes, int* status) {
  if (ws_bytes < qr_ws_bytes(rows, ell)) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(ws);
  switch (lp_for(ell)) {
    case 16: return run<16>(L, Y, rows, ell, Q, w, status);
    case 32: return run<32>(L, Y, rows, ell, Q, w, status);
    case 48: return run<48>(L, Y, rows, ell, Q, w, status);
    case 64: return run<64>(L, Y, rows, ell, Q, w, status);
    case 96: return run<96>(L, Y, rows, ell, Q, w, status);
    default: return run<128>(L, Y, rows, ell, Q, w, status);
  }
}

}  // namespace nmfrp
