// Learned warm start: the per-row network (three layers, ReLU) that corrects the NNDSVD factors,
// trained on solutions of the compressed NMF itself. Forward, gradient and Adam kernels.
//
// Parameter vector (FP32 master copy): [W1 (F x Hd), b1 (Hd), W2 (Hd x Hd), b2 (Hd),
// W3 (Hd x r), b3 (r)], matrices row-major. The weight matrices enter every product rounded to
// BF16 (round to nearest even, applied when a tile is staged); biases, activations and all
// accumulation are FP32. Loss: mean of squared errors over the rows x r outputs; the gradient is
// that of the rounded weights and is applied to the master copy by Adam.
//
// Products: one tiled SIMT kernel (64 x 64 output tile, 16-deep K slices in shared memory,
// 4 x 4 outputs a thread) with the transposes and epilogues the three passes need:
//   forward   A (B x F) . W            + bias, ReLU (hidden layers) / + bias (output)
//   backward  G (B x N) . W^T          masked by the next activation > 0 (ReLU derivative)
//             A^T (K x B) . G          weight gradients
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kT = 64, kK = 16, kThreads = 256;

enum Epi { kStore = 0, kBiasRelu = 1, kBias = 2, kMask = 3 };

__device__ __forceinline__ float round_bf16(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// C[M x N] = epilogue(op(A) op(B)); op(A) = A (M x K, lda) or A^T (A stored K x M);
// op(B) = B (K x N, ldb) or B^T (B stored N x K). round_b: round B's entries to BF16.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(kThreads) mlp_gemm_kernel(int M, int N, int K,
                                                            const float* __restrict__ A, int lda,
                                                            const float* __restrict__ B, int ldb,
                                                            float* __restrict__ C, int ldc,
                                                            const float* __restrict__ bias,
                                                            const float* __restrict__ mask,
                                                            int round_b) {
  __shared__ float As[kK][kT + 4];
  __shared__ float Bs[kK][kT + 4];
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int m0 = blockIdx.y * kT, n0 = blockIdx.x * kT;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kK) {
    for (int e = t; e < kK * kT; e += kThreads) {
      // A tile: As[kk][mm]
      int kk, mm;
      if (TA) {
        kk = e / kT;
        mm = e % kT;
      } else {
        mm = e / kK;
        kk = e % kK;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      float a = 0.f;
      if (gm < M && gk < K) a = TA ? A[static_cast<int64_t>(gk) * lda + gm] : A[static_cast<int64_t>(gm) * lda + gk];
      As[kk][mm] = a;
      // B tile: Bs[kk][nn]
      int kb, nn;
      if (TB) {
        nn = e / kK;
        kb = e % kK;
      } else {
        kb = e / kT;
        nn = e % kT;
      }
      const int gn = n0 + nn, gkb = k0 + kb;
      float b = 0.f;
      if (gn < N && gkb < K) b = TB ? B[static_cast<int64_t>(gn) * ldb + gkb] : B[static_cast<int64_t>(gkb) * ldb + gn];
      Bs[kb][nn] = round_b ? round_bf16(b) : b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (EPI == kBiasRelu) v = fmaxf(v + bias[gn], 0.f);
      if (EPI == kBias) v += bias[gn];
      if (EPI == kMask) v = mask[static_cast<int64_t>(gm) * ldc + gn] > 0.f ? v : 0.f;
      C[static_cast<int64_t>(gm) * ldc + gn] = v;
    }
  }
}

// E = Y - T; G = 2 E / (rows r); per-block partial sums of E^2 for the loss (float-float with
// exact products within a thread, FP64 across threads).
__global__ void __launch_bounds__(256) mse_grad_kernel(const float* __restrict__ Y,
                                                       const float* __restrict__ T, int64_t total,
                                                       float scale, float* __restrict__ G,
                                                       double* __restrict__ part) {
  __shared__ double red[8];
  FSum fs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    G[e] = scale * d;
    fs.add_prod(d, d);
  }
  double s = fs.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < 8; ++w) a += red[w];
    part[blockIdx.x] = a;
  }
}

__global__ void loss_final_kernel(const double* __restrict__ part, int nparts, double inv_total,
                                  double* __restrict__ loss) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) a += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (threadIdx.x == 0) *loss = a * inv_total;
}

// db[j] = sum over rows of G[row][j] (32 columns a block, rows split over 8 warps, fixed order).
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ G, int64_t rows,
                                                     int cols, float* __restrict__ db) {
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (j < cols)
    for (int64_t i = w; i < rows; i += 8) s += G[i * cols + j];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && j < cols) {
    float a = 0.f;
    for (int k = 0; k < 8; ++k) a += red[k][lane];
    db[j] = a;
  }
}

// Adam with bias correction: c1 = 1 - beta1^t, c2 = 1 - beta2^t; o1 = 1 - beta1, o2 = 1 - beta2
// (formed in double on the host: 1 - 0.999f in FP32 is 1.3e-5 away from 0.001).
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t count, float lr, float b1,
                            float b2, float o1, float o2, float eps, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = fmaf(b1, m[e], o1 * gi);
    const float vi = fmaf(b2, v[e], o2 * gi * gi);
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// W0 = max(0, Wb + Dw / sqrt(m)); H0[j][c] = max(0, Hb[j][c] + hscale[j] Dh[c][j] / sqrt(n)).
__global__ void ws_apply_kernel(const float* __restrict__ Wb, const float* __restrict__ Dw,
                                int64_t m, const float* __restrict__ Hb,
                                const float* __restrict__ Dh, const float* __restrict__ hscale,
                                int64_t n, int r, float* __restrict__ W, float* __restrict__ H) {
  const int64_t tw = m * r, th = static_cast<int64_t>(r) * n;
  const float im = rsqrtf(static_cast<float>(m)), in = rsqrtf(static_cast<float>(n));
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tw + th;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < tw) {
      W[e] = fmaxf(0.f, fmaf(Dw[e], im, Wb[e]));
    } else {
      const int64_t g = e - tw;
      const int j = static_cast<int>(g / n);
      const int64_t c = g - static_cast<int64_t>(j) * n;
      H[g] = fmaxf(0.f, fmaf(hscale[j] * Dh[c * r + j], in, Hb[g]));
    }
  }
}

int grid_1d(int64_t work) {
  const int64_t b = cdiv(work, 256);
  return static_cast<int>(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const Launcher& L, int M, int N, int K, const float* A, int lda, const float* B,
                 int ldb, float* C, int ldc, const float* bias, const float* mask, bool round_b) {
  dim3 grid(static_cast<unsigned>(cdiv(N, kT)), static_cast<unsigned>(cdiv(M, kT)));
  mlp_gemm_kernel<TA, TB, EPI><<<grid, kThreads, 0, L.stream>>>(M, N, K, A, lda, B, ldb, C, ldc,
                                                                bias, mask, round_b ? 1 : 0);
  L.count();
  return cudaGetLastError();
}

struct Net {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};

Net unpack(const float* p, int F, int Hd, int r) {
  Net n;
  n.W1 = p;
  n.b1 = n.W1 + static_cast<int64_t>(F) * Hd;
  n.W2 = n.b1 + Hd;
  n.b2 = n.W2 + static_cast<int64_t>(Hd) * Hd;
  n.W3 = n.b2 + Hd;
  n.b3 = n.W3 + static_cast<int64_t>(Hd) * r;
  return n;
}

}  // namespace

int64_t mlp_param_count(int F, int Hd, int r) {
  return static_cast<int64_t>(F) * Hd + Hd + static_cast<int64_t>(Hd) * Hd + Hd +
         static_cast<int64_t>(Hd) * r + r;
}

size_t mlp_ws_bytes(int64_t rows, int Hd, int r) {
  // A1, A2 (rows x Hd), G2, G1 (rows x Hd), Y / G3 (rows x r), loss partials
  return sizeof(float) * static_cast<size_t>(rows) * (4 * Hd + 2 * r) + sizeof(double) * 4096 +
         4 * 256;
}

// Y (rows x r) = net(X); ws holds the two hidden activations.
cudaError_t launch_mlp_forward(const Launcher& L, int F, int Hd, int r, const float* params,
                               const float* X, int64_t rows, float* Y, void* ws, size_t ws_bytes) {
  if (ws_bytes < mlp_ws_bytes(rows, Hd, r) || rows > (int64_t(1) << 30)) return cudaErrorInvalidValue;
  const Net n = unpack(params, F, Hd, r);
  float* A1 = static_cast<float*>(ws);
  float* A2 = A1 + rows * Hd;
  const int R = static_cast<int>(rows);
  cudaError_t e;
  if ((e = gemm<false, false, kBiasRelu>(L, R, Hd, F, X, F, n.W1, Hd, A1, Hd, n.b1, nullptr, true)) != cudaSuccess) return e;
  if ((e = gemm<false, false, kBiasRelu>(L, R, Hd, Hd, A1, Hd, n.W2, Hd, A2, Hd, n.b2, nullptr, true)) != cudaSuccess) return e;
  return gemm<false, false, kBias>(L, R, r, Hd, A2, Hd, n.W3, r, Y, r, n.b3, nullptr, true);
}

// grad (param vector layout) of the mean squared error of net(X) against T; *loss (device).
cudaError_t launch_mlp_loss_grad(const Launcher& L, int F, int Hd, int r, const float* params,
                                 const float* X, const float* T, int64_t rows, float* grad,
                                 double* loss, void* ws, size_t ws_bytes) {
  if (ws_bytes < mlp_ws_bytes(rows, Hd, r) || rows < 1 || rows > (int64_t(1) << 30))
    return cudaErrorInvalidValue;
  const Net n = unpack(params, F, Hd, r);
  float* A1 = static_cast<float*>(ws);
  float* A2 = A1 + rows * Hd;
  float* G2 = A2 + rows * Hd;
  float* G1 = G2 + rows * Hd;
  float* Y = G1 + rows * Hd;
  float* G3 = Y + rows * r;
  double* part = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(G3 + rows * r) + 255) & ~static_cast<uintptr_t>(255));
  float* dW1 = grad;
  float* db1 = dW1 + static_cast<int64_t>(F) * Hd;
  float* dW2 = db1 + Hd;
  float* db2 = dW2 + static_cast<int64_t>(Hd) * Hd;
  float* dW3 = db2 + Hd;
  float* db3 = dW3 + static_cast<int64_t>(Hd) * r;
  const int R = static_cast<int>(rows);
  cudaError_t e;
  if ((e = gemm<false, false, kBiasRelu>(L, R, Hd, F, X, F, n.W1, Hd, A1, Hd, n.b1, nullptr, true)) != cudaSuccess) return e;
  if ((e = gemm<false, false, kBiasRelu>(L, R, Hd, Hd, A1, Hd, n.W2, Hd, A2, Hd, n.b2, nullptr, true)) != cudaSuccess) return e;
  if ((e = gemm<false, false, kBias>(L, R, r, Hd, A2, Hd, n.W3, r, Y, r, n.b3, nullptr, true)) != cudaSuccess) return e;
  const int64_t tot = rows * r;
  const int gb = grid_1d(tot) < 4096 ? grid_1d(tot) : 4096;
  mse_grad_kernel<<<gb, 256, 0, L.stream>>>(Y, T, tot, 2.f / static_cast<float>(tot), G3, part);
  loss_final_kernel<<<1, 32, 0, L.stream>>>(part, gb, 1.0 / static_cast<double>(tot), loss);
  L.count(2);
  // layer 3
  if ((e = gemm<true, false, kStore>(L, Hd, r, R, A2, Hd, G3, r, dW3, r, nullptr, nullptr, false)) != cudaSuccess) return e;
  colsum_kernel<<<static_cast<unsigned>(cdiv(r, 32)), 256, 0, L.stream>>>(G3, rows, r, db3);
  // layer 2: G2 = (G3 W3^T) * [A2 > 0]
  if ((e = gemm<false, true, kMask>(L, R, Hd, r, G3, r, n.W3, r, G2, Hd, nullptr, A2, true)) != cudaSuccess) return e;
  if ((e = gemm<true, false, kStore>(L, Hd, Hd, R, A1, Hd, G2, Hd, dW2, Hd, nullptr, nullptr, false)) != cudaSuccess) return e;
  colsum_kernel<<<static_cast<unsigned>(cdiv(Hd, 32)), 256, 0, L.stream>>>(G2, rows, Hd, db2);
  // layer 1: G1 = (G2 W2^T) * [A1 > 0]
  if ((e = gemm<false, true, kMask>(L, R, Hd, Hd, G2, Hd, n.W2, Hd, G1, Hd, nullptr, A1, true)) != cudaSuccess) return e;
  if ((e = gemm<true, false, kStore>(L, F, Hd, R, X, F, G1, Hd, dW1, Hd, nullptr, nullptr, false)) != cudaSuccess) return e;
  colsum_kernel<<<static_cast<unsigned>(cdiv(Hd, 32)), 256, 0, L.stream>>>(G1, rows, Hd, db1);
  L.count(3);
  return cudaGetLastError();
}

cudaError_t launch_adam(const Launcher& L, float* p, float* m, float* v, const float* g,
                        int64_t count, float lr, int step) {
  if (step < 1) return cudaErrorInvalidValue;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = static_cast<float>(1.0 - pow(b1, step));
  const float c2 = static_cast<float>(1.0 - pow(b2, step));
  adam_kernel<<<grid_1d(count), 256, 0, L.stream>>>(
      p, m, v, g, count, lr, static_cast<float>(b1), static_cast<float>(b2),
      static_cast<float>(1.0 - b1), static_cast<float>(1.0 - b2), 1e-8f, c1, c2);
  L.count();
  return cudaGetLastError();
}

// Training targets (the inverse of the apply map where the solution is positive):
// Tw = sqrt(m) (W* - W_b) (m x r); Th[c][j] = sqrt(n) (H*[j][c] - H_b[j][c]) / hscale_j (n x r,
// a zero scale taken as 1).
__global__ void ws_targets_kernel(const float* __restrict__ Wb, const float* __restrict__ Ws,
                                  int64_t m, const float* __restrict__ Hb,
                                  const float* __restrict__ Hs, const float* __restrict__ hscale,
                                  int64_t n, int r, float* __restrict__ Tw,
                                  float* __restrict__ Th) {
  const float sm = sqrtf(static_cast<float>(m)), sn = sqrtf(static_cast<float>(n));
  const int64_t tw = m * r, tot = tw + n * r;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < tot;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (e < tw) {
      Tw[e] = sm * (Ws[e] - Wb[e]);
    } else {
      const int64_t f = e - tw, c = f / r;
      const int j = static_cast<int>(f - c * r);
      const float h = hscale[j] > 0.f ? hscale[j] : 1.f;
      const int64_t src = static_cast<int64_t>(j) * n + c;
      Th[f] = sn * (Hs[src] - Hb[src]) / h;
    }
  }
}

cudaError_t launch_warmstart_targets(const Launcher& L, int64_t m, int64_t n, int r,
                                     const float* Wb, const float* Hb, const float* hscale,
                                     const float* Wstar, const float* Hstar, float* Tw,
                                     float* Th) {
  ws_targets_kernel<<<grid_1d(m * r + r * n), 256, 0, L.stream>>>(Wb, Wstar, m, Hb, Hstar, hscale,
                                                                   n, r, Tw, Th);
  L.count();
  return cudaGetLastError();
}

cudaError_t launch_warmstart_apply(const Launcher& L, int64_t m, int64_t n, int r,
                                   const float* Wb, const float* Dw, const float* Hb,
                                   const float* Dh, const float* hscale, float* W, float* H) {
  ws_apply_kernel<<<grid_1d(m * r + r * n), 256, 0, L.stream>>>(Wb, Dw, m, Hb, Dh, hscale, n, r,
                                                                 W, H);
  L.count();
  return cudaGetLastError();
}

}  // namespace nmfrp
