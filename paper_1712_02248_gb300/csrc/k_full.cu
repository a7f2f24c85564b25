// Iterations on the full data X (the uncompressed methods the paper compares against):
//   FastHALS (Section 2.2; Cichocki & Phan):  S_W = X H^T, G_W = H H^T, W sweep (Gauss-Seidel over
//     j), normalisation w_j /= ||w_j||, h_j *= ||w_j||, then S_H = W^T X, G_H = W^T W, H sweep.
//   MU (Section 2.1, Algorithm 1, Lee & Seung):  W <- W o (X H^T) / (W H H^T + eps), then
//     H <- H o (W^T X) / (W^T W H + eps) with the new W.
// X H^T and X^T W come from the dual pass over X (one pass each: the H sweep needs the W of
// this iteration). The r x r Grams are sums over row slabs (FP32 partials, fixed-order sum).
// The updates take one thread per row of W (column of H), the factor's r entries and the row of
// S in registers, G in shared memory.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kGramRows = 256;    // rows of a tall matrix one Gram block sums
constexpr int kUpdThreads = 128;

// part[b][p][q] = sum over rows [b kGramRows, ...) of A[i][p] A[i][q] (A rows x r, row-major).
__global__ void __launch_bounds__(256) gram_tall_partial_kernel(const float* __restrict__ A,
                                                                int64_t rows, int r,
                                                                float* __restrict__ part) {
  extern __shared__ float as[];   // [kGramRows][r]
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kGramRows;
  const int nr = static_cast<int>(rows - r0 < kGramRows ? rows - r0 : kGramRows);
  for (int e = threadIdx.x; e < kGramRows * r; e += blockDim.x)
    as[e] = e < nr * r ? A[r0 * r + e] : 0.f;
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e - p * r;
    float s = 0.f;
    for (int i = 0; i < nr; ++i) s = fmaf(as[i * r + p], as[i * r + q], s);
    part[static_cast<int64_t>(blockIdx.x) * r * r + e] = s;
  }
}

// G[e] = sum over blocks of part[b][e] in block order; norm_scale: s_j = sqrt(G_jj) (1 where
// G_jj = 0) into scale, and G[p][q] /= s_p s_q (the Gram of the normalised columns).
__global__ void gram_sum_kernel(const float* __restrict__ part, int nb, int r, int normalize,
                                float* __restrict__ G, float* __restrict__ scale) {
  extern __shared__ float g[];   // [r * r]
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[static_cast<int64_t>(b) * r * r + e];
    g[e] = s;
  }
  __syncthreads();
  if (!normalize) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) G[e] = g[e];
    return;
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e - p * r;
    const float sp = g[p * r + p] > 0.f ? sqrtf(g[p * r + p]) : 1.f;
    const float sq = g[q * r + q] > 0.f ? sqrtf(g[q * r + q]) : 1.f;
    G[e] = g[e] / (sp * sq);
    if (p == q) scale[p] = sp;
  }
}

// W[i][j] /= scale[j]
__global__ void scale_cols_kernel(float* __restrict__ W, int64_t m, int r,
                                  const float* __restrict__ scale) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m * r;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    W[e] /= scale[e % r];
}

// H (r x n) -> Ht (n x r)
__global__ void transpose_rn_kernel(const float* __restrict__ H, int r, int64_t n,
                                    float* __restrict__ Ht) {
  __shared__ float t[32][33];
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int j0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int j = j0 + i;
    const int64_t c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (j < r && c < n) ? H[j * n + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i;
    const int j = j0 + threadIdx.x;
    if (j < r && c < n) Ht[c * r + j] = t[threadIdx.x][i];
  }
}

// One thread per row i of W: S row (S_W = X H^T, m x r), G = H H^T.
//   RULE 0 (FastHALS): for j: w_j <- [w_j + (s_j - sum_q w_q G_qj) / G_jj]_+ (skip G_jj = 0)
//   RULE 1 (Lee-Seung): w_j <- w_j s_j / (sum_q w_q G_qj + eps) (all j from the old w)
template <int RP, int RULE>
__global__ void __launch_bounds__(kUpdThreads) full_w_update_kernel(const float* __restrict__ S,
                                                                    const float* __restrict__ G,
                                                                    int64_t m, int r, float eps,
                                                                    float* __restrict__ W) {
  __shared__ float Gs[RP * RP];
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    const int p = e / RP, q = e - p * RP;
    Gs[e] = (p < r && q < r) ? G[p * r + q] : 0.f;
  }
  __syncthreads();
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float w[RP], s[RP];
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      w[j] = j < r ? W[i * r + j] : 0.f;
      s[j] = j < r ? S[i * r + j] : 0.f;
    }
    if (RULE == 0) {
#pragma unroll
      for (int j = 0; j < RP; ++j) {
        const float g = Gs[j * RP + j];
        if (j < r && g > 0.f) {
          float t = s[j];
#pragma unroll
          for (int q = 0; q < RP; ++q) t = fmaf(-w[q], Gs[q * RP + j], t);
          w[j] = fmaxf(0.f, w[j] + t / g);
        }
      }
    } else {
      float wn[RP];
#pragma unroll
      for (int j = 0; j < RP; ++j) {
        float d = eps;
#pragma unroll
        for (int q = 0; q < RP; ++q) d = fmaf(w[q], Gs[q * RP + j], d);
        wn[j] = j < r ? w[j] * s[j] / d : 0.f;
      }
#pragma unroll
      for (int j = 0; j < RP; ++j) w[j] = wn[j];
    }
#pragma unroll
    for (int j = 0; j < RP; ++j)
      if (j < r) W[i * r + j] = w[j];
  }
}

// One thread per column c of H: the column scaled by scale (FastHALS compensation; null for MU),
// St row c (S_H^T = X^T W, n x r), G = W^T W (of the normalised W).
//   RULE 0: for j: h_j <- [(h_j G_jj + s_j - sum_q G_jq h_q - alpha) / (G_jj + beta)]_+ (the
//     Section 4.1 form; alpha = beta = 0 gives h_j + (s_j - sum_q G_jq h_q) / G_jj)
//   RULE 1: h_j <- h_j s_j / (sum_q G_jq h_q + eps)
template <int RP, int RULE>
__global__ void __launch_bounds__(kUpdThreads) full_h_update_kernel(
    const float* __restrict__ St, const float* __restrict__ G, const float* __restrict__ scale,
    int64_t n, int r, float alpha, float beta, float eps, float* __restrict__ H) {
  __shared__ float Gs[RP * RP];
  __shared__ float sc[RP];
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    const int p = e / RP, q = e - p * RP;
    Gs[e] = (p < r && q < r) ? G[p * r + q] : 0.f;
  }
  for (int j = threadIdx.x; j < RP; j += blockDim.x) sc[j] = (scale && j < r) ? scale[j] : 1.f;
  __syncthreads();
  const bool plain = alpha == 0.f && beta == 0.f;
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c < n;
       c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float h[RP], s[RP];
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      h[j] = j < r ? H[j * n + c] * sc[j] : 0.f;
      s[j] = j < r ? St[c * r + j] : 0.f;
    }
    if (RULE == 0) {
#pragma unroll
      for (int j = 0; j < RP; ++j) {
        if (j >= r) continue;
        const float g = Gs[j * RP + j];
        float t = s[j];
#pragma unroll
        for (int q = 0; q < RP; ++q) t = fmaf(-Gs[j * RP + q], h[q], t);
        if (plain) {
          if (g > 0.f) h[j] = fmaxf(0.f, h[j] + t / g);
        } else if (g + beta > 0.f) {
          h[j] = fmaxf(0.f, (fmaf(h[j], g, t) - alpha) / (g + beta));
        }
      }
    } else {
      float hn[RP];
#pragma unroll
      for (int j = 0; j < RP; ++j) {
        float d = eps;
#pragma unroll
        for (int q = 0; q < RP; ++q) d = fmaf(Gs[j * RP + q], h[q], d);
        hn[j] = j < r ? h[j] * s[j] / d : 0.f;
      }
#pragma unroll
      for (int j = 0; j < RP; ++j) h[j] = hn[j];
    }
#pragma unroll
    for (int j = 0; j < RP; ++j)
      if (j < r) H[j * n + c] = h[j];
  }
}

int blocks_for(int64_t count, int threads) {
  const int64_t b = cdiv(count, threads);
  return static_cast<int>(b < 4096 ? b : 4096);
}

cudaError_t gram_tall(const Launcher& L, const float* A, int64_t rows, int r, float* part,
                      float* G, float* scale, bool normalize) {
  const int nb = static_cast<int>(cdiv(rows, kGramRows));
  const size_t sm = sizeof(float) * kGramRows * r;
  cudaError_t err = cudaFuncSetAttribute(gram_tall_partial_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
  if (err != cudaSuccess) return err;
  gram_tall_partial_kernel<<<nb, 256, sm, L.stream>>>(A, rows, r, part);
  gram_sum_kernel<<<1, 256, sizeof(float) * r * r, L.stream>>>(part, nb, r, normalize ? 1 : 0, G,
                                                                scale);
  L.count(2);
  return cudaGetLastError();
}

template <int RP>
cudaError_t updates_w(const Launcher& L, int rule, const float* S, const float* G, int64_t m,
                      int r, float eps, float* W) {
  if (rule == 0)
    full_w_update_kernel<RP, 0><<<blocks_for(m, kUpdThreads), kUpdThreads, 0, L.stream>>>(S, G, m,
                                                                                         r, eps, W);
  else
    full_w_update_kernel<RP, 1><<<blocks_for(m, kUpdThreads), kUpdThreads, 0, L.stream>>>(S, G, m,
                                                                                         r, eps, W);
  L.count();
  return cudaGetLastError();
}

template <int RP>
cudaError_t updates_h(const Launcher& L, int rule, const float* St, const float* G,
                      const float* scale, int64_t n, int r, float alpha, float beta, float eps,
                      float* H) {
  if (rule == 0)
    full_h_update_kernel<RP, 0><<<blocks_for(n, kUpdThreads), kUpdThreads, 0, L.stream>>>(
        St, G, scale, n, r, alpha, beta, eps, H);
  else
    full_h_update_kernel<RP, 1><<<blocks_for(n, kUpdThreads), kUpdThreads, 0, L.stream>>>(
        St, G, scale, n, r, alpha, beta, eps, H);
  L.count();
  return cudaGetLastError();
}

}  // namespace

size_t iterate_full_ws_bytes(int64_t m, int64_t n, int r) {
  const int64_t nb = cdiv(m > n ? m : n, kGramRows);
  return sizeof(float) * static_cast<size_t>(n * r + m * r + n * r + m * r + nb * r * r +
                                             2 * r * r + 2 * r) +
         dual_pass_ws_bytes(m, n, r) + 8 * 256;
}

cudaError_t launch_iterate_full(const Launcher& L, const void* X, int x_type, int64_t m, int64_t n,
                                int64_t ldx, int r, int rule, float alpha, float beta, float eps,
                                float* W, float* H, int iters, void* ws, size_t ws_bytes,
                                int* status, bool force_simt) {
  if (r < 1 || r > 64) return cudaErrorNotSupported;
  if (ws_bytes < iterate_full_ws_bytes(m, n, r)) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t floats) {
    float* f = reinterpret_cast<float*>(p);
    p += (sizeof(float) * floats + 255) / 256 * 256;
    return f;
  };
  const int64_t nb = cdiv(m > n ? m : n, kGramRows);
  float* Ht = take(n * r);     // H^T (n x r)
  float* SW = take(m * r);     // X H^T
  float* ST = take(n * r);     // X^T W = S_H^T
  float* Ys = take(m * r);     // the pass's other product on the tensor-core path (unused)
  float* part = take(nb * r * r);
  float* GW = take(r * r);
  float* GH = take(r * r);
  float* scale = take(r);
  const size_t used = static_cast<size_t>(p - static_cast<char*>(ws));
  void* pws = p;
  const size_t pbytes = ws_bytes - used;
  // the tensor-core pass needs both products: the unused one goes to scratch (same X read)
  const bool tc = dual_pass_uses_tc(X, x_type, m, n, ldx, r, true, force_simt);
  const int RP = r <= 8 ? 8 : r <= 16 ? 16 : r <= 32 ? 32 : 64;
  const dim3 tg(static_cast<unsigned>(cdiv(n, 32)), static_cast<unsigned>(cdiv(r, 32)));
  cudaError_t err = cudaSuccess;
  for (int it = 0; it < iters; ++it) {
    transpose_rn_kernel<<<tg, dim3(32, 8), 0, L.stream>>>(H, r, n, Ht);
    L.count();
    // S_W = X H^T (the split operands keep H in FP32 accuracy: only X is rounded)
    if ((err = launch_dual_pass(L, X, x_type, m, n, ldx, r, Ht, tc ? W : nullptr, SW,
                                tc ? ST : nullptr, pws, pbytes, status, force_simt, true)) !=
        cudaSuccess)
      return err;
    if ((err = gram_tall(L, Ht, n, r, part, GW, nullptr, false)) != cudaSuccess) return err;
    switch (RP) {
      case 8: err = updates_w<8>(L, rule, SW, GW, m, r, eps, W); break;
      case 16: err = updates_w<16>(L, rule, SW, GW, m, r, eps, W); break;
      case 32: err = updates_w<32>(L, rule, SW, GW, m, r, eps, W); break;
      default: err = updates_w<64>(L, rule, SW, GW, m, r, eps, W); break;
    }
    if (err != cudaSuccess) return err;
    // G_H = W^T W; FastHALS normalises the columns of W (scale moved to the rows of H)
    const bool norm = rule == 0;
    if ((err = gram_tall(L, W, m, r, part, GH, scale, norm)) != cudaSuccess) return err;
    if (norm) {
      scale_cols_kernel<<<blocks_for(m * r, 256), 256, 0, L.stream>>>(W, m, r, scale);
      L.count();
    }
    // S_H^T = X^T W
    if ((err = launch_dual_pass(L, X, x_type, m, n, ldx, r, tc ? Ht : nullptr, W, tc ? Ys : nullptr,
                                ST, pws, pbytes, status, force_simt, true)) != cudaSuccess)
      return err;
    const float* sc = norm ? scale : nullptr;
    switch (RP) {
      case 8: err = updates_h<8>(L, rule, ST, GH, sc, n, r, alpha, beta, eps, H); break;
      case 16: err = updates_h<16>(L, rule, ST, GH, sc, n, r, alpha, beta, eps, H); break;
      case 32: err = updates_h<32>(L, rule, ST, GH, sc, n, r, alpha, beta, eps, H); break;
      default: err = updates_h<64>(L, rule, ST, GH, sc, n, r, alpha, beta, eps, H); break;
    }
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace nmfrp
