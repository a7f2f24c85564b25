// Compressed NMF iterations on W (m x r) and H (r x n); X is never read.
//
// FastHALS-RP (Section 4, Eq. fastHALS_a; Section 4.1 regularised form on H):
//   H_tld = H Q_R,  G_W = H_tld H_tld^T,  S_W = X_chk H_tld^T
//   for j = 1..r:  w_j <- [w_j + (S_W[:,j] - W G_W[:,j]) / G_W[j,j]]_+        (rows independent)
//   s_j = ||w_j||;  w_j /= s_j;  h_j *= s_j                                    (normalisation)
//   W_tld = Q_L^T W,  G_H = W_tld^T W_tld,  S_H = W_tld^T X_hat
//   for j = 1..r:  h_j <- [(h_j G_jj + S_H[j] - G_H[j,:] H - alpha) / (G_jj + beta)]_+   (columns
//   independent; alpha = beta = 0 is h_j + (S_H[j] - G_H[j,:] H) / G_jj)
// MU-RP (Section 3.1, Algorithm 3, semi-NMF rule of Ding, Li & Jordan 2010):
//   W <- W o sqrt((S_W^+ + W G_W^-) / (S_W^- + W G_W^+ + eps)),
//   H <- H o sqrt((S_H^+ + G_H^- H) / (S_H^- + G_H^+ H + eps)).
// The reductions over n (H_tld) and m (W_tld, column norms) write per-block partials that a
// warp-per-entry kernel sums in a fixed order.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kSlab = 128;  // rows (or columns) per reduction block

__device__ __forceinline__ float posp(float v) { return v > 0.f ? v : 0.f; }
__device__ __forceinline__ float negp(float v) { return v < 0.f ? -v : 0.f; }

// Hpart[b][j][k] = sum_{c in slab b} H[j][c] QR[c][k]
__global__ void __launch_bounds__(256) ht_partial_kernel(const float* __restrict__ H,
                                                         const float* __restrict__ QR, int64_t n,
                                                         int r, int ell, float* __restrict__ Hpart) {
  extern __shared__ float sh[];
  float* Hs = sh;                 // [r][kSlab]
  float* Qs = Hs + r * kSlab;     // [kSlab][ell]
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kSlab;
  for (int e = threadIdx.x; e < r * kSlab; e += blockDim.x) {
    const int j = e / kSlab, c = e - j * kSlab;
    Hs[e] = (c0 + c < n) ? H[j * n + c0 + c] : 0.f;
  }
  for (int e = threadIdx.x; e < kSlab * ell; e += blockDim.x) {
    const int c = e / ell;
    Qs[e] = (c0 + c < n) ? QR[c0 * ell + e] : 0.f;
  }
  __syncthreads();
  float* out = Hpart + static_cast<int64_t>(blockIdx.x) * r * ell;
  for (int e = threadIdx.x; e < r * ell; e += blockDim.x) {
    const int j = e / ell, k = e - j * ell;
    float s = 0.f;
#pragma unroll 8
    for (int c = 0; c < kSlab; ++c) s = fmaf(Hs[j * kSlab + c], Qs[c * ell + k], s);
    out[e] = s;
  }
}

// Wpart[b][k][j] = sum_{i in slab b} QL[i][k] W[i][j];  Wpart[b][ell*r + j] = sum_i W[i][j]^2
__global__ void __launch_bounds__(256) wt_partial_kernel(const float* __restrict__ QL,
                                                         const float* __restrict__ W, int64_t m,
                                                         int r, int ell, float* __restrict__ Wpart) {
  extern __shared__ float sh[];
  float* Qs = sh;                 // [kSlab][ell]
  float* Ws = Qs + kSlab * ell;   // [kSlab][r]
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kSlab;
  for (int e = threadIdx.x; e < kSlab * ell; e += blockDim.x) {
    const int i = e / ell;
    Qs[e] = (i0 + i < m) ? QL[i0 * ell + e] : 0.f;
  }
  for (int e = threadIdx.x; e < kSlab * r; e += blockDim.x) {
    const int i = e / r;
    Ws[e] = (i0 + i < m) ? W[i0 * r + e] : 0.f;
  }
  __syncthreads();
  float* out = Wpart + static_cast<int64_t>(blockIdx.x) * (ell * r + r);
  for (int e = threadIdx.x; e < ell * r + r; e += blockDim.x) {
    float s = 0.f;
    if (e < ell * r) {
      const int k = e / r, j = e - k * r;
#pragma unroll 8
      for (int i = 0; i < kSlab; ++i) s = fmaf(Qs[i * ell + k], Ws[i * r + j], s);
    } else {
      const int j = e - ell * r;
#pragma unroll 8
      for (int i = 0; i < kSlab; ++i) s = fmaf(Ws[i * r + j], Ws[i * r + j], s);
    }
    out[e] = s;
  }
}

// out[e] = sum_b part[b][e]; one warp per entry, fixed shuffle tree.
__global__ void sum_slots_kernel(const float* __restrict__ part, int nparts, int entries,
                                 float* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= entries) return;
  float s = 0.f;
  for (int b = lane; b < nparts; b += 32) s += part[static_cast<int64_t>(b) * entries + warp];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[warp] = s;
}

// G_W = H_tld H_tld^T (r x r) from H_tld (r x ell).
__global__ void gram_rows_kernel(const float* __restrict__ Ht, int r, int ell,
                                 float* __restrict__ G) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e - p * r;
    float s = 0.f;
    for (int k = 0; k < ell; ++k) s = fmaf(Ht[p * ell + k], Ht[q * ell + k], s);
    G[e] = s;
  }
}

// From raw W_tld (ell x r) and column sums of squares: scale s_j (= ||w_j|| or 1),
// W_tld[:,j] /= s_j, G_H = W_tld^T W_tld.
__global__ void finish_wt_kernel(const float* __restrict__ raw, int r, int ell, int normalize,
                                 float* __restrict__ Wt, float* __restrict__ GH,
                                 float* __restrict__ scale) {
  extern __shared__ float sh[];
  float* s = sh;          // [r]
  float* Ws = s + r;      // [ell][r]
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    const float c2 = raw[ell * r + j];
    s[j] = (normalize && c2 > 0.f) ? sqrtf(c2) : 1.f;
    scale[j] = s[j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ell * r; e += blockDim.x) {
    const int j = e % r;
    const float v = raw[e] / s[j];
    Ws[e] = v;
    Wt[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e - p * r;
    float a = 0.f;
    for (int k = 0; k < ell; ++k) a = fmaf(Ws[k * r + p], Ws[k * r + q], a);
    GH[e] = a;
  }
}

// One thread per row i of W: S_W row from X_chk row and H_tld, then the update.
template <int RP, int RULE>
__global__ void __launch_bounds__(128) w_update_kernel(const float* __restrict__ Xchk,
                                                       const float* __restrict__ Ht,
                                                       const float* __restrict__ G, int64_t m,
                                                       int r, int ell, float eps,
                                                       float* __restrict__ W) {
  extern __shared__ float sh[];
  float* HtT = sh;             // [ell][RP]
  float* Gs = HtT + ell * RP;  // [RP][RP]
  for (int e = threadIdx.x; e < ell * RP; e += blockDim.x) {
    const int k = e / RP, j = e - k * RP;
    HtT[e] = (j < r) ? Ht[j * ell + k] : 0.f;
  }
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    const int p = e / RP, q = e - p * RP;
    Gs[e] = (p < r && q < r) ? G[p * r + q] : 0.f;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    float w[RP], s[RP];
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      w[j] = (j < r) ? W[i * r + j] : 0.f;
      s[j] = 0.f;
    }
    const float* xr = Xchk + i * ell;
    for (int k = 0; k < ell; ++k) {
      const float xk = xr[k];
#pragma unroll
      for (int j = 0; j < RP; ++j) s[j] = fmaf(xk, HtT[k * RP + j], s[j]);
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
        float num = posp(s[j]), den = negp(s[j]) + eps;
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const float gq = Gs[q * RP + j];
          num = fmaf(w[q], negp(gq), num);
          den = fmaf(w[q], posp(gq), den);
        }
        wn[j] = w[j] * sqrtf(num / den);
      }
#pragma unroll
      for (int j = 0; j < RP; ++j) w[j] = wn[j];
    }
#pragma unroll
    for (int j = 0; j < RP; ++j)
      if (j < r) W[i * r + j] = w[j];
  }
}

// One thread per column c of H: compensation h_j *= s_j, S_H column from W_tld and X_hat, update.
template <int RP, int RULE>
__global__ void __launch_bounds__(128) h_update_kernel(const float* __restrict__ Xhat,
                                                       const float* __restrict__ Wt,
                                                       const float* __restrict__ GH,
                                                       const float* __restrict__ scale, int64_t n,
                                                       int r, int ell, float alpha, float beta,
                                                       float eps, float* __restrict__ H) {
  extern __shared__ float sh[];
  float* Ws = sh;              // [ell][RP]
  float* Gs = Ws + ell * RP;   // [RP][RP]
  float* sc = Gs + RP * RP;    // [RP]
  for (int e = threadIdx.x; e < ell * RP; e += blockDim.x) {
    const int k = e / RP, j = e - k * RP;
    Ws[e] = (j < r) ? Wt[k * r + j] : 0.f;
  }
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    const int p = e / RP, q = e - p * RP;
    Gs[e] = (p < r && q < r) ? GH[p * r + q] : 0.f;
  }
  for (int j = threadIdx.x; j < RP; j += blockDim.x) sc[j] = (j < r) ? scale[j] : 1.f;
  __syncthreads();
  const bool plain = (alpha == 0.f && beta == 0.f);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    float h[RP], s[RP];
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      h[j] = (j < r) ? H[j * n + c] * sc[j] : 0.f;
      s[j] = 0.f;
    }
    for (int k = 0; k < ell; ++k) {
      const float xk = Xhat[k * n + c];
#pragma unroll
      for (int j = 0; j < RP; ++j) s[j] = fmaf(xk, Ws[k * RP + j], s[j]);
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
        float num = posp(s[j]), den = negp(s[j]) + eps;
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const float gq = Gs[j * RP + q];
          num = fmaf(negp(gq), h[q], num);
          den = fmaf(posp(gq), h[q], den);
        }
        hn[j] = h[j] * sqrtf(num / den);
      }
#pragma unroll
      for (int j = 0; j < RP; ++j) h[j] = hn[j];
    }
#pragma unroll
    for (int j = 0; j < RP; ++j)
      if (j < r) H[j * n + c] = h[j];
  }
}


// Variants for 32 < r <= 64: each thread keeps its row (column) of W (H) and of S in its own
// column of shared memory, so the sweeps need no compile-time unrolling.
constexpr int kGT = 128;   // threads per block of the generic kernels
constexpr int kGR = 64;    // maximum r of the generic kernels

template <int RULE>
__global__ void __launch_bounds__(kGT) w_update_generic_kernel(
    const float* __restrict__ Xchk, const float* __restrict__ Ht, const float* __restrict__ G,
    int64_t m, int r, int ell, float eps, float* __restrict__ W) {
  extern __shared__ float sh[];
  float* HtT = sh;                 // [ell][kGR]
  float* Gs = HtT + ell * kGR;     // [kGR][kGR]
  float* wS = Gs + kGR * kGR;      // [kGR][kGT]
  float* sS = wS + kGR * kGT;      // [kGR][kGT]
  float* nS = sS + kGR * kGT;      // [kGR][kGT]
  const int t = threadIdx.x;
  for (int e = t; e < ell * kGR; e += kGT) {
    const int k = e / kGR, j = e - k * kGR;
    HtT[e] = (j < r) ? Ht[j * ell + k] : 0.f;
  }
  for (int e = t; e < kGR * kGR; e += kGT) {
    const int p = e / kGR, q = e - p * kGR;
    Gs[e] = (p < r && q < r) ? G[p * r + q] : 0.f;
  }
  __syncthreads();
  for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * kGT; i0 < m;
       i0 += static_cast<int64_t>(gridDim.x) * kGT) {
    const int64_t i = i0 + t;
    if (i < m) {
      for (int j = 0; j < r; ++j) {
        wS[j * kGT + t] = W[i * r + j];
        sS[j * kGT + t] = 0.f;
      }
      for (int k = 0; k < ell; ++k) {
        const float xk = Xchk[i * ell + k];
        for (int j = 0; j < r; ++j) sS[j * kGT + t] = fmaf(xk, HtT[k * kGR + j], sS[j * kGT + t]);
      }
      if (RULE == 0) {
        for (int j = 0; j < r; ++j) {
          const float g = Gs[j * kGR + j];
          if (g > 0.f) {
            float tt = sS[j * kGT + t];
            for (int q = 0; q < r; ++q) tt = fmaf(-wS[q * kGT + t], Gs[q * kGR + j], tt);
            wS[j * kGT + t] = fmaxf(0.f, wS[j * kGT + t] + tt / g);
          }
        }
        for (int j = 0; j < r; ++j) W[i * r + j] = wS[j * kGT + t];
      } else {
        for (int j = 0; j < r; ++j) {
          const float sj = sS[j * kGT + t];
          float num = posp(sj), den = negp(sj) + eps;
          for (int q = 0; q < r; ++q) {
            const float gq = Gs[q * kGR + j], wq = wS[q * kGT + t];
            num = fmaf(wq, negp(gq), num);
            den = fmaf(wq, posp(gq), den);
          }
          nS[j * kGT + t] = wS[j * kGT + t] * sqrtf(num / den);
        }
        for (int j = 0; j < r; ++j) W[i * r + j] = nS[j * kGT + t];
      }
    }
  }
}

template <int RULE>
__global__ void __launch_bounds__(kGT) h_update_generic_kernel(
    const float* __restrict__ Xhat, const float* __restrict__ Wt, const float* __restrict__ GH,
    const float* __restrict__ scale, int64_t n, int r, int ell, float alpha, float beta,
    float eps, float* __restrict__ H) {
  extern __shared__ float sh[];
  float* Ws = sh;                  // [ell][kGR]
  float* Gs = Ws + ell * kGR;      // [kGR][kGR]
  float* hS = Gs + kGR * kGR;      // [kGR][kGT]
  float* sS = hS + kGR * kGT;      // [kGR][kGT]
  float* nS = sS + kGR * kGT;      // [kGR][kGT]
  const int t = threadIdx.x;
  for (int e = t; e < ell * kGR; e += kGT) {
    const int k = e / kGR, j = e - k * kGR;
    Ws[e] = (j < r) ? Wt[k * r + j] : 0.f;
  }
  for (int e = t; e < kGR * kGR; e += kGT) {
    const int p = e / kGR, q = e - p * kGR;
    Gs[e] = (p < r && q < r) ? GH[p * r + q] : 0.f;
  }
  __syncthreads();
  const bool plain = (alpha == 0.f && beta == 0.f);
  for (int64_t c0 = static_cast<int64_t>(blockIdx.x) * kGT; c0 < n;
       c0 += static_cast<int64_t>(gridDim.x) * kGT) {
    const int64_t c = c0 + t;
    if (c < n) {
      for (int j = 0; j < r; ++j) {
        hS[j * kGT + t] = H[j * n + c] * scale[j];
        sS[j * kGT + t] = 0.f;
      }
      for (int k = 0; k < ell; ++k) {
        const float xk = Xhat[k * n + c];
        for (int j = 0; j < r; ++j) sS[j * kGT + t] = fmaf(xk, Ws[k * kGR + j], sS[j * kGT + t]);
      }
      if (RULE == 0) {
        for (int j = 0; j < r; ++j) {
          const float g = Gs[j * kGR + j];
          float tt = sS[j * kGT + t];
          for (int q = 0; q < r; ++q) tt = fmaf(-Gs[j * kGR + q], hS[q * kGT + t], tt);
          const float hj = hS[j * kGT + t];
          if (plain) {
            if (g > 0.f) hS[j * kGT + t] = fmaxf(0.f, hj + tt / g);
          } else if (g + beta > 0.f) {
            hS[j * kGT + t] = fmaxf(0.f, (fmaf(hj, g, tt) - alpha) / (g + beta));
          }
        }
        for (int j = 0; j < r; ++j) H[j * n + c] = hS[j * kGT + t];
      } else {
        for (int j = 0; j < r; ++j) {
          const float sj = sS[j * kGT + t];
          float num = posp(sj), den = negp(sj) + eps;
          for (int q = 0; q < r; ++q) {
            const float gq = Gs[j * kGR + q], hq = hS[q * kGT + t];
            num = fmaf(negp(gq), hq, num);
            den = fmaf(posp(gq), hq, den);
          }
          nS[j * kGT + t] = hS[j * kGT + t] * sqrtf(num / den);
        }
        for (int j = 0; j < r; ++j) H[j * n + c] = nS[j * kGT + t];
      }
    }
  }
}

__global__ void scale_w_kernel(float* __restrict__ W, int64_t m, int r,
                               const float* __restrict__ scale) {
  const int64_t total = m * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = static_cast<int>(e % r);
    W[e] /= scale[j];
  }
}

int rp_for(int r) {
  if (r <= 8) return 8;
  if (r <= 16) return 16;
  if (r <= 32) return 32;
  return 64;
}

struct IterWs {
  float *Hpart, *Wpart, *Ht, *G, *Wraw, *Wt, *GH, *scale;
};

IterWs carve(void* ws, int64_t m, int64_t n, int r, int ell) {
  float* p = static_cast<float*>(ws);
  IterWs w;
  w.Hpart = p;
  p += cdiv(n, kSlab) * r * ell;
  w.Wpart = p;
  p += cdiv(m, kSlab) * (ell * r + r);
  w.Ht = p;
  p += r * ell;
  w.G = p;
  p += r * r;
  w.Wraw = p;
  p += ell * r + r;
  w.Wt = p;
  p += ell * r;
  w.GH = p;
  p += r * r;
  w.scale = p;
  return w;
}

unsigned grid_cap(int64_t work, int threads, int cap) {
  const int64_t g = cdiv(work, threads);
  return static_cast<unsigned>(g < 1 ? 1 : (g > cap ? cap : g));
}

// The two row/column update kernels of one configuration (register variant for r <= 32,
// shared-memory variant above).
struct UpdateKernels {
  void (*w)(const float*, const float*, const float*, int64_t, int, int, float, float*);
  void (*h)(const float*, const float*, const float*, const float*, int64_t, int, int, float,
            float, float, float*);
  size_t sh_w, sh_h;
  int threads;
};

template <int RP, int RULE>
UpdateKernels reg_kernels(int ell) {
  return {w_update_kernel<RP, RULE>, h_update_kernel<RP, RULE>,
          sizeof(float) * (ell * RP + RP * RP), sizeof(float) * (ell * RP + RP * RP + RP), 128};
}

template <int RULE>
UpdateKernels generic_kernels(int ell) {
  const size_t sh = sizeof(float) * (ell * kGR + kGR * kGR + 3 * kGR * kGT);
  return {w_update_generic_kernel<RULE>, h_update_generic_kernel<RULE>, sh, sh, kGT};
}

UpdateKernels pick(int r, int ell, int rule) {
  switch (rp_for(r)) {
    case 8: return rule ? reg_kernels<8, 1>(ell) : reg_kernels<8, 0>(ell);
    case 16: return rule ? reg_kernels<16, 1>(ell) : reg_kernels<16, 0>(ell);
    case 32: return rule ? reg_kernels<32, 1>(ell) : reg_kernels<32, 0>(ell);
    default: return rule ? generic_kernels<1>(ell) : generic_kernels<0>(ell);
  }
}

cudaError_t run(const Launcher& L, const IterArgs& a, int iters, void* ws) {
  const IterWs w = carve(ws, a.m, a.n, a.r, a.ell);
  const int r = a.r, ell = a.ell;
  const int64_t nb_n = cdiv(a.n, kSlab), nb_m = cdiv(a.m, kSlab);
  const size_t sh_ht = sizeof(float) * (r * kSlab + kSlab * ell);
  const size_t sh_wt = sizeof(float) * (kSlab * ell + kSlab * r);
  const size_t sh_fin = sizeof(float) * (r + ell * r);
  const UpdateKernels K = pick(r, ell, a.rule);
  cudaError_t err;
  if ((err = cudaFuncSetAttribute(ht_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sh_ht))) != cudaSuccess)
    return err;
  if ((err = cudaFuncSetAttribute(wt_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sh_wt))) != cudaSuccess)
    return err;
  if ((err = cudaFuncSetAttribute(K.w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(K.sh_w))) != cudaSuccess)
    return err;
  if ((err = cudaFuncSetAttribute(K.h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(K.sh_h))) != cudaSuccess)
    return err;
  const int normalize = (a.rule == 0) ? 1 : 0;
  for (int it = 0; it < iters; ++it) {
    // W half-step
    ht_partial_kernel<<<static_cast<unsigned>(nb_n), 256, sh_ht, L.stream>>>(a.H, a.QR, a.n, r,
                                                                             ell, w.Hpart);
    sum_slots_kernel<<<grid_cap(static_cast<int64_t>(r) * ell * 32, 256, 1 << 20), 256, 0,
                       L.stream>>>(w.Hpart, static_cast<int>(nb_n), r * ell, w.Ht);
    gram_rows_kernel<<<1, 256, 0, L.stream>>>(w.Ht, r, ell, w.G);
    K.w<<<grid_cap(a.m, K.threads, 4096), K.threads, K.sh_w, L.stream>>>(a.Xchk, w.Ht, w.G, a.m,
                                                                          r, ell, a.eps, a.W);
    // H half-step
    wt_partial_kernel<<<static_cast<unsigned>(nb_m), 256, sh_wt, L.stream>>>(a.QL, a.W, a.m, r,
                                                                             ell, w.Wpart);
    sum_slots_kernel<<<grid_cap(static_cast<int64_t>(ell * r + r) * 32, 256, 1 << 20), 256, 0,
                       L.stream>>>(w.Wpart, static_cast<int>(nb_m), ell * r + r, w.Wraw);
    finish_wt_kernel<<<1, 256, sh_fin, L.stream>>>(w.Wraw, r, ell, normalize, w.Wt, w.GH,
                                                   w.scale);
    K.h<<<grid_cap(a.n, K.threads, 4096), K.threads, K.sh_h, L.stream>>>(
        a.Xhat, w.Wt, w.GH, w.scale, a.n, r, ell, a.alpha, a.beta, a.eps, a.H);
    L.count(8);
    if (normalize) {
      scale_w_kernel<<<grid_cap(a.m * r, 256, 2048), 256, 0, L.stream>>>(a.W, a.m, r, w.scale);
      L.count();
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace

size_t iterate_ws_bytes(int64_t m, int64_t n, int r, int ell) {
  return sizeof(float) * static_cast<size_t>(cdiv(n, kSlab) * r * ell +
                                             cdiv(m, kSlab) * (ell * r + r) + r * ell + r * r +
                                             ell * r + r + ell * r + r * r + r) + 256;
}

cudaError_t launch_iterate(const Launcher& L, const IterArgs& a, int iters, void* ws,
                           size_t ws_bytes) {
  if (ws_bytes < iterate_ws_bytes(a.m, a.n, a.r, a.ell)) return cudaErrorInvalidValue;
  if (iters <= 0) return cudaSuccess;
  if (a.r > kGR) return cudaErrorInvalidValue;
  return run(L, a, iters, ws);
}

}  // namespace nmfrp
