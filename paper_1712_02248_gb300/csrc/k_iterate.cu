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

// store(e, load(e)) for e < count over the block, eight loads of a thread issued before their
// stores so that they are in flight together
template <typename Load, typename Store>
__device__ __forceinline__ void batched_copy(int count, Load load, Store store) {
  for (int base = threadIdx.x; base < count; base += 8 * blockDim.x) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * blockDim.x;
      v[u] = (e < count) ? load(e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * blockDim.x;
      if (e < count) store(e, v[u]);
    }
  }
}

// odd row pitch >= w: rows of one table read by 16 or 32 lanes at once fall in distinct banks
__host__ __device__ __forceinline__ int odd_pitch(int w) { return w | 1; }

// The r(r+1)/2 entries p <= q of the r x r Gram of the rows of T (rows of odd pitch P, length
// ell): G[p][q] = G[q][p] = sum_k T[p][k] T[q][k], four partial sums a row pair.
__device__ __forceinline__ void gram_upper(const float* __restrict__ T, int r, int ell, int P,
                                           float* __restrict__ G) {
  const int np = r * (r + 1) / 2;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    int p = 0, rem = e;
    while (rem >= r - p) {
      rem -= r - p;
      ++p;
    }
    const int q = p + rem;
    const float* a = T + p * P;
    const float* b = T + q * P;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int k = 0;
    for (; k + 4 <= ell; k += 4) {
      s0 = fmaf(a[k], b[k], s0);
      s1 = fmaf(a[k + 1], b[k + 1], s1);
      s2 = fmaf(a[k + 2], b[k + 2], s2);
      s3 = fmaf(a[k + 3], b[k + 3], s3);
    }
    for (; k < ell; ++k) s0 = fmaf(a[k], b[k], s0);
    const float v = (s0 + s1) + (s2 + s3);
    G[p * r + q] = v;
    G[q * r + p] = v;
  }
}

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

// The same partials for 32 < r <= 64 from 4 x 4 register tiles of (j, k): the slab of H is
// stored transposed, both tables with rows padded to multiples of 4 floats, so a step over c
// takes two 16-byte shared loads for 16 FMAs. Each (j, k) sums c in the same order as above.
__global__ void __launch_bounds__(256) ht_partial_tiled_kernel(const float* __restrict__ H,
                                                               const float* __restrict__ QR,
                                                               int64_t n, int r, int ell,
                                                               float* __restrict__ Hpart) {
  extern __shared__ __align__(16) float sh[];
  const int RQ = (r + 3) & ~3, LQ = (ell + 3) & ~3;
  float* Hs = sh;                  // [kSlab][RQ]: H^T over the slab, zero beyond r and n
  float* Qs = Hs + kSlab * RQ;     // [kSlab][LQ]: QR rows of the slab, zero beyond ell and n
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kSlab;
  batched_copy(
      RQ * kSlab,
      [&](int e) {
        const int j = e / kSlab, c = e - j * kSlab;
        return (j < r && c0 + c < n) ? H[j * n + c0 + c] : 0.f;
      },
      [&](int e, float v) {
        const int j = e / kSlab, c = e - j * kSlab;
        Hs[c * RQ + j] = v;
      });
  batched_copy(
      kSlab * LQ,
      [&](int e) {
        const int c = e / LQ, k = e - c * LQ;
        return (k < ell && c0 + c < n) ? QR[(c0 + c) * ell + k] : 0.f;
      },
      [&](int e, float v) { Qs[e] = v; });
  __syncthreads();
  const int JT = RQ / 4, KT = LQ / 4;
  float* out = Hpart + static_cast<int64_t>(blockIdx.x) * r * ell;
  for (int tile = threadIdx.x; tile < JT * KT; tile += blockDim.x) {
    const int jt = tile / KT, kt = tile - jt * KT;
    const float4* h4 = reinterpret_cast<const float4*>(Hs) + jt;
    const float4* q4 = reinterpret_cast<const float4*>(Qs) + kt;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
    for (int c = 0; c < kSlab; ++c) {
      const float4 hv = h4[c * JT], qv = q4[c * KT];
      const float hj[4] = {hv.x, hv.y, hv.z, hv.w}, qk[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(hj[a], qk[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = 4 * jt + a, k = 4 * kt + b;
        if (j < r && k < ell) out[j * ell + k] = acc[a][b];
      }
  }
}

// The same partials for 32 < r <= 64 from 4 x 4 register tiles of (k, j), plus one tile row
// for the sums of squares; each entry sums i in the same order as the scalar kernel.
__global__ void __launch_bounds__(256) wt_partial_tiled_kernel(const float* __restrict__ QL,
                                                               const float* __restrict__ W,
                                                               int64_t m, int r, int ell,
                                                               float* __restrict__ Wpart) {
  extern __shared__ __align__(16) float sh[];
  const int RQ = (r + 3) & ~3, LQ = (ell + 3) & ~3;
  float* Qs = sh;                  // [kSlab][LQ]: QL rows of the slab, zero beyond ell and m
  float* Ws = Qs + kSlab * LQ;     // [kSlab][RQ]: W rows of the slab, zero beyond r and m
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kSlab;
  batched_copy(
      kSlab * LQ,
      [&](int e) {
        const int i = e / LQ, k = e - i * LQ;
        return (k < ell && i0 + i < m) ? QL[(i0 + i) * ell + k] : 0.f;
      },
      [&](int e, float v) { Qs[e] = v; });
  batched_copy(
      kSlab * RQ,
      [&](int e) {
        const int i = e / RQ, j = e - i * RQ;
        return (j < r && i0 + i < m) ? W[(i0 + i) * r + j] : 0.f;
      },
      [&](int e, float v) { Ws[e] = v; });
  __syncthreads();
  const int JT = RQ / 4, KT = LQ / 4;
  float* out = Wpart + static_cast<int64_t>(blockIdx.x) * (ell * r + r);
  for (int tile = threadIdx.x; tile < KT * JT + JT; tile += blockDim.x) {
    if (tile < KT * JT) {
      const int kt = tile / JT, jt = tile - kt * JT;
      const float4* q4 = reinterpret_cast<const float4*>(Qs) + kt;
      const float4* w4 = reinterpret_cast<const float4*>(Ws) + jt;
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
      for (int i = 0; i < kSlab; ++i) {
        const float4 qv = q4[i * KT], wv = w4[i * JT];
        const float qk[4] = {qv.x, qv.y, qv.z, qv.w}, wj[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(qk[a], wj[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int k = 4 * kt + a, j = 4 * jt + b;
          if (k < ell && j < r) out[k * r + j] = acc[a][b];
        }
    } else {
      const int jt = tile - KT * JT;
      const float4* w4 = reinterpret_cast<const float4*>(Ws) + jt;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
      for (int i = 0; i < kSlab; ++i) {
        const float4 wv = w4[i * JT];
        acc[0] = fmaf(wv.x, wv.x, acc[0]);
        acc[1] = fmaf(wv.y, wv.y, acc[1]);
        acc[2] = fmaf(wv.z, wv.z, acc[2]);
        acc[3] = fmaf(wv.w, wv.w, acc[3]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * jt + b < r) out[ell * r + 4 * jt + b] = acc[b];
    }
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

// G_W = H_tld H_tld^T (r x r) from H_tld (r x ell); one block, rows staged in shared memory.
__global__ void __launch_bounds__(512) gram_rows_kernel(const float* __restrict__ Ht, int r,
                                                        int ell, float* __restrict__ G) {
  extern __shared__ float hs[];   // [r][odd_pitch(ell)]
  const int P = odd_pitch(ell);
  batched_copy(r * ell, [&](int e) { return Ht[e]; },
               [&](int e, float v) { hs[(e / ell) * P + e % ell] = v; });
  __syncthreads();
  gram_upper(hs, r, ell, P, G);
}

// From raw W_tld (ell x r) and column sums of squares: scale s_j (= ||w_j|| or 1),
// W_tld[:,j] /= s_j, G_H = W_tld^T W_tld. One block; W_tld^T staged in shared memory.
__global__ void __launch_bounds__(512) finish_wt_kernel(const float* __restrict__ raw, int r,
                                                        int ell, int normalize,
                                                        float* __restrict__ Wt,
                                                        float* __restrict__ GH,
                                                        float* __restrict__ scale) {
  extern __shared__ float sh[];
  const int P = odd_pitch(ell);
  float* s = sh;          // [r]
  float* WsT = s + r;     // [r][P]: W_tld^T
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    const float c2 = raw[ell * r + j];
    s[j] = (normalize && c2 > 0.f) ? sqrtf(c2) : 1.f;
    scale[j] = s[j];
  }
  __syncthreads();
  batched_copy(ell * r, [&](int e) { return raw[e]; }, [&](int e, float v) {
    const int k = e / r, j = e - k * r;
    const float x = v / s[j];
    WsT[j * P + k] = x;
    Wt[e] = x;
  });
  __syncthreads();
  gram_upper(WsT, r, ell, P, GH);
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


// Variants for 32 < r <= 64: a group of four adjacent lanes takes two rows of W (columns of H);
// lane quarter q keeps entries j = 16 q .. 16 q + 15 of both rows (columns) and of their S in
// registers, so every table value read from shared memory feeds two FMAs. Step j of the
// Gauss-Seidel sweep sums G[j][q'] h_q' over each quarter and adds the four quarters by two
// shuffles; the lane holding j applies the update. G is symmetric, so row j serves both sides.
// The shared tables keep quarter q of a row at offset 20 q (row pitch 80): the four 16-byte
// loads of one instruction then fall in distinct banks.
constexpr int kQT = 128;   // threads per block of the quad kernels (64 rows or columns a pass)
constexpr int kQR = 64;    // maximum r of the quad kernels
constexpr int kQP = 80;    // row pitch of the shared tables

__device__ __forceinline__ float quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

// this lane's quarter of sum_q g[q] a[q] and sum_q g[q] b[q] (g: 16 floats, 16-byte aligned)
__device__ __forceinline__ void quarter_dot2(const float* __restrict__ g, const float (&a)[16],
                                             const float (&b)[16], float& da, float& db) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float4 x = g4[u];
    a0 = fmaf(x.x, a[4 * u], a0);
    b0 = fmaf(x.x, b[4 * u], b0);
    a1 = fmaf(x.y, a[4 * u + 1], a1);
    b1 = fmaf(x.y, b[4 * u + 1], b1);
    a0 = fmaf(x.z, a[4 * u + 2], a0);
    b0 = fmaf(x.z, b[4 * u + 2], b0);
    a1 = fmaf(x.w, a[4 * u + 3], a1);
    b1 = fmaf(x.w, b[4 * u + 3], b1);
  }
  da = a0 + a1;
  db = b0 + b1;
}

// MU: this lane's quarter of sum_q G-[j][q] v_q (num) and sum_q G+[j][q] v_q (den) for one row
__device__ __forceinline__ void quarter_mu(const float* __restrict__ g, const float (&v)[16],
                                           float& num, float& den) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float n0 = 0.f, n1 = 0.f, d0 = 0.f, d1 = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float4 x = g4[u];
    n0 = fmaf(negp(x.x), v[4 * u], n0);
    d0 = fmaf(posp(x.x), v[4 * u], d0);
    n1 = fmaf(negp(x.y), v[4 * u + 1], n1);
    d1 = fmaf(posp(x.y), v[4 * u + 1], d1);
    n0 = fmaf(negp(x.z), v[4 * u + 2], n0);
    d0 = fmaf(posp(x.z), v[4 * u + 2], d0);
    n1 = fmaf(negp(x.w), v[4 * u + 3], n1);
    d1 = fmaf(posp(x.w), v[4 * u + 3], d1);
  }
  num = n0 + n1;
  den = d0 + d1;
}

// sa += xa tab, sb += xb tab over this lane's 16 entries of a shared row (16-byte aligned)
__device__ __forceinline__ void axpy16x2(float xa, float xb, const float* __restrict__ tab,
                                         float (&sa)[16], float (&sb)[16]) {
  const float4* t4 = reinterpret_cast<const float4*>(tab);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float4 v = t4[u];
    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      sa[4 * u + e] = fmaf(xa, x[e], sa[4 * u + e]);
      sb[4 * u + e] = fmaf(xb, x[e], sb[4 * u + e]);
    }
  }
}

// tab[k][20 (j / 16) + j % 16] = src(k, j) for j < r, 0 elsewhere (pads included), k < rows;
// the loads are batched (a block fills ~10^4 entries from L2 before its first pass)
template <typename Src>
__device__ __forceinline__ void fill_quarter_table(float* __restrict__ tab, int rows, int r,
                                                   Src src) {
  batched_copy(
      rows * kQP,
      [&](int e) {
        const int k = e / kQP, pos = e - k * kQP;
        const int quarter = pos / 20, within = pos - quarter * 20;
        const int j = quarter * 16 + within;
        return (within < 16 && j < r) ? src(k, j) : 0.f;
      },
      [&](int e, float v) { tab[e] = v; });
}

template <int RULE>
__global__ void __launch_bounds__(kQT) w_update_quad_kernel(
    const float* __restrict__ Xchk, const float* __restrict__ Ht, const float* __restrict__ G,
    int64_t m, int r, int ell, float eps, float* __restrict__ W) {
  extern __shared__ __align__(16) float sh[];
  float* HtT = sh;                 // [ell][kQP]: H_tld^T by quarters
  float* Gs = HtT + ell * kQP;     // [kQR][kQP]: G_W by quarters
  float* Xs = Gs + kQR * kQP;      // [kQT / 2][odd_pitch(ell)]: the pass's rows of X_chk
  const int XP = odd_pitch(ell);
  fill_quarter_table(HtT, ell, r, [&](int k, int j) { return Ht[j * ell + k]; });
  fill_quarter_table(Gs, kQR, r, [&](int p, int q) { return p < r ? G[p * r + q] : 0.f; });
  const int t = threadIdx.x, q = t & 3, g = t >> 2, j0 = q * 16;
  for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * (kQT / 2); i0 < m;
       i0 += static_cast<int64_t>(gridDim.x) * (kQT / 2)) {
    // every lane stays in the loop (the shuffles); rows past m work on zeros and store nothing
    const int64_t ia = i0 + g, ib = i0 + 32 + g;
    const bool la = ia < m, lb = ib < m;
    __syncthreads();   // the tables are filled; the previous pass is done with Xs
    const int64_t xoff = i0 * ell, xend = m * ell;
    batched_copy(
        (kQT / 2) * ell,
        [&](int e) { return xoff + e < xend ? Xchk[xoff + e] : 0.f; },
        [&](int e, float v) { Xs[(e / ell) * XP + e % ell] = v; });
    __syncthreads();
    float wa[16], wb[16], sa[16], sb[16];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const bool in = j0 + jj < r;
      wa[jj] = (la && in) ? W[ia * r + j0 + jj] : 0.f;
      wb[jj] = (lb && in) ? W[ib * r + j0 + jj] : 0.f;
      sa[jj] = 0.f;
      sb[jj] = 0.f;
    }
#pragma unroll 2
    for (int k = 0; k < ell; ++k)
      axpy16x2(Xs[g * XP + k], Xs[(g + 32) * XP + k], HtT + k * kQP + q * 20, sa, sb);
    // the sweep runs over the quarters (a loop) and their 16 entries (unrolled, so that the
    // register arrays take fixed indices): a fully unrolled 64-step sweep overruns the
    // instruction cache
    if (RULE == 0) {
      for (int jq = 0; jq * 16 < r; ++jq) {
        const bool own = (q == jq);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = jq * 16 + jj;
          if (j >= r) break;
          float da, db;
          quarter_dot2(Gs + j * kQP + q * 20, wa, wb, da, db);
          da = quad_sum(da);
          db = quad_sum(db);
          const float gj = Gs[j * kQP + jq * 20 + jj];
          if (own && gj > 0.f) {
            wa[jj] = fmaxf(0.f, wa[jj] + (sa[jj] - da) / gj);
            wb[jj] = fmaxf(0.f, wb[jj] + (sb[jj] - db) / gj);
          }
        }
      }
    } else {
      float na[16], nb[16];
      for (int jq = 0; jq * 16 < r; ++jq) {
        const bool own = (q == jq);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = jq * 16 + jj;
          if (j >= r) break;
          float nua, dea, nub, deb;
          quarter_mu(Gs + j * kQP + q * 20, wa, nua, dea);
          quarter_mu(Gs + j * kQP + q * 20, wb, nub, deb);
          nua = quad_sum(nua);
          dea = quad_sum(dea);
          nub = quad_sum(nub);
          deb = quad_sum(deb);
          if (own) {
            const float xa = sa[jj], xb = sb[jj];
            na[jj] = wa[jj] * sqrtf((posp(xa) + nua) / (negp(xa) + dea + eps));
            nb[jj] = wb[jj] * sqrtf((posp(xb) + nub) / (negp(xb) + deb + eps));
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        wa[jj] = na[jj];
        wb[jj] = nb[jj];
      }
    }
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      if (j0 + jj < r) {
        if (la) W[ia * r + j0 + jj] = wa[jj];
        if (lb) W[ib * r + j0 + jj] = wb[jj];
      }
    }
  }
}

template <int RULE>
__global__ void __launch_bounds__(kQT) h_update_quad_kernel(
    const float* __restrict__ Xhat, const float* __restrict__ Wt, const float* __restrict__ GH,
    const float* __restrict__ scale, int64_t n, int r, int ell, float alpha, float beta,
    float eps, float* __restrict__ H) {
  extern __shared__ __align__(16) float sh[];
  float* Ws = sh;                  // [ell][kQP]: W_tld by quarters
  float* Gs = Ws + ell * kQP;      // [kQR][kQP]: G_H by quarters
  float* sc = Gs + kQR * kQP;      // [kQR]
  float* Xs = sc + kQR;            // [ell][kQT / 2]: the pass's columns of X_hat
  fill_quarter_table(Ws, ell, r, [&](int k, int j) { return Wt[k * r + j]; });
  fill_quarter_table(Gs, kQR, r, [&](int p, int q) { return p < r ? GH[p * r + q] : 0.f; });
  for (int j = threadIdx.x; j < kQR; j += kQT) sc[j] = (j < r) ? scale[j] : 1.f;
  const bool plain = (alpha == 0.f && beta == 0.f);
  const int t = threadIdx.x, q = t & 3, g = t >> 2, j0 = q * 16;
  for (int64_t c0 = static_cast<int64_t>(blockIdx.x) * (kQT / 2); c0 < n;
       c0 += static_cast<int64_t>(gridDim.x) * (kQT / 2)) {
    const int64_t ca = c0 + g, cb = c0 + 32 + g;
    const bool la = ca < n, lb = cb < n;
    __syncthreads();   // the tables are filled; the previous pass is done with Xs
    batched_copy(
        ell * (kQT / 2),
        [&](int e) {
          const int64_t cc = c0 + (e & (kQT / 2 - 1));
          return cc < n ? Xhat[static_cast<int64_t>(e / (kQT / 2)) * n + cc] : 0.f;
        },
        [&](int e, float v) { Xs[e] = v; });
    __syncthreads();
    float ha[16], hb[16], sa[16], sb[16];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int j = j0 + jj;
      const bool in = j < r;
      ha[jj] = (la && in) ? H[j * n + ca] * sc[j] : 0.f;
      hb[jj] = (lb && in) ? H[j * n + cb] * sc[j] : 0.f;
      sa[jj] = 0.f;
      sb[jj] = 0.f;
    }
#pragma unroll 2
    for (int k = 0; k < ell; ++k)
      axpy16x2(Xs[k * (kQT / 2) + g], Xs[k * (kQT / 2) + 32 + g], Ws + k * kQP + q * 20, sa, sb);
    if (RULE == 0) {
      for (int jq = 0; jq * 16 < r; ++jq) {
        const bool own = (q == jq);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = jq * 16 + jj;
          if (j >= r) break;
          float da, db;
          quarter_dot2(Gs + j * kQP + q * 20, ha, hb, da, db);
          da = quad_sum(da);
          db = quad_sum(db);
          const float gj = Gs[j * kQP + jq * 20 + jj];
          if (own) {
            const float ta = sa[jj] - da, tb = sb[jj] - db;
            const float xa = ha[jj], xb = hb[jj];
            if (plain) {
              if (gj > 0.f) {
                ha[jj] = fmaxf(0.f, xa + ta / gj);
                hb[jj] = fmaxf(0.f, xb + tb / gj);
              }
            } else if (gj + beta > 0.f) {
              ha[jj] = fmaxf(0.f, (fmaf(xa, gj, ta) - alpha) / (gj + beta));
              hb[jj] = fmaxf(0.f, (fmaf(xb, gj, tb) - alpha) / (gj + beta));
            }
          }
        }
      }
    } else {
      float na[16], nb[16];
      for (int jq = 0; jq * 16 < r; ++jq) {
        const bool own = (q == jq);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = jq * 16 + jj;
          if (j >= r) break;
          float nua, dea, nub, deb;
          quarter_mu(Gs + j * kQP + q * 20, ha, nua, dea);
          quarter_mu(Gs + j * kQP + q * 20, hb, nub, deb);
          nua = quad_sum(nua);
          dea = quad_sum(dea);
          nub = quad_sum(nub);
          deb = quad_sum(deb);
          if (own) {
            const float xa = sa[jj], xb = sb[jj];
            na[jj] = ha[jj] * sqrtf((posp(xa) + nua) / (negp(xa) + dea + eps));
            nb[jj] = hb[jj] * sqrtf((posp(xb) + nub) / (negp(xb) + deb + eps));
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        ha[jj] = na[jj];
        hb[jj] = nb[jj];
      }
    }
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int j = j0 + jj;
      if (j < r) {
        if (la) H[j * n + ca] = ha[jj];
        if (lb) H[j * n + cb] = hb[jj];
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
  int rows;   // rows of W (columns of H) a block takes per pass
};

template <int RP, int RULE>
UpdateKernels reg_kernels(int ell) {
  return {w_update_kernel<RP, RULE>, h_update_kernel<RP, RULE>,
          sizeof(float) * (ell * RP + RP * RP), sizeof(float) * (ell * RP + RP * RP + RP), 128,
          128};
}

template <int RULE>
UpdateKernels quad_kernels(int ell) {
  return {w_update_quad_kernel<RULE>, h_update_quad_kernel<RULE>,
          sizeof(float) * (ell * kQP + kQR * kQP + (kQT / 2) * odd_pitch(ell)),
          sizeof(float) * (ell * kQP + kQR * kQP + kQR + ell * (kQT / 2)), kQT, kQT / 2};
}

UpdateKernels pick(int r, int ell, int rule) {
  switch (rp_for(r)) {
    case 8: return rule ? reg_kernels<8, 1>(ell) : reg_kernels<8, 0>(ell);
    case 16: return rule ? reg_kernels<16, 1>(ell) : reg_kernels<16, 0>(ell);
    case 32: return rule ? reg_kernels<32, 1>(ell) : reg_kernels<32, 0>(ell);
    default: return rule ? quad_kernels<1>(ell) : quad_kernels<0>(ell);
  }
}

cudaError_t run(const Launcher& L, const IterArgs& a, int iters, void* ws) {
  const IterWs w = carve(ws, a.m, a.n, a.r, a.ell);
  const int r = a.r, ell = a.ell;
  const int64_t nb_n = cdiv(a.n, kSlab), nb_m = cdiv(a.m, kSlab);
  const bool tiled = r > 32;   // the quad kernels' range
  const size_t sh_ht = tiled ? sizeof(float) * kSlab * (((r + 3) & ~3) + ((ell + 3) & ~3))
                             : sizeof(float) * (r * kSlab + kSlab * ell);
  void (*ht_k)(const float*, const float*, int64_t, int, int, float*) =
      tiled ? ht_partial_tiled_kernel : ht_partial_kernel;
  const size_t sh_wt = tiled ? sizeof(float) * kSlab * (((r + 3) & ~3) + ((ell + 3) & ~3))
                             : sizeof(float) * (kSlab * ell + kSlab * r);
  void (*wt_k)(const float*, const float*, int64_t, int, int, float*) =
      tiled ? wt_partial_tiled_kernel : wt_partial_kernel;
  const size_t sh_fin = sizeof(float) * (r + r * odd_pitch(ell));
  const size_t sh_gram = sizeof(float) * r * odd_pitch(ell);
  const UpdateKernels K = pick(r, ell, a.rule);
  cudaError_t err;
  if ((err = cudaFuncSetAttribute(ht_k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sh_ht))) != cudaSuccess)
    return err;
  if ((err = cudaFuncSetAttribute(wt_k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sh_wt))) != cudaSuccess)
    return err;
  if ((err = cudaFuncSetAttribute(K.w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(K.sh_w))) != cudaSuccess)
    return err;
  if ((err = cudaFuncSetAttribute(K.h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(K.sh_h))) != cudaSuccess)
    return err;
  // update grids: one wave of resident blocks at most, so that a block fills its shared tables
  // once for several passes
  int dev = 0, sms = 0, occ_w = 0, occ_h = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return err;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, K.w, K.threads, K.sh_w)) !=
      cudaSuccess)
    return err;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_h, K.h, K.threads, K.sh_h)) !=
      cudaSuccess)
    return err;
  const unsigned grid_w = grid_cap(a.m, K.rows, (occ_w > 0 ? occ_w : 1) * sms);
  const unsigned grid_h = grid_cap(a.n, K.rows, (occ_h > 0 ? occ_h : 1) * sms);
  const int normalize = (a.rule == 0) ? 1 : 0;
  for (int it = 0; it < iters; ++it) {
    // W half-step
    ht_k<<<static_cast<unsigned>(nb_n), 256, sh_ht, L.stream>>>(a.H, a.QR, a.n, r, ell, w.Hpart);
    sum_slots_kernel<<<grid_cap(static_cast<int64_t>(r) * ell * 32, 256, 1 << 20), 256, 0,
                       L.stream>>>(w.Hpart, static_cast<int>(nb_n), r * ell, w.Ht);
    gram_rows_kernel<<<1, 512, sh_gram, L.stream>>>(w.Ht, r, ell, w.G);
    K.w<<<grid_w, K.threads, K.sh_w, L.stream>>>(a.Xchk, w.Ht, w.G, a.m,
                                                                          r, ell, a.eps, a.W);
    // H half-step
    wt_k<<<static_cast<unsigned>(nb_m), 256, sh_wt, L.stream>>>(a.QL, a.W, a.m, r, ell, w.Wpart);
    sum_slots_kernel<<<grid_cap(static_cast<int64_t>(ell * r + r) * 32, 256, 1 << 20), 256, 0,
                       L.stream>>>(w.Wpart, static_cast<int>(nb_m), ell * r + r, w.Wraw);
    finish_wt_kernel<<<1, 512, sh_fin, L.stream>>>(w.Wraw, r, ell, normalize, w.Wt, w.GH,
                                                   w.scale);
    K.h<<<grid_h, K.threads, K.sh_h, L.stream>>>(
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
  if (a.r > kQR) return cudaErrorInvalidValue;
  return run(L, a, iters, ws);
}

}  // namespace nmfrp
