// Sparse X (CSR) for the sketch, the compression and the residual (Section 5.2 applies the
// methods to a sparse term-frequency matrix). X is m x n with row_ptr (m + 1, int64), col (nnz,
// int32, distinct within a row) and val (nnz, FP32).
//
//   Y = X V   (m x l): one warp a row, lanes over the l columns of V; the row's nonzeros are
//             taken in storage order, so every sum has a fixed order.
//   Z = X^T U (n x l): the same kernel on the transpose in CSC form (column pointers, row indices
//             in increasing row order within a column), built once per matrix.
// CSC build, deterministic: per row block b the nonzeros of each column are counted; a column-
// wise exclusive scan over the blocks and a scan over the columns give each (block, column) its
// first slot; each block then places its rows in order (one warp, the entries of a row in
// parallel: their columns are distinct), so the rows of a column keep their order.
// Residual: ||X - W H||^2 = ||X||^2 - 2 <X, W H> + <W^T W, H H^T>, the first two summed over the
// nonzeros (each x_ic (w_i . h_c), FP64 per lane, one partial per block), the Gram term from the
// two r x r Grams (FP32 within 256-row slabs, FP64 over slabs).
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kSpThreads = 256;     // 8 warps a block, one row a warp
constexpr int kUnroll = 8;          // nonzeros whose gathers a warp issues together
constexpr int kRowsPerBlockCount = 512;
constexpr int kResThreads = 256;
constexpr int kResBlocks = 1024;
constexpr int kSlab = 256;

// Y[i][k] = sum over the nonzeros (c, x) of row i of x * V[c][k], k < ell (<= 128).
template <int KPL>
__global__ void __launch_bounds__(kSpThreads) csr_spmm_kernel(const int64_t* __restrict__ ptr,
                                                              const int* __restrict__ idx,
                                                              const float* __restrict__ val,
                                                              int64_t rows, int ell,
                                                              const float* __restrict__ V,
                                                              float* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kSpThreads + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * kSpThreads) >> 5;
  for (int64_t i = warp; i < rows; i += nw) {
    float acc[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) acc[q] = 0.f;
    const int64_t e0 = ptr[i], e1 = ptr[i + 1];
    for (int64_t b = e0; b < e1; b += 32) {
      // the warp fetches up to 32 nonzeros, then walks them in groups of kUnroll (broadcast by
      // shuffle): the group's gathers of V are issued before its FMAs, so kUnroll rows of V
      // are in flight per lane; the FMAs still run in storage order
      const int64_t e = b + lane;
      const int c = e < e1 ? idx[e] : 0;
      const float x = e < e1 ? val[e] : 0.f;
      const int cnt = static_cast<int>(e1 - b < 32 ? e1 - b : 32);
      for (int t0 = 0; t0 < cnt; t0 += kUnroll) {
        float v[kUnroll][KPL], xs[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int t = t0 + u < cnt ? t0 + u : cnt - 1;   // padded steps reuse a valid index
          const int ct = __shfl_sync(0xffffffffu, c, t);
          xs[u] = t0 + u < cnt ? __shfl_sync(0xffffffffu, x, t) : 0.f;
          const float* vr = V + static_cast<int64_t>(ct) * ell;
#pragma unroll
          for (int q = 0; q < KPL; ++q) {
            const int k = lane + 32 * q;
            v[u][q] = k < ell ? __ldg(vr + k) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
          for (int q = 0; q < KPL; ++q) acc[q] = fmaf(xs[u], v[u][q], acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      const int k = lane + 32 * q;
      if (k < ell) Y[i * ell + k] = acc[q];
    }
  }
}

// counts[b][c] = nonzeros of column c in rows [b R, (b + 1) R) (R = kRowsPerBlockCount).
__global__ void csc_count_kernel(const int64_t* __restrict__ ptr, const int* __restrict__ idx,
                                 int64_t m, int64_t n, int* __restrict__ counts) {
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kRowsPerBlockCount;
  const int64_t r1 = r0 + kRowsPerBlockCount < m ? r0 + kRowsPerBlockCount : m;
  int* cb = counts + static_cast<int64_t>(blockIdx.x) * n;
  for (int64_t e = ptr[r0] + threadIdx.x; e < ptr[r1]; e += blockDim.x) atomicAdd(cb + idx[e], 1);
}

// Per column: base[b][c] = sum over blocks b' < b of counts[b'][c] (in place), total[c].
__global__ void csc_scan_blocks_kernel(int* __restrict__ counts, int nb, int64_t n,
                                       int64_t* __restrict__ total) {
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c < n;
       c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t s = 0;
    for (int b = 0; b < nb; ++b) {
      const int v = counts[static_cast<int64_t>(b) * n + c];
      counts[static_cast<int64_t>(b) * n + c] = static_cast<int>(s);
      s += v;
    }
    total[c] = s;
  }
}

// cptr[c] = sum over c' < c of total[c'] (cptr[n] = nnz): one block, a chunk a thread.
__global__ void __launch_bounds__(1024) csc_scan_cols_kernel(const int64_t* __restrict__ total,
                                                             int64_t n, int64_t* __restrict__ cptr) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t c0 = t * chunk, c1 = c0 + chunk < n ? c0 + chunk : n;
  int64_t s = 0;
  for (int64_t c = c0; c < c1; ++c) s += total[c];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < 1024; ++k) {
      const int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    cptr[n] = run;
  }
  __syncthreads();
  s = part[t];
  for (int64_t c = c0; c < c1; ++c) {
    cptr[c] = s;
    s += total[c];
  }
}

// Block b (one warp) places rows [b R, (b + 1) R) in order: entry (i, c, x) goes to slot
// cptr[c] + base[b][c] + (entries of column c in earlier rows of this block).
__global__ void __launch_bounds__(32) csc_place_kernel(const int64_t* __restrict__ ptr,
                                                       const int* __restrict__ idx,
                                                       const float* __restrict__ val, int64_t m,
                                                       int64_t n, int* __restrict__ base,
                                                       const int64_t* __restrict__ cptr,
                                                       int* __restrict__ crow,
                                                       float* __restrict__ cval) {
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kRowsPerBlockCount;
  const int64_t r1 = r0 + kRowsPerBlockCount < m ? r0 + kRowsPerBlockCount : m;
  int* bb = base + static_cast<int64_t>(blockIdx.x) * n;   // running offsets of this block
  for (int64_t i = r0; i < r1; ++i) {
    for (int64_t e = ptr[i] + threadIdx.x; e < ptr[i + 1]; e += 32) {
      const int c = idx[e];
      const int64_t pos = cptr[c] + bb[c];
      bb[c] += 1;   // columns are distinct within a row: no two lanes share c
      crow[pos] = static_cast<int>(i);
      cval[pos] = val[e];
    }
    __syncwarp();
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per block: sum of x^2 and of x (w_i . h_c) over the nonzeros it takes (HT = H^T, n x r).
__global__ void __launch_bounds__(kResThreads) csr_cross_kernel(
    const int64_t* __restrict__ ptr, const int* __restrict__ idx, const float* __restrict__ val,
    int64_t m, const float* __restrict__ W, const float* __restrict__ HT, int r,
    double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kResThreads + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * kResThreads) >> 5;
  double sx = 0.0, sc = 0.0;
  for (int64_t i = warp; i < m; i += nw) {
    const float* wi = W + i * r;
    for (int64_t e = ptr[i] + lane; e < ptr[i + 1]; e += 32) {
      const float* hc = HT + static_cast<int64_t>(idx[e]) * r;
      float d = 0.f;
      for (int q = 0; q < r; ++q) d = fmaf(__ldg(wi + q), __ldg(hc + q), d);
      const float x = val[e];
      sx = fma(static_cast<double>(x), x, sx);
      sc = fma(static_cast<double>(x), d, sc);
    }
  }
  __shared__ double bx[kResThreads / 32], bc[kResThreads / 32];
  sx = warp_sum_d(sx);
  sc = warp_sum_d(sc);
  if (lane == 0) {
    bx[threadIdx.x >> 5] = sx;
    bc[threadIdx.x >> 5] = sc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kResThreads / 32; ++w) {
      a += bx[w];
      b += bc[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// part[s][p][q] = sum over rows of slab s of A[i][p] A[i][q] (FP32 within the slab).
__global__ void __launch_bounds__(256) slab_gram_kernel(const float* __restrict__ A, int64_t rows,
                                                        int r, double* __restrict__ part) {
  extern __shared__ float as[];   // [kSlab][r]
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kSlab;
  const int nr = static_cast<int>(rows - r0 < kSlab ? rows - r0 : kSlab);
  for (int e = threadIdx.x; e < kSlab * r; e += blockDim.x) as[e] = e < nr * r ? A[r0 * r + e] : 0.f;
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e - p * r;
    float s = 0.f;
    for (int i = 0; i < nr; ++i) s = fmaf(as[i * r + p], as[i * r + q], s);
    part[static_cast<int64_t>(blockIdx.x) * r * r + e] = s;
  }
}

// out[0] = ||X - W H||^2, out[1] = ||X||^2 from the block partials and the two slab Grams.
__global__ void sparse_res_final_kernel(const double* __restrict__ part, int nblocks,
                                        const double* __restrict__ gw, int nsw,
                                        const double* __restrict__ gh, int nsh, int r,
                                        double* __restrict__ out) {
  __shared__ double red[256];
  double q = 0.0;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int s = 0; s < nsw; ++s) a += gw[static_cast<int64_t>(s) * r * r + e];
    for (int s = 0; s < nsh; ++s) b += gh[static_cast<int64_t>(s) * r * r + e];
    q += a * b;
  }
  red[threadIdx.x] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double qq = 0.0;
    for (int t = 0; t < blockDim.x; ++t) qq += red[t];
    double x2 = 0.0, cr = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      x2 += part[2 * b];
      cr += part[2 * b + 1];
    }
    out[0] = x2 - 2.0 * cr + qq;
    out[1] = x2;
  }
}

// H (r x n) -> HT (n x r)
__global__ void transpose_h_kernel(const float* __restrict__ H, int r, int64_t n,
                                   float* __restrict__ HT) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n * r;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = e / r;
    const int j = static_cast<int>(e - c * r);
    HT[e] = H[static_cast<int64_t>(j) * n + c];
  }
}

unsigned grid_for(int64_t work, int per_block, int cap) {
  const int64_t b = cdiv(work, per_block);
  return static_cast<unsigned>(b < cap ? (b > 0 ? b : 1) : cap);
}

cudaError_t spmm(const Launcher& L, const int64_t* ptr, const int* idx, const float* val,
                 int64_t rows, int ell, const float* V, float* Y) {
  const unsigned g = grid_for(rows, kSpThreads / 32, 1 << 16);
  if (ell <= 32) csr_spmm_kernel<1><<<g, kSpThreads, 0, L.stream>>>(ptr, idx, val, rows, ell, V, Y);
  else if (ell <= 64) csr_spmm_kernel<2><<<g, kSpThreads, 0, L.stream>>>(ptr, idx, val, rows, ell, V, Y);
  else csr_spmm_kernel<4><<<g, kSpThreads, 0, L.stream>>>(ptr, idx, val, rows, ell, V, Y);
  L.count();
  return cudaGetLastError();
}

}  // namespace

size_t csc_ws_bytes(int64_t m, int64_t n, int64_t nnz) {
  const int64_t nb = cdiv(m, kRowsPerBlockCount);
  return sizeof(int) * static_cast<size_t>(nb * n) + sizeof(int64_t) * static_cast<size_t>(2 * n + 1) +
         1024;
}

size_t csc_bytes(int64_t n, int64_t nnz) {
  return sizeof(int64_t) * static_cast<size_t>(n + 1) + (sizeof(int) + sizeof(float)) *
         static_cast<size_t>(nnz) + 1024;
}

cudaError_t launch_csc_build(const Launcher& L, const int64_t* ptr, const int* idx,
                             const float* val, int64_t m, int64_t n, int64_t nnz, void* csc,
                             void* ws, size_t ws_bytes, CscView* out) {
  if (ws_bytes < csc_ws_bytes(m, n, nnz)) return cudaErrorInvalidValue;
  const int nb = static_cast<int>(cdiv(m, kRowsPerBlockCount));
  int* counts = static_cast<int*>(ws);
  uintptr_t q = reinterpret_cast<uintptr_t>(counts + static_cast<int64_t>(nb) * n);
  q = (q + 255) & ~uintptr_t(255);
  int64_t* total = reinterpret_cast<int64_t*>(q);
  char* c = static_cast<char*>(csc);
  out->ptr = reinterpret_cast<int64_t*>(c);
  q = reinterpret_cast<uintptr_t>(out->ptr + n + 1);
  q = (q + 255) & ~uintptr_t(255);
  out->idx = reinterpret_cast<int*>(q);
  q = reinterpret_cast<uintptr_t>(out->idx + nnz);
  q = (q + 255) & ~uintptr_t(255);
  out->val = reinterpret_cast<float*>(q);
  cudaError_t err = cudaMemsetAsync(counts, 0, sizeof(int) * static_cast<size_t>(nb) * n, L.stream);
  if (err != cudaSuccess) return err;
  csc_count_kernel<<<nb, 256, 0, L.stream>>>(ptr, idx, m, n, counts);
  csc_scan_blocks_kernel<<<grid_for(n, 256, 4096), 256, 0, L.stream>>>(counts, nb, n, total);
  csc_scan_cols_kernel<<<1, 1024, 0, L.stream>>>(total, n, out->ptr);
  csc_place_kernel<<<nb, 32, 0, L.stream>>>(ptr, idx, val, m, n, counts, out->ptr, out->idx,
                                             out->val);
  L.count(4);
  return cudaGetLastError();
}

cudaError_t launch_csr_dual(const Launcher& L, const CsrView& X, const CscView& XT, int64_t m,
                            int64_t n, int ell, const float* V, const float* U, float* Y,
                            float* Z) {
  if (ell < 1 || ell > 128) return cudaErrorInvalidValue;
  cudaError_t err = cudaSuccess;
  if (V && (err = spmm(L, X.ptr, X.idx, X.val, m, ell, V, Y)) != cudaSuccess) return err;
  if (U && (err = spmm(L, XT.ptr, XT.idx, XT.val, n, ell, U, Z)) != cudaSuccess) return err;
  return cudaSuccess;
}

size_t sparse_residual_ws_bytes(int64_t m, int64_t n, int r) {
  return sizeof(double) * static_cast<size_t>(2 * kResBlocks + (cdiv(m, kSlab) + cdiv(n, kSlab)) * r * r) +
         sizeof(float) * static_cast<size_t>(n * r) + 1024;
}

cudaError_t launch_sparse_residual(const Launcher& L, const CsrView& X, int64_t m, int64_t n,
                                   const float* W, const float* H, int r, double* out2, void* ws,
                                   size_t ws_bytes) {
  if (ws_bytes < sparse_residual_ws_bytes(m, n, r) || r < 1 || r > 128) return cudaErrorInvalidValue;
  double* part = static_cast<double*>(ws);
  const int nsw = static_cast<int>(cdiv(m, kSlab)), nsh = static_cast<int>(cdiv(n, kSlab));
  double* gw = part + 2 * kResBlocks;
  double* gh = gw + static_cast<int64_t>(nsw) * r * r;
  uintptr_t q = reinterpret_cast<uintptr_t>(gh + static_cast<int64_t>(nsh) * r * r);
  q = (q + 255) & ~uintptr_t(255);
  float* HT = reinterpret_cast<float*>(q);
  transpose_h_kernel<<<grid_for(n * r, 256, 8192), 256, 0, L.stream>>>(H, r, n, HT);
  const unsigned nbk = grid_for(m, kResThreads / 32, kResBlocks);
  csr_cross_kernel<<<nbk, kResThreads, 0, L.stream>>>(X.ptr, X.idx, X.val, m, W, HT, r, part);
  const size_t sm = sizeof(float) * kSlab * r;
  cudaError_t err = cudaFuncSetAttribute(slab_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
  if (err != cudaSuccess) return err;
  slab_gram_kernel<<<nsw, 256, sm, L.stream>>>(W, m, r, gw);
  slab_gram_kernel<<<nsh, 256, sm, L.stream>>>(HT, n, r, gh);
  sparse_res_final_kernel<<<1, 256, 0, L.stream>>>(part, static_cast<int>(nbk), gw, nsw, gh, nsh,
                                                   r, out2);
  L.count(5);
  return cudaGetLastError();
}

}  // namespace nmfrp
