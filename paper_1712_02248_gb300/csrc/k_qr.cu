// Thin QR of tall FP32 matrices (Section 3, Eq. 3.4-3.5: Q from the QR decomposition of the
// sketch) by CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa & Yamamoto 2014): twice
//   G = Y^T Y,  G = R^T R (Cholesky),  Y <- Y R^{-1}.
//
// Precision. Sweep 1 sees cond(G) = cond(Y)^2, so its Gram matrix is accumulated in float-float
// arithmetic (error-free products by FMA and Knuth's TwoSum; about 48 significant bits, relative
// error near 1e-12 over a 128-row slab) and summed across slabs in FP64; its Cholesky factor and
// R^{-1} are formed in float-float too (an l x l problem, ~44 bits) and R^{-1} is applied in
// float-float, since its entries reach cond(Y) and their products cancel. The FP64 pipe of this
// GPU runs at 1/58 of the FP32 rate (a warp-wide FP64 instruction holds its scheduler's FP64
// pipe for ~67 cycles), so everything runs on the FP32 pipes. Sweep 2 starts from a nearly
// orthonormal matrix: its Gram and factor are float-float as well, its application FP32. The
// result is the Q of the QR factorisation whose R has a positive diagonal.
//
// Up to two independent matrices (the two chains of the sketch) go through each kernel in one
// launch: blockIdx.y (blockIdx.x for the Cholesky) selects the matrix.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kGramRows = 128;   // rows per Gram block
constexpr int kGramThreads = 256;
constexpr int kMaxMats = 2;

struct QrBatch {
  const float* Y[kMaxMats];     // inputs of this sweep
  float* Q[kMaxMats];           // outputs of this sweep
  int64_t rows[kMaxMats];
  int64_t part_off[kMaxMats];   // first Gram-partial slot of each matrix
  int nmat;
};

// hi + lo += a * b with an error-free product and Knuth's TwoSum on the running sum.
__device__ __forceinline__ void ff_fma(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float v = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// Partial Gram of a 128-row slab in float-float: Gp[slot][p][q] (FP64) for p <= q.
template <int LP>
__global__ void __launch_bounds__(kGramThreads) gram_partial_kernel(QrBatch b, int ell,
                                                                    double* __restrict__ Gp) {
  extern __shared__ __align__(16) float Ysm[];   // [kGramRows][LP]
  const int mat = blockIdx.y;
  if (mat >= b.nmat) return;
  const int64_t rows = b.rows[mat];
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kGramRows;
  if (r0 >= rows) return;
  const float* Y = b.Y[mat];
  const int t = threadIdx.x;
  for (int e = t; e < kGramRows * LP; e += kGramThreads) {
    const int i = e / LP, k = e - i * LP;
    const int64_t gr = r0 + i;
    Ysm[e] = (gr < rows && k < ell) ? Y[gr * ell + k] : 0.f;
  }
  __syncthreads();
  constexpr int T2 = LP / 2;
  double* out = Gp + (b.part_off[mat] + blockIdx.x) * LP * LP;
  // upper-triangle tiles only: tile u -> (P, Qi) with P <= Qi, row P holding T2 - P tiles
  for (int tile = t; tile < T2 * (T2 + 1) / 2; tile += kGramThreads) {
    int P = 0, u = tile;
    while (u >= T2 - P) {
      u -= T2 - P;
      ++P;
    }
    const int Qi = P + u;
    float h00 = 0, h01 = 0, h10 = 0, h11 = 0, l00 = 0, l01 = 0, l10 = 0, l11 = 0;
#pragma unroll 4
    for (int i = 0; i < kGramRows; ++i) {
      const float2 a = *reinterpret_cast<const float2*>(&Ysm[i * LP + 2 * P]);
      const float2 c = *reinterpret_cast<const float2*>(&Ysm[i * LP + 2 * Qi]);
      ff_fma(a.x, c.x, h00, l00);
      ff_fma(a.x, c.y, h01, l01);
      ff_fma(a.y, c.x, h10, l10);
      ff_fma(a.y, c.y, h11, l11);
    }
    out[(2 * P) * LP + 2 * Qi] = static_cast<double>(h00) + static_cast<double>(l00);
    out[(2 * P) * LP + 2 * Qi + 1] = static_cast<double>(h01) + static_cast<double>(l01);
    out[(2 * P + 1) * LP + 2 * Qi] = static_cast<double>(h10) + static_cast<double>(l10);
    out[(2 * P + 1) * LP + 2 * Qi + 1] = static_cast<double>(h11) + static_cast<double>(l11);
  }
}

// G[mat][e] = sum over the matrix's slabs of Gp[slot][e]: one warp per entry, lanes stride the
// slabs, then a fixed shuffle tree (deterministic).
__global__ void sum_parts_kernel(const double* __restrict__ Gp, QrBatch b, int entries,
                                 double* __restrict__ G) {
  const int mat = blockIdx.y;
  if (mat >= b.nmat) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= entries) return;
  const int64_t nparts = cdiv(b.rows[mat], kGramRows);
  const double* base = Gp + b.part_off[mat] * entries;
  double s = 0.0;
  for (int64_t k = lane; k < nparts; k += 32) s += base[k * entries + warp];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) G[mat * entries + warp] = s;
}

// ---- float-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2; about 44 significant
// bits): Knuth's TwoSum, the FMA-based exact product, and Newton-corrected square root and
// reciprocal. Used for the l x l Cholesky factor and its inverse, which need more than FP32 when
// the sketch is ill-conditioned; the FP64 pipe of this GPU runs at 1/58 of the FP32 rate.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_quick(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  FF s = ff_two_sum(x.hi, y.hi);
  const FF t = ff_two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = ff_quick(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return ff_quick(s.hi, s.lo);
}
__device__ __forceinline__ FF ff_neg(FF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return ff_quick(p, e);
}
// 1 / x: FP32 estimate, one Newton step in float-float (r + r (1 - x r))
__device__ __forceinline__ FF ff_recip(FF x) {
  const float r = __frcp_rn(x.hi);
  const FF e = ff_add({1.f, 0.f}, ff_neg(ff_mul(x, {r, 0.f})));
  return ff_add({r, 0.f}, ff_mul({r, 0.f}, e));
}
// sqrt(x): FP32 estimate q, one correction (x - q^2) / (2 q)
__device__ __forceinline__ FF ff_sqrt(FF x) {
  const float q = __fsqrt_rn(x.hi);
  const FF d = ff_add(x, ff_neg(ff_mul({q, 0.f}, {q, 0.f})));
  return ff_quick(q, __fdiv_rn(d.hi, __fmul_rn(2.f, q)));
}

// One block per matrix: Cholesky G = R^T R in float-float (in place on the upper triangle; G
// arrives in FP64), then T = R^{-1} by back substitution, one column per thread (T[k][c] for
// k < c kept transposed in the lower triangle), four partial sums a column for latency. Writes T
// as T_hi + T_lo (two FP32 arrays, ell x ell row-major).
template <int LP>
__global__ void __launch_bounds__(256) chol_inv_ff_kernel(const double* __restrict__ Gin,
                                                          QrBatch b, int ell,
                                                          float* __restrict__ Thi,
                                                          float* __restrict__ Tlo, int* status) {
  constexpr int S = LP + 1;
  extern __shared__ __align__(16) float chol_ff_sm[];
  float* Ah = chol_ff_sm;         // [LP][S]
  float* Al = Ah + LP * S;        // [LP][S]
  float* dh = Al + LP * S;        // [LP]  1 / R[j][j]
  float* dl = dh + LP;
  __shared__ int bad;
  const int mat = blockIdx.x;
  if (mat >= b.nmat) return;
  const double* G = Gin + static_cast<int64_t>(mat) * LP * LP;
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) bad = 0;
  for (int p = t >> 5; p < LP; p += nt >> 5)
    for (int q = t & 31; q < LP; q += 32) {
      const double g = (p <= q && q < ell) ? G[p * LP + q] : 0.0;
      const float hi = static_cast<float>(g);
      Ah[p * S + q] = hi;
      Al[p * S + q] = static_cast<float>(g - static_cast<double>(hi));
    }
  __syncthreads();
  for (int j = 0; j < ell; ++j) {
    if (t == 0) {
      FF d = {Ah[j * S + j], Al[j * S + j]};
      // a non-positive pivot: the sketch is numerically rank deficient
      if (!(d.hi > 0.f)) {
        bad = 1;
        d = {1e-30f, 0.f};
      }
      const FF r = ff_sqrt(d);
      const FF ri = ff_recip(r);
      Ah[j * S + j] = r.hi;
      Al[j * S + j] = r.lo;
      dh[j] = ri.hi;
      dl[j] = ri.lo;
    }
    __syncthreads();
    const FF ri = {dh[j], dl[j]};
    for (int q = j + 1 + t; q < ell; q += nt) {
      const FF v = ff_mul({Ah[j * S + q], Al[j * S + q]}, ri);
      Ah[j * S + q] = v.hi;
      Al[j * S + q] = v.lo;
    }
    __syncthreads();
    for (int p = j + 1 + (t >> 5); p < ell; p += nt >> 5) {
      const FF ajp = {Ah[j * S + p], Al[j * S + p]};
      for (int q = p + (t & 31); q < ell; q += 32) {
        const FF v = ff_add({Ah[p * S + q], Al[p * S + q]},
                            ff_neg(ff_mul(ajp, {Ah[j * S + q], Al[j * S + q]})));
        Ah[p * S + q] = v.hi;
        Al[p * S + q] = v.lo;
      }
    }
    __syncthreads();
  }
  // T[c][c] = 1 / R[c][c];  T[i][c] = -(sum_{k=i+1..c} R[i][k] T[k][c]) / R[i][i]
  for (int c = t; c < ell; c += nt) {
    const FF tcc = {dh[c], dl[c]};
    for (int i = c - 1; i >= 0; --i) {
      FF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      acc[0] = ff_mul({Ah[i * S + c], Al[i * S + c]}, tcc);
      int k = i + 1;
      for (; k + 3 < c; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          acc[u] = ff_add(acc[u], ff_mul({Ah[i * S + k + u], Al[i * S + k + u]},
                                         {Ah[c * S + k + u], Al[c * S + k + u]}));
      }
      for (; k < c; ++k)
        acc[0] = ff_add(acc[0], ff_mul({Ah[i * S + k], Al[i * S + k]}, {Ah[c * S + k], Al[c * S + k]}));
      const FF sum = ff_add(ff_add(acc[0], acc[1]), ff_add(acc[2], acc[3]));
      const FF v = ff_neg(ff_mul(sum, {dh[i], dl[i]}));
      Ah[c * S + i] = v.hi;
      Al[c * S + i] = v.lo;
    }
  }
  __syncthreads();
  float* th = Thi + static_cast<int64_t>(mat) * ell * ell;
  float* tl = Tlo + static_cast<int64_t>(mat) * ell * ell;
  for (int p = t >> 5; p < ell; p += nt >> 5)
    for (int q = t & 31; q < ell; q += 32) {
      float hi = 0.f, lo = 0.f;
      if (p == q) {
        hi = dh[p];
        lo = dl[p];
      } else if (p < q) {
        hi = Ah[q * S + p];
        lo = Al[q * S + p];
      }
      th[p * ell + q] = hi;
      tl[p * ell + q] = lo;
    }
  if (t == 0 && bad) latch(status, kStQrBreakdown);
}

// Q = Y (T_hi + T_lo), T upper triangular. FF: float-float accumulation of the T_hi part.
// One thread per (row, block of 8 columns).
template <int LP, bool FF>
__global__ void __launch_bounds__(256) apply_tri_kernel(QrBatch b, int ell,
                                                        const float* __restrict__ Thi,
                                                        const float* __restrict__ Tlo) {
  extern __shared__ __align__(16) float tsm[];
  float* Th = tsm;             // [LP][LP]
  float* Tl = tsm + LP * LP;   // [LP][LP]
  const int mat = blockIdx.y;
  if (mat >= b.nmat) return;
  const float* th = Thi + static_cast<int64_t>(mat) * ell * ell;
  const float* tl = Tlo + static_cast<int64_t>(mat) * ell * ell;
  for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
    const int p = e / LP, q = e - p * LP;
    const bool in = p < ell && q < ell;
    Th[e] = in ? th[p * ell + q] : 0.f;
    Tl[e] = (FF && in) ? tl[p * ell + q] : 0.f;
  }
  __syncthreads();
  const float* Y = b.Y[mat];
  float* Q = b.Q[mat];
  const int64_t rows = b.rows[mat];
  constexpr int CB = 8, NCB = LP / CB;
  const int64_t total = rows * NCB;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / NCB;
    const int cb = static_cast<int>(e - i * NCB);
    float hi[CB], lo[CB];
#pragma unroll
    for (int q = 0; q < CB; ++q) hi[q] = lo[q] = 0.f;
    const float* yr = Y + i * ell;
    const int kmax = min(ell, (cb + 1) * CB);
    for (int k = 0; k < kmax; ++k) {
      const float y = yr[k];
#pragma unroll
      for (int q = 0; q < CB; ++q) {
        if (FF) {
          ff_fma(y, Th[k * LP + cb * CB + q], hi[q], lo[q]);
          lo[q] = fmaf(y, Tl[k * LP + cb * CB + q], lo[q]);
        } else {
          hi[q] = fmaf(y, Th[k * LP + cb * CB + q], hi[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const int c = cb * CB + q;
      if (c < ell) Q[i * ell + c] = FF ? __fadd_rn(hi[q], lo[q]) : hi[q];
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

size_t ws_bytes_for(const int64_t* rows, int nmat, int ell) {
  const int LP = lp_for(ell);
  size_t slabs = 0;
  for (int i = 0; i < nmat; ++i) slabs += cdiv(rows[i], kGramRows);
  size_t b = sizeof(double) * (slabs + nmat) * LP * LP;
  b += 2 * sizeof(float) * nmat * ell * ell + 256;
  for (int i = 0; i < nmat; ++i) b += sizeof(float) * rows[i] * ell + 256;
  return b + 4096;
}

template <int LP>
cudaError_t run(const Launcher& L, QrBatch b, int ell, char* ws, int* status) {
  const int nmat = b.nmat;
  int64_t slabs = 0, max_slabs = 0, max_rows = 0;
  for (int i = 0; i < nmat; ++i) {
    b.part_off[i] = slabs;
    const int64_t s = cdiv(b.rows[i], kGramRows);
    slabs += s;
    max_slabs = s > max_slabs ? s : max_slabs;
    max_rows = b.rows[i] > max_rows ? b.rows[i] : max_rows;
  }
  double* Gp = reinterpret_cast<double*>(ws);
  double* G = Gp + slabs * LP * LP;
  float* Thi = reinterpret_cast<float*>(G + nmat * LP * LP);
  float* Tlo = Thi + nmat * ell * ell;
  char* p = reinterpret_cast<char*>(Tlo + nmat * ell * ell);
  float* Q1[kMaxMats] = {nullptr, nullptr};
  for (int i = 0; i < nmat; ++i) {
    p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
    Q1[i] = reinterpret_cast<float*>(p);
    p += sizeof(float) * b.rows[i] * ell;
  }
  const size_t gram_smem = sizeof(float) * kGramRows * LP;
  const size_t apply_smem = sizeof(float) * 2 * LP * LP;
  const size_t chol_smemff = sizeof(float) * (2 * LP * (LP + 1) + 2 * LP);
  cudaError_t err;
  if ((err = cudaFuncSetAttribute(chol_inv_ff_kernel<LP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(chol_smemff))) != cudaSuccess ||

      (err = cudaFuncSetAttribute(gram_partial_kernel<LP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(gram_smem))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(apply_tri_kernel<LP, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(apply_smem))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(apply_tri_kernel<LP, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(apply_smem))) != cudaSuccess)
    return err;
  const int64_t apply_work = max_rows * (LP / 8);
  const unsigned apply_grid =
      static_cast<unsigned>(cdiv(apply_work, 256) < 2048 ? cdiv(apply_work, 256) : 2048);
  const unsigned sum_grid = static_cast<unsigned>(cdiv(static_cast<int64_t>(LP) * LP * 32, 256));
  for (int sweep = 0; sweep < 2; ++sweep) {
    // sweep 0 reads Y and writes the scratch Q1; sweep 1 reads Q1 and writes Q (Q may alias Y)
    QrBatch bb = b;
    for (int i = 0; i < nmat; ++i) {
      bb.Y[i] = sweep == 0 ? b.Y[i] : Q1[i];
      bb.Q[i] = sweep == 0 ? Q1[i] : b.Q[i];
    }
    gram_partial_kernel<LP><<<dim3(static_cast<unsigned>(max_slabs), nmat), kGramThreads,
                              gram_smem, L.stream>>>(bb, ell, Gp);
    sum_parts_kernel<<<dim3(sum_grid, nmat), 256, 0, L.stream>>>(Gp, bb, LP * LP, G);
    if (sweep == 0) {
      chol_inv_ff_kernel<LP><<<nmat, 256, chol_smemff, L.stream>>>(G, bb, ell, Thi, Tlo, status);
      apply_tri_kernel<LP, true><<<dim3(apply_grid, nmat), 256, apply_smem, L.stream>>>(
          bb, ell, Thi, Tlo);
    } else {
      chol_inv_ff_kernel<LP><<<nmat, 256, chol_smemff, L.stream>>>(G, bb, ell, Thi, Tlo, status);
      apply_tri_kernel<LP, false><<<dim3(apply_grid, nmat), 256, apply_smem, L.stream>>>(
          bb, ell, Thi, Tlo);
    }
    L.count(4);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace

size_t qr_ws_bytes(int64_t rows, int ell) {
  const int64_t r[2] = {rows, rows};
  return ws_bytes_for(r, 2, ell);
}

cudaError_t launch_qr_batch(const Launcher& L, int nmat, const float* const* Y,
                            const int64_t* rows, int ell, float* const* Q, void* ws,
                            size_t ws_bytes, int* status) {
  if (nmat < 1 || nmat > kMaxMats) return cudaErrorInvalidValue;
  if (ws_bytes < ws_bytes_for(rows, nmat, ell)) return cudaErrorInvalidValue;
  QrBatch b{};
  b.nmat = nmat;
  for (int i = 0; i < nmat; ++i) {
    b.Y[i] = Y[i];
    b.Q[i] = Q[i];
    b.rows[i] = rows[i];
  }
  char* w = static_cast<char*>(ws);
  switch (lp_for(ell)) {
    case 16: return run<16>(L, b, ell, w, status);
    case 32: return run<32>(L, b, ell, w, status);
    case 48: return run<48>(L, b, ell, w, status);
    case 64: return run<64>(L, b, ell, w, status);
    case 96: return run<96>(L, b, ell, w, status);
    default: return run<128>(L, b, ell, w, status);
  }
}

cudaError_t launch_qr(const Launcher& L, const float* Y, int64_t rows, int ell, float* Q,
                      void* ws, size_t ws_bytes, int* status) {
  return launch_qr_batch(L, 1, &Y, &rows, ell, &Q, ws, ws_bytes, status);
}

}  // namespace nmfrp
