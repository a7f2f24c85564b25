// Thin QR of tall FP32 matrices (Section 3, Eq. 3.4-3.5: Q from the QR decomposition of the
// sketch) by CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa & Yamamoto 2014): twice
//   G = Y^T Y,  G = R^T R (Cholesky),  Y <- Y R^{-1}.
//
// Precision. Sweep 1 sees cond(G) = cond(Y)^2, so its Gram matrix is accumulated in float-float
// arithmetic (error-free products by FMA and Knuth's TwoSum; about 48 significant bits, relative
// error near 1e-12 over a slab) and summed across slabs in float-float; R^{-1} is formed in
// float-float too (an l x l problem, ~44 bits) and applied in float-float, since its entries
// reach cond(Y) and their products cancel. The FP64 pipe of this GPU runs at 1/58 of the FP32
// rate (a warp-wide FP64 instruction holds its scheduler's FP64 pipe for ~67 cycles), so
// everything runs on the FP32 pipes. Sweep 2 starts from a nearly orthonormal matrix: its Gram
// and factor are float-float as well, its application FP32. The result is the Q of the QR
// factorisation whose R has a positive diagonal.
//
// R^{-1} without a triangular solve: symmetric Gaussian elimination of G carried along on an
// identity block, [G | I] -> [D L^T | L^{-1}] with G = L D L^T (L unit lower triangular), one
// barrier a pivot and every trailing entry updated in parallel; then R = D^{1/2} L^T and
// R^{-1} = L^{-T} D^{-1/2}, i.e. R^{-1}[k][c] = L^{-1}[c][k] / sqrt(D_c).
// Sweep 2 sees G = I + E with E small (the orthogonality error of sweep 1). There, with
// R = I + N (N upper triangular), R^T R = G reads N + N^T = E - N^T N: N is the upper triangle
// of E - N^T N with its diagonal halved, a fixed point reached from N = 0 with error of order
// |E|^(k+1) after k steps, and R^{-1} = I - N + N^2 - ... (Horner). When a = l max |E_ij| (a
// bound on the 2-norm of E) is at most 1e-3, a few steps and terms (the first is N = triu(E),
// no product) give R^{-1} to 1e-8 with matrix products only; otherwise the elimination runs.
//
// The Gram and apply kernels run two blocks an SM, each on an equal contiguous range of rows,
// taken in chunks of up to 64 rows (one contiguous run of floats) staged in shared memory with
// every global load in flight before the first store. Up to two independent matrices (the two
// chains of the sketch) go through each kernel in one launch: the blocks of matrix 0 come first,
// then those of matrix 1, split in proportion to their rows (blockIdx.x for the Cholesky).
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kSlab = 64;          // rows a Gram / apply chunk
constexpr int kQrThreads = 256;
constexpr int kMaxMats = 2;

struct QrBatch {
  const float* Y[kMaxMats];     // inputs of this sweep
  float* Q[kMaxMats];           // outputs of this sweep
  int64_t rows[kMaxMats];
  int64_t part_off[kMaxMats];   // first block (and Gram-partial slot) of each matrix
  int nblk[kMaxMats];           // blocks of each matrix
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
// x - a b with one renormalisation (the low parts of x and of the product combined by a plain
// add: error about 2^-44 (|x| + |a b|), the bound a backward-stable elimination step needs)
__device__ __forceinline__ FF ff_fms(FF x, FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  FF s = ff_two_sum(x.hi, -p);
  s.lo = __fadd_rn(s.lo, __fsub_rn(x.lo, e));
  return ff_quick(s.hi, s.lo);
}
// 1 / x: FP32 estimate (the fast approximate reciprocal: one Newton step squares its ~1e-7
// relative error), one Newton step in float-float (r + r (1 - x r))
__device__ __forceinline__ FF ff_recip(FF x) {
  const float r = __fdividef(1.f, x.hi);
  const FF e = ff_add({1.f, 0.f}, ff_neg(ff_mul(x, {r, 0.f})));
  return ff_add({r, 0.f}, ff_mul({r, 0.f}, e));
}
// sqrt(x): FP32 estimate q, one correction (x - q^2) / (2 q)
__device__ __forceinline__ FF ff_sqrt(FF x) {
  const float q = __fsqrt_rn(x.hi);
  const FF d = ff_add(x, ff_neg(ff_mul({q, 0.f}, {q, 0.f})));
  return ff_quick(q, __fdiv_rn(d.hi, __fmul_rn(2.f, q)));
}

// b.x[mat] without a local-memory copy of the by-value struct (mat is 0 or 1).
template <class T>
__device__ __forceinline__ T pick(const T (&a)[kMaxMats], int mat) {
  return mat ? a[1] : a[0];
}

// Block -> (matrix, block within it, its rows [r0, r1)); equal ranges, never empty.
__device__ __forceinline__ void range_of(const QrBatch& b, int& mat, int& blk, int64_t& r0,
                                         int64_t& r1) {
  int bb = blockIdx.x;
  mat = 0;
  if (b.nmat > 1 && bb >= b.nblk[0]) {
    bb -= b.nblk[0];
    mat = 1;
  }
  const int64_t rows = pick(b.rows, mat), nb = pick(b.nblk, mat);
  blk = bb;
  r0 = rows * bb / nb;
  r1 = rows * (bb + 1) / nb;
}

// sm[i * (LP + 1) + k] = Y[r0 + i][k] for rows r0 + i < r1 (at most 64) and k < ell, zero
// elsewhere (columns ell .. LP - 1, rows past r1). The rows are the contiguous run Y + r0 * ell,
// read as float4 when it is 16-byte aligned, all loads of a thread issued before its stores.
// The odd row stride spreads a column read by 32 consecutive rows over all banks.
template <int LP>
__device__ __forceinline__ void stage_slab(const float* __restrict__ Y, int64_t r1, int ell,
                                           int64_t r0, float* __restrict__ sm) {
  constexpr int S = LP + 1;
  constexpr int kV = (kSlab * LP / 4 + kQrThreads - 1) / kQrThreads;
  const int t = threadIdx.x;
  const int nrows = static_cast<int>(r1 - r0 < kSlab ? r1 - r0 : kSlab);
  const int count = nrows * ell;
  const float* src = Y + r0 * ell;
  for (int e = t; e < kSlab * S; e += kQrThreads) {   // padding (disjoint from the data)
    const int i = e / S, k = e - i * S;
    if (i >= nrows || k >= ell) sm[e] = 0.f;
  }
  int nv = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    nv = count >> 2;
    float4 buf[kV];
#pragma unroll
    for (int u = 0; u < kV; ++u) {
      const int v = t + u * kQrThreads;
      if (v < nv) buf[u] = reinterpret_cast<const float4*>(src)[v];
    }
#pragma unroll
    for (int u = 0; u < kV; ++u) {
      const int v = t + u * kQrThreads;
      if (v < nv) {
        int i = (4 * v) / ell, k = 4 * v - i * ell;
        const float x[4] = {buf[u].x, buf[u].y, buf[u].z, buf[u].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          sm[i * S + k] = x[c];
          if (++k == ell) {
            k = 0;
            ++i;
          }
        }
      }
    }
  }
  for (int f = 4 * nv + t; f < count; f += kQrThreads) {
    const int i = f / ell;
    sm[i * S + f - i * ell] = src[f];
  }
}

// Partial Gram of a block's rows in float-float: Gp[slot][p][q] = (hi, lo) for p <= q < ell
// (2 x 2 tiles of the upper triangle of the ell x ell block, each thread's tiles accumulated
// in registers over the block's chunks; other entries are not written).
template <int LP>
__global__ void __launch_bounds__(kQrThreads) gram_partial_kernel(QrBatch b, int ell,
                                                                  float2* __restrict__ Gp) {
  constexpr int S = LP + 1;
  constexpr int kT = ((LP / 2) * (LP / 2 + 1) / 2 + kQrThreads - 1) / kQrThreads;
  extern __shared__ float Ysm[];   // [kSlab][S]
  int mat, blk;
  int64_t r0, r1;
  range_of(b, mat, blk, r0, r1);
  const float* Y = pick(b.Y, mat);
  const int T2 = (ell + 1) >> 1, ntiles = T2 * (T2 + 1) / 2;
  int a0[kT], c0[kT];
#pragma unroll
  for (int v = 0; v < kT; ++v) {   // tile u -> (P, Qi), P <= Qi, row P holding T2 - P tiles
    int P = 0, u = threadIdx.x + v * kQrThreads;
    a0[v] = -1;
    if (u < ntiles) {
      while (u >= T2 - P) {
        u -= T2 - P;
        ++P;
      }
      a0[v] = 2 * P;
      c0[v] = 2 * (P + u);
    }
  }
  float h[kT][4], l[kT][4];
#pragma unroll
  for (int v = 0; v < kT; ++v)
#pragma unroll
    for (int x = 0; x < 4; ++x) h[v][x] = l[v][x] = 0.f;
  // equal chunks of at most 64 rows
  const int64_t nch = (r1 - r0 + kSlab - 1) / kSlab;
  for (int64_t ch = 0; ch < nch; ++ch) {
    const int64_t c = r0 + (r1 - r0) * ch / nch, c1 = r0 + (r1 - r0) * (ch + 1) / nch;
    if (ch > 0) __syncthreads();   // the previous chunk is consumed
    stage_slab<LP>(Y, c1, ell, c, Ysm);
    __syncthreads();
    const int nrows = static_cast<int>(c1 - c);
#pragma unroll
    for (int v = 0; v < kT; ++v) {
      if (a0[v] < 0) continue;
      const float* ya = Ysm + a0[v];
      const float* yc = Ysm + c0[v];
#pragma unroll 4
      for (int i = 0; i < nrows; ++i) {
        const float ax = ya[i * S], ay = ya[i * S + 1];
        const float cx = yc[i * S], cy = yc[i * S + 1];
        ff_fma(ax, cx, h[v][0], l[v][0]);
        ff_fma(ax, cy, h[v][1], l[v][1]);
        ff_fma(ay, cx, h[v][2], l[v][2]);
        ff_fma(ay, cy, h[v][3], l[v][3]);
      }
    }
  }
  float2* out = Gp + (pick(b.part_off, mat) + blk) * LP * LP;
#pragma unroll
  for (int v = 0; v < kT; ++v) {
    if (a0[v] < 0) continue;
    const int p = a0[v], q = c0[v];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const FF f = ff_quick(h[v][x], l[v][x]);
      out[(p + (x >> 1)) * LP + q + (x & 1)] = make_float2(f.hi, f.lo);
    }
  }
}

// G[mat][p][q] = sum over the matrix's blocks of Gp[slot][p][q] in float-float for p <= q < ell.
// A block takes 8 consecutive entries of row p (coalesced reads) and 32 groups over the slots,
// 8 loads in flight a thread, then a fixed-order tree (deterministic). Blocks holding no entry
// of the upper triangle return.
template <int LP>
__global__ void __launch_bounds__(256) sum_parts_kernel(const float2* __restrict__ Gp, QrBatch b,
                                                        int ell, float2* __restrict__ G) {
  constexpr int E = LP * LP;
  __shared__ FF red[32][8];
  const int mat = blockIdx.z;
  if (mat >= b.nmat) return;
  const int p = blockIdx.y, q0 = blockIdx.x * 8;
  if (p >= ell || q0 >= ell || q0 + 7 < p) return;
  const int x = threadIdx.x & 7, g = threadIdx.x >> 3;
  const int nparts = pick(b.nblk, mat);
  const float2* base = Gp + pick(b.part_off, mat) * E + p * LP + q0 + x;
  FF s = {0.f, 0.f};
  for (int k0 = g; k0 < nparts; k0 += 32 * 8) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + 32 * u;
      v[u] = k < nparts ? base[static_cast<int64_t>(k) * E] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) s = ff_add(s, {v[u].x, v[u].y});
  }
  red[g][x] = s;
  __syncthreads();
  for (int w = 16; w > 0; w >>= 1) {
    if (g < w) red[g][x] = ff_add(red[g][x], red[g + w][x]);
    __syncthreads();
  }
  if (g == 0) G[mat * E + p * LP + q0 + x] = make_float2(red[0][x].hi, red[0][x].lo);
}

// One block per matrix: T = R^{-1} (G = R^T R) by the elimination of [G | I] described at the
// top, in float-float. M holds the upper triangle of the trailing matrix (k >= i) and the strict
// lower triangle of L^{-1} (k < i; its unit diagonal is implicit). Step j reads row j and
// updates the rows below it: M[i][k] -= (M[j][i] / M[j][j]) * y_k with y_k = M[j][k] (k != j)
// and y_j = 1. The thread that updates the next pivot M[j + 1][j + 1] also forms its reciprocal
// (double-buffered in shared memory), so each step has one barrier. Writes T as T_hi + T_lo
// (two FP32 arrays, ell x ell row-major). A pivot below kPivotTol times its column's original
// diagonal (beyond what the float-float factor resolves: the column depends on the ones before
// it) is replaced by that bound, latches kStQrBreakdown and sets the column's bit in bad_cols
// (4 words a matrix, may be null).
constexpr float kPivotTol = 1e-12f;

template <int LP, bool NEAR_I>
__global__ void __launch_bounds__(512) chol_inv_ff_kernel(const float2* __restrict__ Gin,
                                                          QrBatch b, int ell,
                                                          float* __restrict__ Thi,
                                                          float* __restrict__ Tlo, int* status,
                                                          uint32_t* bad_cols) {
  constexpr int S = LP + 1;
  constexpr int kNT = 512, kPer = (LP * LP + kNT - 1) / kNT;
  extern __shared__ __align__(16) float chol_ff_sm[];
  float* Mh = chol_ff_sm;         // [LP][S]
  float* Ml = Mh + LP * S;        // [LP][S]
  float* rh = Ml + LP * S;        // [LP]  1 / sqrt(D_c)
  float* rl = rh + LP;
  float* d0 = rl + LP;            // [LP]  original diagonal G[c][c]
  float* Mx = d0 + LP;            // [LP][S] (sweep 2's product path)
  __shared__ FF pinv[2];          // 1 / M[j][j] of the current and the next pivot
  const int mat = blockIdx.x;
  if (mat >= b.nmat) return;
  const float2* G = Gin + static_cast<int64_t>(mat) * LP * LP;
  const int t = threadIdx.x;
  for (int e = t; e < LP * LP; e += kNT) {
    const int i = e / LP, k = e - i * LP;
    const float2 g = (i <= k && k < ell) ? G[e] : make_float2(0.f, 0.f);
    Mh[i * S + k] = g.x;
    Ml[i * S + k] = g.y;
    if (i == k) d0[i] = g.x;
  }
  if constexpr (NEAR_I) {
    __shared__ unsigned emax_bits;
    if (t == 0) emax_bits = 0u;
    __syncthreads();
    // E = G - I (FP32; the float-float Gram rounded once), in Mh (upper triangle, mirrored)
    unsigned mine = 0u;
    for (int e = t; e < ell * ell; e += kNT) {
      const int i = e / ell, k = e - i * ell;
      if (i > k) continue;
      const float v = __fadd_rn(__fadd_rn(Mh[i * S + k], -(i == k ? 1.f : 0.f)), Ml[i * S + k]);
      mine = max(mine, __float_as_uint(fabsf(v)));
      Mx[i * S + k] = v;
      Mx[k * S + i] = v;
    }
    atomicMax(&emax_bits, mine);
    __syncthreads();
    const float a2 = static_cast<float>(ell) * __uint_as_float(emax_bits);   // >= |E|_2
    if (a2 <= 1e-3f) {
      // error budget 1e-8: N after `steps` fixed-point steps is off by a2^(steps+1), the series
      // cut after N^terms by a2^(terms+1)
      const int steps = a2 <= 1e-4f ? 1 : 2, terms = a2 <= 1e-4f ? 2 : 3;
      float* E = Mx;
      float* N = Ml;
      float* Nn = Mh;
      // four partial sums: the dot products are latency-bound chains through shared memory
      auto dot = [&](const float* x, int xs, const float* y, int ys, int u0, int u1) {
        float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
        int u = u0;
        for (; u + 3 < u1; u += 4) {
          q0 = fmaf(x[u * xs], y[u * ys], q0);
          q1 = fmaf(x[(u + 1) * xs], y[(u + 1) * ys], q1);
          q2 = fmaf(x[(u + 2) * xs], y[(u + 2) * ys], q2);
          q3 = fmaf(x[(u + 3) * xs], y[(u + 3) * ys], q3);
        }
        for (; u < u1; ++u) q0 = fmaf(x[u * xs], y[u * ys], q0);
        return (q0 + q1) + (q2 + q3);
      };
      // first step from N = 0: N = triu(E), diagonal halved
      for (int e = t; e < LP * S; e += kNT) {
        const int i = e / S, k = e - i * S;
        N[e] = (i < ell && k < ell && i <= k) ? (i == k ? 0.5f : 1.f) * E[e] : 0.f;
      }
      __syncthreads();
      for (int step = 1; step < steps; ++step) {   // N <- triu(E - N^T N), diagonal halved
        for (int e = t; e < ell * ell; e += kNT) {
          const int i = e / ell, k = e - i * ell;
          float v = 0.f;
          if (i <= k) {
            v = E[i * S + k] - dot(N + i, S, N + k, S, 0, i + 1);   // (N^T N)_ik
            if (i == k) v *= 0.5f;
          }
          Nn[i * S + k] = v;
        }
        __syncthreads();
        for (int e = t; e < ell * ell; e += kNT) {
          const int i = e / ell, k = e - i * ell;
          N[i * S + k] = Nn[i * S + k];
        }
        __syncthreads();
      }
      // T = (I + N)^{-1} = I - N (I - N (I - ...)): P = I - N, then P <- I - N P
      float* P = Mx;
      float* Pn = Mh;
      for (int e = t; e < ell * ell; e += kNT) {
        const int i = e / ell, k = e - i * ell;
        P[i * S + k] = (i == k ? 1.f : 0.f) - N[i * S + k];
      }
      __syncthreads();
      for (int term = 1; term < terms; ++term) {
        for (int e = t; e < ell * ell; e += kNT) {
          const int i = e / ell, k = e - i * ell;
          float v = 0.f;
          if (i <= k) v = (i == k ? 1.f : 0.f) - dot(N + i * S, 1, P + k, S, i, k + 1);   // (N P)_ik
          Pn[i * S + k] = v;
        }
        __syncthreads();
        for (int e = t; e < ell * ell; e += kNT) {
          const int i = e / ell, k = e - i * ell;
          P[i * S + k] = Pn[i * S + k];
        }
        __syncthreads();
      }
      float* th = Thi + static_cast<int64_t>(mat) * ell * ell;
      float* tl = Tlo + static_cast<int64_t>(mat) * ell * ell;
      for (int e = t; e < ell * ell; e += kNT) {
        const int i = e / ell, k = e - i * ell;
        th[e] = P[i * S + k];
        tl[e] = 0.f;
      }
      return;
    }
    __syncthreads();
  }
  // this thread's entries (i, k) of the ell x ell block, fixed for all pivots
  int ei[kPer], ek[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = t + u * kNT;
    ei[u] = e / ell;
    ek[u] = e - ei[u] * ell;
    if (e >= ell * ell) ei[u] = -1;
  }
  // a pivot below kPivotTol of its original diagonal: the sketch is numerically rank deficient
  bool bad = false;
  auto floor_of = [&](int c) { return fmaxf(kPivotTol * d0[c], 1e-30f); };
  auto pivot_inv = [&](FF d, int c) {
    if (!(d.hi > floor_of(c))) {
      bad = true;
      if (bad_cols) atomicOr(&bad_cols[4 * mat + (c >> 5)], 1u << (c & 31));
      d = {floor_of(c), 0.f};
    }
    return ff_recip(d);
  };
  __syncthreads();
  if (t == 0) pinv[0] = pivot_inv({G[0].x, G[0].y}, 0);
  __syncthreads();
  for (int j = 0; j < ell; ++j) {
    const FF inv = pinv[j & 1];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int i = ei[u], k = ek[u];
      if (i > j && (k <= j || k >= i)) {
        const FF l = ff_mul({Mh[j * S + i], Ml[j * S + i]}, inv);
        const FF y = k == j ? FF{1.f, 0.f} : FF{Mh[j * S + k], Ml[j * S + k]};
        const FF v = ff_fms({Mh[i * S + k], Ml[i * S + k]}, l, y);
        Mh[i * S + k] = v.hi;
        Ml[i * S + k] = v.lo;
        if (i == j + 1 && k == i) pinv[(j + 1) & 1] = pivot_inv(v, i);
      }
    }
    __syncthreads();
  }
  for (int c = t; c < ell; c += kNT) {
    FF d = {Mh[c * S + c], Ml[c * S + c]};
    if (!(d.hi > floor_of(c))) d = {floor_of(c), 0.f};
    const FF r = ff_recip(ff_sqrt(d));
    rh[c] = r.hi;
    rl[c] = r.lo;
  }
  bad = __syncthreads_or(bad);
  float* th = Thi + static_cast<int64_t>(mat) * ell * ell;
  float* tl = Tlo + static_cast<int64_t>(mat) * ell * ell;
  for (int e = t; e < LP * LP; e += kNT) {
    const int p = e / LP, q = e - p * LP;
    if (p >= ell || q >= ell) continue;
    FF v = {0.f, 0.f};
    if (p == q) v = {rh[q], rl[q]};
    else if (p < q) v = ff_mul({Mh[q * S + p], Ml[q * S + p]}, {rh[q], rl[q]});
    th[p * ell + q] = v.hi;
    tl[p * ell + q] = v.lo;
  }
  if (t == 0 && bad) latch(status, kStQrBreakdown);
}

// Q = Y (T_hi + T_lo), T upper triangular, over a block's rows in 64-row chunks. FFA:
// float-float accumulation of the T_hi part. A task is (8-column block cb, row i) with cb
// uniform across a warp (so is the length of its inner loop) and the longest blocks first.
template <int LP, bool FFA>
__global__ void __launch_bounds__(kQrThreads) apply_tri_kernel(QrBatch b, int ell,
                                                               const float* __restrict__ Thi,
                                                               const float* __restrict__ Tlo) {
  constexpr int S = LP + 1;
  extern __shared__ __align__(16) float tsm[];
  float* Th = tsm;                             // [LP][LP]
  float* Tl = Th + LP * LP;                    // [LP][LP] (FFA only)
  float* Ysm = Tl + (FFA ? LP * LP : 0);       // [kSlab][S]
  int mat, blk;
  int64_t r0, r1;
  range_of(b, mat, blk, r0, r1);
  const float* th = Thi + static_cast<int64_t>(mat) * ell * ell;
  const float* tl = Tlo + static_cast<int64_t>(mat) * ell * ell;
#pragma unroll 8
  for (int e = threadIdx.x; e < LP * LP; e += kQrThreads) {
    const int p = e / LP, q = e - p * LP;
    const bool in = p < ell && q < ell;
    Th[e] = in ? th[p * ell + q] : 0.f;
    if (FFA) Tl[e] = in ? tl[p * ell + q] : 0.f;
  }
  const float* Y = pick(b.Y, mat);
  float* Q = pick(b.Q, mat);
  const int ncb = (ell + 7) >> 3;
  // equal chunks of at most 64 rows
  const int64_t nch = (r1 - r0 + kSlab - 1) / kSlab;
  for (int64_t ch = 0; ch < nch; ++ch) {
    const int64_t c = r0 + (r1 - r0) * ch / nch, c1 = r0 + (r1 - r0) * (ch + 1) / nch;
    if (ch > 0) __syncthreads();   // the previous chunk is consumed
    stage_slab<LP>(Y, c1, ell, c, Ysm);
    __syncthreads();
    const int nrows = static_cast<int>(c1 - c);
    for (int e = threadIdx.x; e < ncb * nrows; e += kQrThreads) {
      const int cb = ncb - 1 - e / nrows, i = e - (ncb - 1 - cb) * nrows;
      float hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) hi[q] = lo[q] = 0.f;
      const int kmax = min(ell, (cb + 1) * 8);
      const float* yr = Ysm + i * S;
      for (int k = 0; k < kmax; ++k) {
        const float y = yr[k];
        const float4 a0 = *reinterpret_cast<const float4*>(Th + k * LP + cb * 8);
        const float4 a1 = *reinterpret_cast<const float4*>(Th + k * LP + cb * 8 + 4);
        const float ta[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        if (FFA) {
          const float4 b0 = *reinterpret_cast<const float4*>(Tl + k * LP + cb * 8);
          const float4 b1 = *reinterpret_cast<const float4*>(Tl + k * LP + cb * 8 + 4);
          const float tb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            ff_fma(y, ta[q], hi[q], lo[q]);
            lo[q] = fmaf(y, tb[q], lo[q]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) hi[q] = fmaf(y, ta[q], hi[q]);
        }
      }
      float* qr = Q + (c + i) * ell + cb * 8;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (cb * 8 + q < ell) qr[q] = FFA ? __fadd_rn(hi[q], lo[q]) : hi[q];
    }
  }
}

int qr_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v > 0 ? v : 148;
  }
  return sms;
}

// Blocks of each matrix: two an SM in all (never more), split in proportion to the rows, none
// without rows.
void split_blocks(const int64_t* rows, int nmat, int* nblk) {
  const int64_t total = 2 * static_cast<int64_t>(qr_sms());
  int64_t want[kMaxMats] = {total, 0};
  if (nmat == 2) {
    int64_t n0 = (total * rows[0] + (rows[0] + rows[1]) / 2) / (rows[0] + rows[1]);
    n0 = n0 < 1 ? 1 : n0 > total - 1 ? total - 1 : n0;
    want[0] = n0;
    want[1] = total - n0;
  }
  for (int i = 0; i < nmat; ++i)
    nblk[i] = static_cast<int>(want[i] < rows[i] ? want[i] : rows[i]);
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
  int nblk[kMaxMats] = {0, 0};
  split_blocks(rows, nmat, nblk);
  size_t parts = 0;
  for (int i = 0; i < nmat; ++i) parts += nblk[i];
  size_t b = sizeof(float2) * (parts + nmat) * LP * LP;
  b += 2 * sizeof(float) * nmat * ell * ell + 256;
  for (int i = 0; i < nmat; ++i) b += sizeof(float) * rows[i] * ell + 256;
  return b + 4096;
}

template <int LP>
cudaError_t run(const Launcher& L, QrBatch b, int ell, char* ws, int* status, uint32_t* bad_cols) {
  const int nmat = b.nmat;
  split_blocks(b.rows, nmat, b.nblk);
  int64_t parts = 0;
  for (int i = 0; i < nmat; ++i) {
    b.part_off[i] = parts;
    parts += b.nblk[i];
  }
  float2* Gp = reinterpret_cast<float2*>(ws);
  float2* G = Gp + parts * LP * LP;
  float* Thi = reinterpret_cast<float*>(G + nmat * LP * LP);
  float* Tlo = Thi + nmat * ell * ell;
  char* p = reinterpret_cast<char*>(Tlo + nmat * ell * ell);
  float* Q1[kMaxMats] = {nullptr, nullptr};
  for (int i = 0; i < nmat; ++i) {
    p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
    Q1[i] = reinterpret_cast<float*>(p);
    p += sizeof(float) * b.rows[i] * ell;
  }
  const size_t slab_smem = sizeof(float) * kSlab * (LP + 1);
  const size_t apply_ff_smem = sizeof(float) * 2 * LP * LP + slab_smem;
  const size_t apply_smem = sizeof(float) * LP * LP + slab_smem;
  const size_t chol_smem = sizeof(float) * (2 * LP * (LP + 1) + 3 * LP);
  const size_t chol_smem2 = chol_smem + sizeof(float) * LP * (LP + 1);
  cudaError_t err;
  if ((err = cudaFuncSetAttribute(chol_inv_ff_kernel<LP, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(chol_smem))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(chol_inv_ff_kernel<LP, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(chol_smem2))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(gram_partial_kernel<LP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(slab_smem))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(apply_tri_kernel<LP, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(apply_ff_smem))) != cudaSuccess ||
      (err = cudaFuncSetAttribute(apply_tri_kernel<LP, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(apply_smem))) != cudaSuccess)
    return err;
  const unsigned grid = static_cast<unsigned>(parts);
  for (int sweep = 0; sweep < 2; ++sweep) {
    // sweep 0 reads Y and writes the scratch Q1; sweep 1 reads Q1 and writes Q (Q may alias Y)
    QrBatch bb = b;
    for (int i = 0; i < nmat; ++i) {
      bb.Y[i] = sweep == 0 ? b.Y[i] : Q1[i];
      bb.Q[i] = sweep == 0 ? Q1[i] : b.Q[i];
    }
    gram_partial_kernel<LP><<<grid, kQrThreads, slab_smem, L.stream>>>(bb, ell, Gp);
    sum_parts_kernel<LP><<<dim3(LP / 8, ell, nmat), 256, 0, L.stream>>>(Gp, bb, ell, G);
    if (sweep == 0)
      chol_inv_ff_kernel<LP, false><<<nmat, 512, chol_smem, L.stream>>>(G, bb, ell, Thi, Tlo,
                                                                        status, bad_cols);
    else
      chol_inv_ff_kernel<LP, true><<<nmat, 512, chol_smem2, L.stream>>>(G, bb, ell, Thi, Tlo,
                                                                        status, bad_cols);
    if (sweep == 0)
      apply_tri_kernel<LP, true><<<grid, kQrThreads, apply_ff_smem, L.stream>>>(bb, ell, Thi, Tlo);
    else
      apply_tri_kernel<LP, false><<<grid, kQrThreads, apply_smem, L.stream>>>(bb, ell, Thi, Tlo);
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
                            size_t ws_bytes, int* status, uint32_t* bad_cols) {
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
    case 16: return run<16>(L, b, ell, w, status, bad_cols);
    case 32: return run<32>(L, b, ell, w, status, bad_cols);
    case 48: return run<48>(L, b, ell, w, status, bad_cols);
    case 64: return run<64>(L, b, ell, w, status, bad_cols);
    case 96: return run<96>(L, b, ell, w, status, bad_cols);
    default: return run<128>(L, b, ell, w, status, bad_cols);
  }
}

cudaError_t launch_qr(const Launcher& L, const float* Y, int64_t rows, int ell, float* Q,
                      void* ws, size_t ws_bytes, int* status) {
  return launch_qr_batch(L, 1, &Y, &rows, ell, &Q, ws, ws_bytes, status, nullptr);
}

}  // namespace nmfrp
