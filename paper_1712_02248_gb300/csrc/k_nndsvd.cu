// NNDSVD initial factors (Boutsidis & Gallopoulos 2008) from compressed data.
//
// X ~ Q_L X_hat (Section 3, Eq. 3.4), so the top singular triplets of X are taken from X_hat:
// the eigenvectors U' of M = X_hat X_hat^T (l x l) give u_j = Q_L u'_j, sigma_j = sqrt(lambda_j)
// and v_j = X_hat^T u'_j / sigma_j. For each component the larger-norm sign part of the pair
// (u_j, v_j) is kept (the first pair in absolute value):
//   w_j = sqrt(sigma_j s') u_j^{+/-} / ||u_j^{+/-}||,  h_j = sqrt(sigma_j s') v_j^{+/-} / ||v_j^{+/-}||,
//   s' = ||u_j^{+/-}|| ||v_j^{+/-}||.
// The result does not depend on the sign of each eigenvector.
//
// Kernels: float-float Gram of the rows of X_hat (partials over column slabs, FP64 sum); one-block
// cyclic Jacobi eigensolver (round-robin ordering, ell/2 disjoint rotations per round, FP32,
// Rutishauser's stable rotation); U and V with per-block sums of the squared sign parts; one
// block that picks the signs and scales; the elementwise assembly of W and H.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kMaxL = 128;
constexpr int kSlabCols = 32;      // Gram blocks take multiples of 32 columns of X_hat ...
constexpr int kMaxSlabs = 256;     // ... wide enough to need at most 256 blocks
constexpr int kRowThreads = 128;   // threads (rows of U) a u_rows block
constexpr int kColThreads = 64;    // threads (columns of V) a v_cols block

__device__ __forceinline__ void ff_fma(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float v = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Partial M[p][q] = sum over a slab of `width` columns of X_hat[p][c] X_hat[q][c], p <= q.
__global__ void __launch_bounds__(256) xgram_partial_kernel(const float* __restrict__ Xhat,
                                                            int64_t n, int ell, int width,
                                                            double* __restrict__ part) {
  extern __shared__ float xs[];   // [ell][width + 1]
  const int S = width + 1;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * width;
  for (int e = threadIdx.x; e < ell * width; e += blockDim.x) {
    const int k = e / width, c = e - k * width;
    xs[k * S + c] = (c0 + c < n) ? Xhat[k * n + c0 + c] : 0.f;
  }
  __syncthreads();
  double* out = part + static_cast<int64_t>(blockIdx.x) * ell * ell;
  for (int e = threadIdx.x; e < ell * ell; e += blockDim.x) {
    const int p = e / ell, q = e - p * ell;
    if (p > q) continue;
    float hi = 0.f, lo = 0.f;
    for (int c = 0; c < width; ++c) ff_fma(xs[p * S + c], xs[q * S + c], hi, lo);
    out[e] = static_cast<double>(hi) + static_cast<double>(lo);
  }
}

// M[e] = sum over slabs of part[slab][e] (upper triangle, mirrored): one warp per entry.
__global__ void xgram_sum_kernel(const double* __restrict__ part, int nparts, int ell,
                                 double* __restrict__ M) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ell * ell) return;
  const int p = warp / ell, q = warp - p * ell;
  const int a = p < q ? p : q, b = p < q ? q : p;
  double v = 0.0;
  for (int s = lane; s < nparts; s += 32) v += part[static_cast<int64_t>(s) * ell * ell + a * ell + b];
  v = warp_sum(v);
  if (lane == 0) M[warp] = v;
}

// One Jacobi task: a column rotation (c_k, s_k) of a 1 x 2 or 2 x 2 block of A or V, then for a
// 2 x 2 block of A the row rotation (c_i, s_i). The entries are loaded first and stored later so
// that the loads of two tasks overlap (the tasks of one round touch disjoint entries).
struct JTask {
  int o0, o1, o2, o3;   // offsets into the shared A | V storage
  float x0, x1, x2, x3;
  float ci, si, ck, sk;
  bool two, live;
};

// floor(e / d) for e < 2^14 and 1 <= d <= 128: e * ceil(2^32 / d) / 2^32 is exact there
__device__ __forceinline__ int div_small(int e, unsigned long long magic) {
  return static_cast<int>((static_cast<unsigned long long>(e) * magic) >> 32);
}

// One block: cyclic Jacobi on M (FP32). Writes the eigenvectors of the
// r largest eigenvalues (columns, ell x r, row-major) and sigma_j = sqrt(lambda_j) (descending).
__global__ void __launch_bounds__(512) jacobi_kernel(const double* __restrict__ Mg, int ell, int r,
                                                     float* __restrict__ Ur,
                                                     float* __restrict__ sigma) {
  extern __shared__ float jsm[];
  const int L = (ell + 1) / 2 * 2;   // even size (a zero row/column pads odd ell)
  const int LS = L + 1, L1 = L - 1, half = L / 2;
  float* Am = jsm;                   // [L][LS]
  float* Vm = Am + L * LS;           // [L][LS]
  const int voff = L * LS;
#define A(p, q) Am[(p) * LS + (q)]
#define V(p, q) Vm[(p) * LS + (q)]
  __shared__ float cs[kMaxL / 2], sn[kMaxL / 2];
  __shared__ int order[kMaxL];
  __shared__ int rflag[2];           // "some pair rotates" of the current and the next round
  __shared__ unsigned dmax_bits;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < L * L; e += nt) {
    const int p = e / L, q = e - p * L;
    A(p, q) = (p < ell && q < ell) ? static_cast<float>(Mg[p * ell + q]) : 0.f;
    V(p, q) = (p == q) ? 1.f : 0.f;
  }
  if (t == 0) rflag[0] = rflag[1] = 0;
  const unsigned long long mag_half = ((1ull << 32) + half - 1) / half;
  const unsigned long long mag_L = ((1ull << 32) + L - 1) / L;
  const int nblk = half * half, ntask = nblk + L * half;
  int g = 0;   // rounds so far (over all sweeps): selects the round's flag
  for (int sweep = 0; sweep < 30; ++sweep) {
    // a sweep that rotates no pair ends the iteration. A pair is rotated while |a_pq| exceeds
    // 4 eps32 max_p |a_pp|: FP32 rounding leaves off-diagonal noise of order eps32 lambda_max
    // in every entry, which is also the eigenvector error the results are held to
    // (ell eps32 lambda_max / gap)
    if (t == 0) dmax_bits = 0u;
    __syncthreads();
    for (int p = t; p < L; p += nt) atomicMax(&dmax_bits, __float_as_uint(fabsf(A(p, p))));
    __syncthreads();
    const float thr = 4.f * 1.1920929e-7f * __uint_as_float(dmax_bits);
    int sweep_rot = 0;
    for (int round = 0; round < L1; ++round, ++g) {
      // round-robin pairing (circle method): position 0 fixed, positions 1..L-1 rotated by
      // `round`; pair i joins positions i and L-1-i (each index once per round, every pair of
      // indices once per sweep)
      auto pos = [&](int j) {
        const int u = j - 1 + round;
        return j == 0 ? 0 : (u >= L1 ? u - L1 : u) + 1;
      };
      auto pair = [&](int i, int& p, int& q) {
        const int a = pos(i), b = pos(L1 - i);
        p = a < b ? a : b;
        q = a < b ? b : a;
      };
      // the next round's flag is free: its last readers passed this round's first barrier
      if (t == 0) rflag[(g + 1) & 1] = 0;
      for (int i = t; i < half; i += nt) {
        int p, q;
        pair(i, p, q);
        const float apq = A(p, q);
        float c = 1.f, sv = 0.f;
        if (fabsf(apq) > 1e-30f && fabsf(apq) > thr) {
          // Rutishauser's rotation: t = sign(theta) / (|theta| + sqrt(theta^2 + 1))
          const float theta = __fdividef(A(q, q) - A(p, p), 2.f * apq);
          const float tt =
              copysignf(__frcp_rn(fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f))), theta);
          c = rsqrtf(fmaf(tt, tt, 1.f));
          sv = tt * c;
          rflag[g & 1] = 1;
        }
        cs[i] = c;
        sn[i] = sv;
      }
      __syncthreads();
      if (!rflag[g & 1]) continue;   // no pair rotates: A and V stay as they are
      sweep_rot = 1;
      // A <- J^T A J as 2 x 2 blocks (rows of pair i, columns of pair k), V <- V J
      auto load = [&](int e, JTask& k) {
        k.live = false;
        if (e >= ntask) return;
        if (e < nblk) {
          const int i = div_small(e, mag_half), kk = e - i * half;
          k.ci = cs[i];
          k.si = sn[i];
          k.ck = cs[kk];
          k.sk = sn[kk];
          if (k.si == 0.f && k.sk == 0.f) return;
          int p, q, pk, qk;
          pair(i, p, q);
          pair(kk, pk, qk);
          k.o0 = p * LS + pk;
          k.o1 = p * LS + qk;
          k.o2 = q * LS + pk;
          k.o3 = q * LS + qk;
          k.x0 = jsm[k.o0];
          k.x1 = jsm[k.o1];
          k.x2 = jsm[k.o2];
          k.x3 = jsm[k.o3];
          k.two = true;
        } else {
          const int f = e - nblk;
          const int i = div_small(f, mag_L), row = f - i * L;
          k.ck = cs[i];
          k.sk = sn[i];
          if (k.sk == 0.f) return;
          int p, q;
          pair(i, p, q);
          k.o0 = voff + row * LS + p;
          k.o1 = voff + row * LS + q;
          k.x0 = jsm[k.o0];
          k.x1 = jsm[k.o1];
          k.two = false;
        }
        k.live = true;
      };
      auto store = [&](const JTask& k) {
        if (!k.live) return;
        // columns: [c_k -s_k; s_k c_k] on the right, then rows with (c_i, s_i) on the left
        const float b0 = k.ck * k.x0 - k.sk * k.x1, b1 = k.sk * k.x0 + k.ck * k.x1;
        if (k.two) {
          const float b2 = k.ck * k.x2 - k.sk * k.x3, b3 = k.sk * k.x2 + k.ck * k.x3;
          jsm[k.o0] = k.ci * b0 - k.si * b2;
          jsm[k.o1] = k.ci * b1 - k.si * b3;
          jsm[k.o2] = k.si * b0 + k.ci * b2;
          jsm[k.o3] = k.si * b1 + k.ci * b3;
        } else {
          jsm[k.o0] = b0;
          jsm[k.o1] = b1;
        }
      };
      for (int e = t; e < ntask; e += 2 * nt) {
        JTask k0, k1;
        load(e, k0);
        load(e + nt, k1);
        store(k0);
        store(k1);
      }
      __syncthreads();
    }
    if (!sweep_rot) break;
  }
  // order by eigenvalue, descending: the rank of each diagonal entry (ties by index)
  for (int j = t; j < L; j += nt) order[j] = j;
  __syncthreads();
  for (int j = t; j < L; j += nt) {
    const float dj = A(j, j);
    int rank = 0;
    for (int k = 0; k < L; ++k) {
      const float dk = A(k, k);
      rank += (dk > dj || (dk == dj && k < j)) ? 1 : 0;
    }
    if (rank < r) order[rank] = j;
  }
  __syncthreads();
  for (int e = t; e < ell * r; e += nt) {
    const int k = e / r, j = e - k * r;
    Ur[e] = V(k, order[j]);
  }
  for (int j = t; j < r; j += nt) sigma[j] = sqrtf(fmaxf(A(order[j], order[j]), 0.f));
#undef A
#undef V
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// rows: U[i][j] = sum_k QL[i][k] Ur[k][j] into W (scratch); per-block sums of the squared
// positive and negative parts of each column. A thread takes one row: the row is read once and
// the r outputs accumulate side by side (independent chains).
template <int RM>   // RM >= r: the register arrays of a thread
__global__ void __launch_bounds__(kRowThreads) u_rows_kernel(const float* __restrict__ QL,
                                                             int64_t m, int ell, int r,
                                                             const float* __restrict__ Ur,
                                                             float* __restrict__ U,
                                                             double* __restrict__ part) {
  __shared__ float us[kMaxL * 64];
  __shared__ float acc[2][64];
  for (int e = threadIdx.x; e < ell * r; e += blockDim.x) us[e] = Ur[e];
  for (int e = threadIdx.x; e < 2 * 64; e += blockDim.x) acc[e / 64][e % 64] = 0.f;
  __syncthreads();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  float pp[RM], nn[RM];
#pragma unroll
  for (int j = 0; j < RM; ++j) pp[j] = nn[j] = 0.f;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += stride) {
    float s[RM];
#pragma unroll
    for (int j = 0; j < RM; ++j) s[j] = 0.f;
    const float* q = QL + i * ell;
    for (int k = 0; k < ell; ++k) {
      const float qk = q[k];
#pragma unroll
      for (int j = 0; j < RM; ++j)
        if (j < r) s[j] = fmaf(qk, us[k * r + j], s[j]);
    }
#pragma unroll
    for (int j = 0; j < RM; ++j)
      if (j < r) {
        U[i * r + j] = s[j];
        pp[j] = fmaf(s[j] > 0.f ? s[j] : 0.f, s[j], pp[j]);
        nn[j] = fmaf(s[j] < 0.f ? s[j] : 0.f, s[j], nn[j]);
      }
  }
#pragma unroll
  for (int j = 0; j < RM; ++j)
    if (j < r) {
      const float a = warp_sumf(pp[j]), b = warp_sumf(nn[j]);
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0][j], a);
        atomicAdd(&acc[1][j], b);
      }
    }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * r; e += blockDim.x)
    part[static_cast<int64_t>(blockIdx.x) * 2 * r + e] = acc[e / r][e % r];
}

// columns: V[j][c] = sum_k Xhat[k][c] Ur[k][j] / sigma_j into H (scratch); sign-part sums. A
// thread takes one column (coalesced over the block), read once.
template <int RM>
__global__ void __launch_bounds__(kColThreads) v_cols_kernel(const float* __restrict__ Xhat,
                                                             int64_t n, int ell, int r,
                                                             const float* __restrict__ Ur,
                                                             const float* __restrict__ sigma,
                                                             float* __restrict__ V,
                                                             double* __restrict__ part) {
  __shared__ float us[kMaxL * 64];
  __shared__ float isg[64];
  __shared__ float acc[2][64];
  for (int e = threadIdx.x; e < ell * r; e += blockDim.x) us[e] = Ur[e];
  for (int j = threadIdx.x; j < r; j += blockDim.x) isg[j] = sigma[j] > 0.f ? 1.f / sigma[j] : 0.f;
  for (int e = threadIdx.x; e < 2 * 64; e += blockDim.x) acc[e / 64][e % 64] = 0.f;
  __syncthreads();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  float pp[RM], nn[RM];
#pragma unroll
  for (int j = 0; j < RM; ++j) pp[j] = nn[j] = 0.f;
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c < n; c += stride) {
    float s[RM];
#pragma unroll
    for (int j = 0; j < RM; ++j) s[j] = 0.f;
    for (int k = 0; k < ell; ++k) {
      const float x = Xhat[k * n + c];
#pragma unroll
      for (int j = 0; j < RM; ++j)
        if (j < r) s[j] = fmaf(x, us[k * r + j], s[j]);
    }
#pragma unroll
    for (int j = 0; j < RM; ++j)
      if (j < r) {
        const float v = s[j] * isg[j];
        V[j * n + c] = v;
        pp[j] = fmaf(v > 0.f ? v : 0.f, v, pp[j]);
        nn[j] = fmaf(v < 0.f ? v : 0.f, v, nn[j]);
      }
  }
#pragma unroll
  for (int j = 0; j < RM; ++j)
    if (j < r) {
      const float a = warp_sumf(pp[j]), b = warp_sumf(nn[j]);
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0][j], a);
        atomicAdd(&acc[1][j], b);
      }
    }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * r; e += blockDim.x)
    part[static_cast<int64_t>(blockIdx.x) * 2 * r + e] = acc[e / r][e % r];
}

// out[e] = sum over the nb blocks of part[b][e] (e < 2 r): one warp a sum, lanes over the blocks,
// so the coefficient kernels read a single partial.
__global__ void part_sum_kernel(const double* __restrict__ part, int nb, int r,
                                double* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= 2 * r) return;
  double v = 0.0;
  for (int b = lane; b < nb; b += 32) v += part[static_cast<int64_t>(b) * 2 * r + w];
  v = warp_sum(v);
  if (lane == 0) out[w] = v;
}

// per component: which sign part to keep and the two scale factors
__global__ void nndsvd_coef_kernel(const double* __restrict__ upart, int nu,
                                   const double* __restrict__ vpart, int nv, int r,
                                   const float* __restrict__ sigma, float* __restrict__ coef) {
  // coef[j] = scale of u part, coef[r + j] = scale of v part, coef[2r + j] = mode
  // (0: absolute value, 1: positive parts, 2: negative parts, 3: zero component)
  const int j = threadIdx.x;
  if (j >= r) return;
  double up = 0, un = 0, vp = 0, vn = 0;
  for (int b = 0; b < nu; ++b) {
    up += upart[b * 2 * r + j];
    un += upart[b * 2 * r + r + j];
  }
  for (int b = 0; b < nv; ++b) {
    vp += vpart[b * 2 * r + j];
    vn += vpart[b * 2 * r + r + j];
  }
  const double sg = sigma[j];
  float cu = 0.f, cv = 0.f, mode = 3.f;
  if (j == 0) {
    cu = cv = static_cast<float>(sqrt(sg));
    mode = 0.f;
  } else {
    const double nup = sqrt(up), nun = sqrt(un), nvp = sqrt(vp), nvn = sqrt(vn);
    const double mp = nup * nvp, mn = nun * nvn;
    if (mp >= mn) {
      if (mp > 0.0) {
        const double f = sqrt(sg * mp);
        cu = static_cast<float>(f / nup);
        cv = static_cast<float>(f / nvp);
        mode = 1.f;
      }
    } else {
      const double f = sqrt(sg * mn);
      cu = static_cast<float>(f / nun);
      cv = static_cast<float>(f / nvn);
      mode = 2.f;
    }
  }
  coef[j] = cu;
  coef[r + j] = cv;
  coef[2 * r + j] = mode;
}

__device__ __forceinline__ float part_of(float x, int mode) {
  if (mode == 0) return fabsf(x);
  if (mode == 1) return x > 0.f ? x : 0.f;
  if (mode == 2) return x < 0.f ? -x : 0.f;
  return 0.f;
}

__global__ void nndsvd_apply_kernel(float* __restrict__ W, int64_t m, float* __restrict__ H,
                                    int64_t n, int r, const float* __restrict__ coef) {
  const int64_t tw = m * r, th = static_cast<int64_t>(r) * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tw + th;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < tw) {
      const int j = static_cast<int>(e % r);
      W[e] = coef[j] * part_of(W[e], static_cast<int>(coef[2 * r + j]));
    } else {
      const int64_t f = e - tw;
      const int j = static_cast<int>(f / n);
      H[f] = coef[r + j] * part_of(H[f], static_cast<int>(coef[2 * r + j]));
    }
  }
}

// columns a Gram block takes: a multiple of 32, at most kMaxSlabs blocks
int slab_width(int64_t n) {
  const int64_t w = (cdiv(n, kMaxSlabs) + kSlabCols - 1) / kSlabCols * kSlabCols;
  return static_cast<int>(w < kSlabCols ? kSlabCols : w);
}

int blocks_for(int64_t work, int threads = 256) {
  const int64_t b = cdiv(work, threads);
  return static_cast<int>(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

// Warm-start features. Per component j (one thread each): the sign part NNDSVD keeps (mode as
// in nndsvd_coef_kernel), 1 / ||p(u_j)||, 1 / ||p(v_j)||, f2_j = sigma_j ||p(u_j)|| ||p(v_j)||
// and sigma_j / sigma_0. cw: [mode, inu, inv, f2, ratio] x r.
__global__ void ws_coef_kernel(const double* __restrict__ upart, int nu,
                               const double* __restrict__ vpart, int nv, int r,
                               const float* __restrict__ sigma, float* __restrict__ cw,
                               float* __restrict__ hscale) {
  const int j = threadIdx.x;
  if (j >= r) return;
  double up = 0, un = 0, vp = 0, vn = 0;
  for (int b = 0; b < nu; ++b) {
    up += upart[b * 2 * r + j];
    un += upart[b * 2 * r + r + j];
  }
  for (int b = 0; b < nv; ++b) {
    vp += vpart[b * 2 * r + j];
    vn += vpart[b * 2 * r + r + j];
  }
  int mode;
  double nx, ny;
  if (j == 0) {
    mode = 0;
    nx = sqrt(up + un);
    ny = sqrt(vp + vn);
  } else {
    const double mp = sqrt(up) * sqrt(vp), mn = sqrt(un) * sqrt(vn);
    if (mp >= mn) {
      mode = mp > 0.0 ? 1 : 3;
      nx = sqrt(up);
      ny = sqrt(vp);
    } else {
      mode = 2;
      nx = sqrt(un);
      ny = sqrt(vn);
    }
  }
  const bool live = mode != 3 && nx > 0.0 && ny > 0.0;
  const double f2 = live ? static_cast<double>(sigma[j]) * nx * ny : 0.0;
  cw[j] = static_cast<float>(mode);
  cw[r + j] = live ? static_cast<float>(1.0 / nx) : 0.f;
  cw[2 * r + j] = live ? static_cast<float>(1.0 / ny) : 0.f;
  cw[3 * r + j] = static_cast<float>(f2);
  cw[4 * r + j] = sigma[0] > 0.f ? sigma[j] / sigma[0] : 0.f;
  hscale[j] = static_cast<float>(f2);
}

__device__ __forceinline__ float signed_part(float x, int mode) {
  if (mode == 0) return fabsf(x);
  if (mode == 1) return x;
  if (mode == 2) return -x;
  return 0.f;
}

// W side (in place on U -> W_b) and H side (in place on V -> H_b), features F_w (m x 3r),
// F_h (n x 3r).
__global__ void ws_feature_kernel(float* __restrict__ Wb, int64_t m, float* __restrict__ Hb,
                                  int64_t n, int r, const float* __restrict__ cw,
                                  float* __restrict__ Fw, float* __restrict__ Fh) {
  const int64_t tw = m * r, th = static_cast<int64_t>(r) * n;
  const float sm = sqrtf(static_cast<float>(m)), sn = sqrtf(static_cast<float>(n));
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tw + th;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < tw) {
      const int64_t i = e / r;
      const int j = static_cast<int>(e - i * r);
      const int mode = static_cast<int>(cw[j]);
      const float x = Wb[e];
      const float w = part_of(x, mode) * cw[r + j];
      Wb[e] = w;
      float* f = Fw + i * 3 * r;
      f[j] = sm * signed_part(x, mode);
      f[r + j] = sm * w;
      f[2 * r + j] = cw[4 * r + j];
    } else {
      const int64_t g = e - tw;
      const int j = static_cast<int>(g / n);
      const int64_t c = g - static_cast<int64_t>(j) * n;
      const int mode = static_cast<int>(cw[j]);
      const float y = Hb[g];
      const float h = part_of(y, mode) * cw[2 * r + j];
      Hb[g] = cw[3 * r + j] * h;
      float* f = Fh + c * 3 * r;
      f[j] = sn * signed_part(y, mode);
      f[r + j] = sn * h;
      f[2 * r + j] = cw[4 * r + j];
    }
  }
}

}  // namespace

size_t nndsvd_ws_bytes(int64_t m, int64_t n, int r, int ell) {
  const int64_t slabs = cdiv(n, slab_width(n));
  const int bu = blocks_for(m, kRowThreads), bv = blocks_for(n, kColThreads);
  return sizeof(double) * ((slabs + 1) * ell * ell + 2 * r * (bu + bv) + 4 * r) +
         sizeof(float) * (ell * r + r + 5 * r) + 4096;
}

cudaError_t launch_nndsvd(const Launcher& L, int64_t m, int64_t n, int r, int ell,
                          const float* QL, const float* Xhat, float* W, float* H, void* ws,
                          size_t ws_bytes, int* status) {
  (void)status;
  if (ell > kMaxL || r > 64 || r > ell) return cudaErrorNotSupported;
  if (ws_bytes < nndsvd_ws_bytes(m, n, r, ell)) return cudaErrorInvalidValue;
  const int width = slab_width(n);
  const int64_t slabs = cdiv(n, width);
  const int bu = blocks_for(m, kRowThreads), bv = blocks_for(n, kColThreads);
  double* gpart = static_cast<double*>(ws);
  double* M = gpart + slabs * ell * ell;
  double* upart = M + ell * ell;
  double* vpart = upart + 2 * r * bu;
  double* usum = vpart + 2 * r * bv;   // [2 r] sums over the u blocks, then [2 r] over the v blocks
  double* vsum = usum + 2 * r;
  float* Ur = reinterpret_cast<float*>(vsum + 2 * r);
  float* sigma = Ur + ell * r;
  float* coef = sigma + r;
  const size_t gsm = sizeof(float) * ell * (width + 1);
  cudaError_t err = cudaFuncSetAttribute(xgram_partial_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(gsm));
  if (err != cudaSuccess) return err;
  const int Lp = (ell + 1) / 2 * 2;
  const size_t jsm = sizeof(float) * 2 * Lp * (Lp + 1);
  if ((err = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(jsm))) != cudaSuccess)
    return err;
  xgram_partial_kernel<<<static_cast<unsigned>(slabs), 256, gsm, L.stream>>>(Xhat, n, ell, width,
                                                                            gpart);
  xgram_sum_kernel<<<static_cast<unsigned>(cdiv(static_cast<int64_t>(ell) * ell * 32, 256)), 256, 0,
                     L.stream>>>(gpart, static_cast<int>(slabs), ell, M);
  jacobi_kernel<<<1, 512, jsm, L.stream>>>(M, ell, r, Ur, sigma);
  if (r <= 16) {
    u_rows_kernel<16><<<bu, kRowThreads, 0, L.stream>>>(QL, m, ell, r, Ur, W, upart);
    v_cols_kernel<16><<<bv, kColThreads, 0, L.stream>>>(Xhat, n, ell, r, Ur, sigma, H, vpart);
  } else if (r <= 32) {
    u_rows_kernel<32><<<bu, kRowThreads, 0, L.stream>>>(QL, m, ell, r, Ur, W, upart);
    v_cols_kernel<32><<<bv, kColThreads, 0, L.stream>>>(Xhat, n, ell, r, Ur, sigma, H, vpart);
  } else {
    u_rows_kernel<64><<<bu, kRowThreads, 0, L.stream>>>(QL, m, ell, r, Ur, W, upart);
    v_cols_kernel<64><<<bv, kColThreads, 0, L.stream>>>(Xhat, n, ell, r, Ur, sigma, H, vpart);
  }
  part_sum_kernel<<<static_cast<unsigned>(cdiv(2 * r * 32, 256)), 256, 0, L.stream>>>(upart, bu, r,
                                                                                    usum);
  part_sum_kernel<<<static_cast<unsigned>(cdiv(2 * r * 32, 256)), 256, 0, L.stream>>>(vpart, bv, r,
                                                                                    vsum);
  nndsvd_coef_kernel<<<1, 64, 0, L.stream>>>(usum, 1, vsum, 1, r, sigma, coef);
  nndsvd_apply_kernel<<<blocks_for(m * r + r * n), 256, 0, L.stream>>>(W, m, H, n, r, coef);
  L.count(9);
  return cudaGetLastError();
}

size_t spectrum_ws_bytes(int64_t n, int ell) {
  const int64_t slabs = cdiv(n, slab_width(n));
  return sizeof(double) * ((slabs + 1) * ell * ell) + sizeof(float) * (ell * ell + ell) + 1024;
}

// Singular values of X_hat (ell x n): sigma_j = sqrt(lambda_j(X_hat X_hat^T)), descending, from
// the float-float Gram and the FP32 Jacobi eigensolver of the NNDSVD start (an eigenvalue's
// absolute error is about ell eps32 lambda_1).
cudaError_t launch_spectrum(const Launcher& L, int64_t n, int ell, const float* Xhat, void* ws,
                            size_t ws_bytes, float* sigma) {
  if (ell > kMaxL) return cudaErrorNotSupported;
  if (ws_bytes < spectrum_ws_bytes(n, ell)) return cudaErrorInvalidValue;
  const int width = slab_width(n);
  const int64_t slabs = cdiv(n, width);
  double* gpart = static_cast<double*>(ws);
  double* M = gpart + slabs * ell * ell;
  float* Ur = reinterpret_cast<float*>(M + ell * ell);
  const size_t gsm = sizeof(float) * ell * (width + 1);
  cudaError_t err = cudaFuncSetAttribute(xgram_partial_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(gsm));
  if (err != cudaSuccess) return err;
  const int Lp = (ell + 1) / 2 * 2;
  const size_t jsm = sizeof(float) * 2 * Lp * (Lp + 1);
  if ((err = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(jsm))) != cudaSuccess)
    return err;
  xgram_partial_kernel<<<static_cast<unsigned>(slabs), 256, gsm, L.stream>>>(Xhat, n, ell, width,
                                                                            gpart);
  xgram_sum_kernel<<<static_cast<unsigned>(cdiv(static_cast<int64_t>(ell) * ell * 32, 256)), 256, 0,
                     L.stream>>>(gpart, static_cast<int>(slabs), ell, M);
  jacobi_kernel<<<1, 512, jsm, L.stream>>>(M, ell, ell, Ur, sigma);
  L.count(3);
  return cudaGetLastError();
}

cudaError_t launch_warmstart_features(const Launcher& L, int64_t m, int64_t n, int r, int ell,
                                      const float* QL, const float* Xhat, float* Wb, float* Hb,
                                      float* hscale, float* Fw, float* Fh, void* ws,
                                      size_t ws_bytes) {
  if (ell > kMaxL || r > 64 || r > ell) return cudaErrorNotSupported;
  if (ws_bytes < nndsvd_ws_bytes(m, n, r, ell)) return cudaErrorInvalidValue;
  const int width = slab_width(n);
  const int64_t slabs = cdiv(n, width);
  const int bu = blocks_for(m, kRowThreads), bv = blocks_for(n, kColThreads);
  double* gpart = static_cast<double*>(ws);
  double* M = gpart + slabs * ell * ell;
  double* upart = M + ell * ell;
  double* vpart = upart + 2 * r * bu;
  double* usum = vpart + 2 * r * bv;   // [2 r] sums over the u blocks, then [2 r] over the v blocks
  double* vsum = usum + 2 * r;
  float* Ur = reinterpret_cast<float*>(vsum + 2 * r);
  float* sigma = Ur + ell * r;
  float* cw = sigma + r;
  const size_t gsm = sizeof(float) * ell * (width + 1);
  cudaError_t err = cudaFuncSetAttribute(xgram_partial_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(gsm));
  if (err != cudaSuccess) return err;
  const int Lp = (ell + 1) / 2 * 2;
  const size_t jsm = sizeof(float) * 2 * Lp * (Lp + 1);
  if ((err = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(jsm))) != cudaSuccess)
    return err;
  xgram_partial_kernel<<<static_cast<unsigned>(slabs), 256, gsm, L.stream>>>(Xhat, n, ell, width,
                                                                            gpart);
  xgram_sum_kernel<<<static_cast<unsigned>(cdiv(static_cast<int64_t>(ell) * ell * 32, 256)), 256, 0,
                     L.stream>>>(gpart, static_cast<int>(slabs), ell, M);
  jacobi_kernel<<<1, 512, jsm, L.stream>>>(M, ell, r, Ur, sigma);
  if (r <= 16) {
    u_rows_kernel<16><<<bu, kRowThreads, 0, L.stream>>>(QL, m, ell, r, Ur, Wb, upart);
    v_cols_kernel<16><<<bv, kColThreads, 0, L.stream>>>(Xhat, n, ell, r, Ur, sigma, Hb, vpart);
  } else if (r <= 32) {
    u_rows_kernel<32><<<bu, kRowThreads, 0, L.stream>>>(QL, m, ell, r, Ur, Wb, upart);
    v_cols_kernel<32><<<bv, kColThreads, 0, L.stream>>>(Xhat, n, ell, r, Ur, sigma, Hb, vpart);
  } else {
    u_rows_kernel<64><<<bu, kRowThreads, 0, L.stream>>>(QL, m, ell, r, Ur, Wb, upart);
    v_cols_kernel<64><<<bv, kColThreads, 0, L.stream>>>(Xhat, n, ell, r, Ur, sigma, Hb, vpart);
  }
  part_sum_kernel<<<static_cast<unsigned>(cdiv(2 * r * 32, 256)), 256, 0, L.stream>>>(upart, bu, r,
                                                                                    usum);
  part_sum_kernel<<<static_cast<unsigned>(cdiv(2 * r * 32, 256)), 256, 0, L.stream>>>(vpart, bv, r,
                                                                                    vsum);
  ws_coef_kernel<<<1, 64, 0, L.stream>>>(usum, 1, vsum, 1, r, sigma, cw, hscale);
  ws_feature_kernel<<<blocks_for(m * r + r * n), 256, 0, L.stream>>>(Wb, m, Hb, n, r, cw, Fw, Fh);
  L.count(9);
  return cudaGetLastError();
}

}  // namespace nmfrp
