// All iterations of FastHALS-RP / MU-RP in one cooperative (persistent) launch.
//
// The update rules are those of k_iterate.cu (Section 4, Eq. fastHALS_a with the Section 4.1
// terms; Section 3.1, Algorithm 3 with the semi-NMF rule). Each block owns a fixed slice of the
// rows of W and of the columns of H for the whole run. The slice's rows of X_chk and Q_L and its
// columns of X_hat and rows of Q_R are staged in shared memory once. A row of W is handled by a
// group of kGA = 4 lanes and a column of H by kGB = 16 lanes, each lane owning the components
// j = g, g + G, g + 2G, ... (g its index in the group); the factors stay in registers across
// iterations. One iteration:
//
//   A  (rows of W)    H_tld, G_W from the cross-block sums; S_W row; Gauss-Seidel sweep over j;
//                     the block adds its rows' W_tld_raw = Q_L^T W and W_raw^T W_raw (whose
//                     diagonal holds the squared column norms) into the cross-block sums.
//   -- grid barrier --
//   B  (columns of H) s_j = ||w_j||, W_tld = raw / s, G_H; compensation h_j *= s_j; S_H column;
//                     sweep; the block adds H Q_R, H H^T and <S_H, H> into the sums read by the
//                     next phase A and by the error monitor.
//   -- grid barrier --
//
// G_W and G_H are symmetric; every lane reads them along a row (consecutive lanes, distinct
// shared-memory banks).
//
// The sweep is incremental: t_j = S_j - sum_q w_q G_qj is formed for every j; when w_j moves by d
// (computed by the lane owning j and broadcast in the group) every later t_j' drops by d G_jj'.
// These are the Gauss-Seidel values of the paper's component-by-component update.
//
// Cross-block sums: FP32 red.add into kCopies copies (block b adds into copy b % kCopies), read
// back through L2 as a fixed-order sum of the copies. The order of the adds within a copy varies
// from run to run, so results can differ in the last bits between runs.
//
// Error monitor (no read of X): after the last iteration the kernel leaves in mon[0] the cross
// term <W_tld^T X_hat, H> and in mon[1] the quadratic term <W^T W, H H^T>; with ||X||^2 they give
// ||X - W H||^2 ~ ||X||^2 - 2 mon[0] + mon[1] (X replaced by Q_L Q_L^T X in the cross term,
// Section 3 Eq. 3.4).
//
// If *done is set on entry (an earlier residual check reached the target) the kernel returns at
// once. Every wait is bounded: on time-out the kernel latches NMF_ERR_TIMEOUT and all blocks leave.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kPT = 768;          // threads per block (one block per SM, 85 registers a thread)
constexpr int kGA = 4;            // lanes per row of W
constexpr int kGB = 16;           // lanes per column of H
constexpr int kMaxRows = kPT / kGA;   // rows of W per block
constexpr int kMaxCols = kPT / kGB;   // columns of H per block
constexpr int kCopies = 8;        // copies of each cross-block sum
constexpr long long kWaitCycles = 4000000000LL;   // about two seconds of polling

struct Barrier {
  unsigned int count;
  unsigned int gen;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a co-resident grid. Returns false if the wait ran out.
__device__ bool grid_sync(Barrier* bar, unsigned nblocks, int* status, int* abort_flag) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = ld_acquire(&bar->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire(&bar->gen) == g) {
        if (clock64() - t0 > kWaitCycles || *reinterpret_cast<volatile int*>(abort_flag)) {
          ok = 0;
          break;
        }
      }
      if (!ok) {
        latch(status, kStTimeout);
        atomicExch(abort_flag, 1);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ float posp(float v) { return v > 0.f ? v : 0.f; }
__device__ __forceinline__ float negp(float v) { return v < 0.f ? -v : 0.f; }

struct PArgs {
  int64_t m, n;
  int r, ell, iters, rule;
  int RB, CB;     // rows / columns per block
  float alpha, beta, eps;
  const float* QL;
  const float* QR;
  const float* Xhat;
  const float* Xchk;
  float* W;
  float* H;
  float* accA;    // [2][kCopies][EA]: phase-A sums (W_tld_raw, W^T W)
  float* accB;    // [2][kCopies][EB]: phase-B sums (H_tld, H H^T, cross)
  float* mon;     // [2]: cross term and quadratic term of the last iteration
  const int* done;
  Barrier* bar;
  int* status;
  int* abort_flag;
};

// Phase-A entries: W_tld_raw (ell x r) then W^T W (r x r). Phase-B entries: H_tld (r x ell),
// H H^T (r x r), cross (1).
__host__ __device__ __forceinline__ int ea_size(int r, int ell) { return ell * r + r * r; }
__host__ __device__ __forceinline__ int eb_size(int r, int ell) { return r * ell + r * r + 1; }

// Fixed-order sum of the kCopies copies of entry e, read through L2 (the copies are written by
// other blocks' atomics).
__device__ __forceinline__ float acc_read(const float* base, int E, int e) {
  float v[kCopies];
#pragma unroll
  for (int c = 0; c < kCopies; ++c) v[c] = __ldcg(base + c * E + e);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kCopies; ++c) s += v[c];
  return s;
}

// CA components per lane in phase A (RP = kGA * CA), CB_ per lane in phase B (kGB * CB_ >= RP).
template <int CA, int CB_, int RULE>
__global__ void __launch_bounds__(kPT, 1) iterate_persistent_kernel(PArgs a) {
  constexpr int RP = kGA * CA;
  constexpr int RPB = kGB * CB_;
  static_assert(RPB >= RP, "phase B must cover the components of phase A");
  extern __shared__ __align__(16) float sh[];
  const int r = a.r, ell = a.ell, t = threadIdx.x;
  const int EA = ea_size(r, ell), EB = eb_size(r, ell);
  const int LS = ell | 1;                // odd stride of staged rows (conflict-free reads)
  float* HtT = sh;                       // [ell][RPB]  H_tld^T
  float* Gw = HtT + ell * RPB;           // [RPB][RPB]
  float* WtS = Gw + RPB * RPB;           // [ell][RPB]  W_tld (normalised)
  float* Gh = WtS + ell * RPB;           // [RPB][RPB]
  float* sc = Gh + RPB * RPB;            // [RPB]       s_j of the last W phase
  float* inv = sc + RPB;                 // [RPB]       1 / G_jj of the current phase
  float* stA = inv + RPB;                // [kMaxRows][RP]  rows of W, later columns of H
  float* stX = stA + kMaxRows * RPB;     // [RB][LS]    rows of X_chk
  float* stB = stX + a.RB * LS;          // [RB][LS]    rows of Q_L
  float* stX2 = stB + a.RB * LS;         // [CB][LS]    columns of X_hat
  float* stB2 = stX2 + a.CB * LS;        // [CB][LS]    rows of Q_R
  __shared__ float red[kPT / 32];
  const unsigned G = gridDim.x;
  const int64_t rb = (a.m + G - 1) / G, cbk = (a.n + G - 1) / G;
  const int64_t r0 = blockIdx.x * rb, r1 = min(a.m, r0 + rb);
  const int64_t c0 = blockIdx.x * cbk, c1 = min(a.n, c0 + cbk);
  const int nrows = r1 > r0 ? static_cast<int>(r1 - r0) : 0;
  const int ncols = c1 > c0 ? static_cast<int>(c1 - c0) : 0;
  const bool normalize = (RULE == 0);
  const bool plain = (a.alpha == 0.f && a.beta == 0.f);

  if (*reinterpret_cast<const volatile int*>(a.done)) return;   // the solve has converged

  for (int j = t; j < RPB; j += kPT) sc[j] = 1.f;

  // phase-A role: row slot ra (row r0 + ra), lane ga in its group; phase-B role: column slot cb
  const int ra = t / kGA, ga = t % kGA;
  const int cb = t / kGB, gb = t % kGB;
  const bool has_row = ra < nrows, has_col = cb < ncols;
  const int64_t myrow = r0 + ra, mycol = c0 + cb;
  float w[CA], h[CB_];
#pragma unroll
  for (int c = 0; c < CA; ++c) {
    const int j = ga + kGA * c;
    w[c] = (has_row && j < r) ? a.W[myrow * r + j] : 0.f;
  }
#pragma unroll
  for (int c = 0; c < CB_; ++c) {
    const int j = gb + kGB * c;
    h[c] = (has_col && j < r) ? a.H[j * a.n + mycol] : 0.f;
  }
  for (int e = t; e < a.RB * ell; e += kPT) {
    const int i = e / ell, k = e - i * ell;
    const bool in = i < nrows;
    stX[i * LS + k] = in ? a.Xchk[(r0 + i) * ell + k] : 0.f;
    stB[i * LS + k] = in ? a.QL[(r0 + i) * ell + k] : 0.f;
  }
  for (int e = t; e < a.CB * ell; e += kPT) {
    const int cI = e / ell, k = e - cI * ell;
    const bool in = cI < ncols;
    stX2[cI * LS + k] = in ? a.Xhat[k * a.n + c0 + cI] : 0.f;
    stB2[cI * LS + k] = in ? a.QR[(c0 + cI) * ell + k] : 0.f;
  }

  // phase-B block sums: H_tld (staged columns of H in stA x rows of Q_R), H H^T, cross term
  auto add_b = [&](float* dst, float cross) {
    for (int e = t; e < r * ell; e += kPT) {
      const int j = e / ell, k = e - j * ell;
      float v = 0.f;
      for (int q = 0; q < ncols; ++q) v = fmaf(stA[q * RPB + j], stB2[q * LS + k], v);
      atomicAdd(&dst[e], v);
    }
    for (int e = t; e < r * r; e += kPT) {
      const int p = e / r, q2 = e - p * r;
      float v = 0.f;
      for (int q = 0; q < ncols; ++q) v = fmaf(stA[q * RPB + p], stA[q * RPB + q2], v);
      atomicAdd(&dst[r * ell + e], v);
    }
    if (t == 0) atomicAdd(&dst[r * ell + r * r], cross);
  };
  // stage this thread's components of its column of H
  auto stage_h = [&]() {
    if (has_col) {
#pragma unroll
      for (int c = 0; c < CB_; ++c) stA[cb * RPB + gb + kGB * c] = h[c];
    }
  };

  // prologue: H_tld, H H^T of the initial H into accB[1]
  for (int e = t; e < kMaxRows * RPB; e += kPT) stA[e] = 0.f;
  __syncthreads();
  stage_h();
  __syncthreads();
  add_b(a.accB + (1 * kCopies + blockIdx.x % kCopies) * EB, 0.f);
  if (!grid_sync(a.bar, G, a.status, a.abort_flag)) return;

  for (int it = 0; it < a.iters; ++it) {
    const int ph = it & 1, pr = ph ^ 1;
    float* accA_w = a.accA + (ph * kCopies + blockIdx.x % kCopies) * EA;
    const float* accB_r = a.accB + pr * kCopies * EB;
    // ---------------- phase A: rows of W
    // clear the phase-A sums written two phases ago (already read), a slice per block
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * kPT + t; e < kCopies * EA;
         e += static_cast<int64_t>(G) * kPT)
      a.accA[pr * kCopies * EA + e] = 0.f;
    for (int e = t; e < ell * RPB; e += kPT) {
      const int k = e / RPB, j = e - k * RPB;
      HtT[e] = (j < r) ? acc_read(accB_r, EB, j * ell + k) : 0.f;
    }
    __syncthreads();
    for (int e = t; e < RPB * RPB; e += kPT) {
      const int p = e / RPB, q = e - p * RPB;
      float g = 0.f;
      if (p < r && q < r)
        for (int k = 0; k < ell; ++k) g = fmaf(HtT[k * RPB + p], HtT[k * RPB + q], g);
      Gw[e] = g;
      if (p == q) inv[p] = g > 0.f ? 1.f / g : 0.f;
    }
    __syncthreads();
    {
      float s[CA];
#pragma unroll
      for (int c = 0; c < CA; ++c) {
        w[c] = w[c] / sc[ga + kGA * c];   // normalisation of the previous W phase (1 for MU)
        s[c] = 0.f;
      }
      const float* xr = stX + (has_row ? ra : 0) * LS;
      for (int k = 0; k < ell; ++k) {
        const float xk = xr[k];
#pragma unroll
        for (int c = 0; c < CA; ++c) s[c] = fmaf(xk, HtT[k * RPB + ga + kGA * c], s[c]);
      }
      if (RULE == 0) {
        // t_j = S_j - sum_q w_q G_qj with w_q gathered from the group
        // j = kGA * cj + o: the slot cj is unrolled (register index), the owner lane o is not
#pragma unroll
        for (int cq = 0; cq < CA; ++cq) {
#pragma unroll 1
          for (int o = 0; o < kGA; ++o) {
            const int q = kGA * cq + o;
            const float wq = __shfl_sync(0xffffffffu, w[cq], o, kGA);
#pragma unroll
            for (int c = 0; c < CA; ++c) s[c] = fmaf(-wq, Gw[q * RPB + ga + kGA * c], s[c]);
          }
        }
#pragma unroll
        for (int cj = 0; cj < CA; ++cj) {
#pragma unroll 1
          for (int o = 0; o < kGA; ++o) {
            const int j = kGA * cj + o;
            float d = 0.f;
            if (ga == o && j < r && Gw[j * RPB + j] > 0.f) {
              const float wn = fmaxf(0.f, w[cj] + s[cj] * inv[j]);
              d = wn - w[cj];
              w[cj] = wn;
            }
            d = __shfl_sync(0xffffffffu, d, o, kGA);
#pragma unroll
            for (int c = 0; c < CA; ++c)
              if (ga + kGA * c > j) s[c] = fmaf(-d, Gw[j * RPB + ga + kGA * c], s[c]);
          }
        }
      } else {
        float num[CA], den[CA];
#pragma unroll
        for (int c = 0; c < CA; ++c) {
          num[c] = posp(s[c]);
          den[c] = negp(s[c]) + a.eps;
        }
#pragma unroll
        for (int cq = 0; cq < CA; ++cq) {
#pragma unroll 1
          for (int o = 0; o < kGA; ++o) {
            const int q = kGA * cq + o;
            const float wq = __shfl_sync(0xffffffffu, w[cq], o, kGA);
#pragma unroll
            for (int c = 0; c < CA; ++c) {
              const float gq = Gw[q * RPB + ga + kGA * c];
              num[c] = fmaf(wq, negp(gq), num[c]);
              den[c] = fmaf(wq, posp(gq), den[c]);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < CA; ++c)
          w[c] = (ga + kGA * c < r) ? w[c] * sqrtf(num[c] / den[c]) : 0.f;
      }
      if (!has_row) {
#pragma unroll
        for (int c = 0; c < CA; ++c) w[c] = 0.f;
      }
      if (ra < kMaxRows) {
#pragma unroll
        for (int c = 0; c < CA; ++c) stA[ra * RPB + ga + kGA * c] = w[c];
      }
    }
    __syncthreads();
    for (int e = t; e < ell * r; e += kPT) {
      const int k = e / r, j = e - k * r;
      float v = 0.f;
      for (int q = 0; q < nrows; ++q) v = fmaf(stB[q * LS + k], stA[q * RPB + j], v);
      atomicAdd(&accA_w[e], v);
    }
    for (int e = t; e < r * r; e += kPT) {
      const int p = e / r, q2 = e - p * r;
      float v = 0.f;
      for (int q = 0; q < nrows; ++q) v = fmaf(stA[q * RPB + p], stA[q * RPB + q2], v);
      atomicAdd(&accA_w[ell * r + e], v);
    }
    if (!grid_sync(a.bar, G, a.status, a.abort_flag)) return;

    // ---------------- phase B: columns of H
    const float* accA_r = a.accA + ph * kCopies * EA;
    float* accB_w = a.accB + (ph * kCopies + blockIdx.x % kCopies) * EB;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * kPT + t; e < kCopies * EB;
         e += static_cast<int64_t>(G) * kPT)
      a.accB[pr * kCopies * EB + e] = 0.f;
    for (int j = t; j < RPB; j += kPT) {
      const float c2 = (j < r) ? acc_read(accA_r, EA, ell * r + j * r + j) : 0.f;
      sc[j] = (normalize && j < r && c2 > 0.f) ? sqrtf(c2) : 1.f;
    }
    __syncthreads();
    for (int e = t; e < ell * RPB; e += kPT) {
      const int k = e / RPB, j = e - k * RPB;
      WtS[e] = (j < r) ? acc_read(accA_r, EA, k * r + j) / sc[j] : 0.f;
    }
    __syncthreads();
    for (int e = t; e < RPB * RPB; e += kPT) {
      const int p = e / RPB, q = e - p * RPB;
      float g = 0.f;
      if (p < r && q < r)
        for (int k = 0; k < ell; ++k) g = fmaf(WtS[k * RPB + p], WtS[k * RPB + q], g);
      Gh[e] = g;
      if (p == q) inv[p] = g > 0.f ? 1.f / g : 0.f;
    }
    __syncthreads();
    float cross = 0.f;
    {
      float s[CB_], shc[CB_];
#pragma unroll
      for (int c = 0; c < CB_; ++c) {
        h[c] *= sc[gb + kGB * c];
        s[c] = 0.f;
      }
      const float* xc = stX2 + (has_col ? cb : 0) * LS;
      for (int k = 0; k < ell; ++k) {
        const float xk = xc[k];
#pragma unroll
        for (int c = 0; c < CB_; ++c) s[c] = fmaf(xk, WtS[k * RPB + gb + kGB * c], s[c]);
      }
#pragma unroll
      for (int c = 0; c < CB_; ++c) shc[c] = s[c];   // S_H column for the monitor
      if (RULE == 0) {
#pragma unroll
        for (int cq = 0; cq < CB_; ++cq) {
#pragma unroll 1
          for (int o = 0; o < kGB; ++o) {
            const int q = kGB * cq + o;
            const float hq = __shfl_sync(0xffffffffu, h[cq], o, kGB);
#pragma unroll
            for (int c = 0; c < CB_; ++c) s[c] = fmaf(-Gh[q * RPB + gb + kGB * c], hq, s[c]);
          }
        }
#pragma unroll
        for (int cj = 0; cj < CB_; ++cj) {
#pragma unroll 1
          for (int o = 0; o < kGB; ++o) {
          const int j = kGB * cj + o;
          float d = 0.f;
          if (gb == o && j < r) {
            const float g = Gh[j * RPB + j];
            float hn = h[cj];
            if (plain) {
              if (g > 0.f) hn = fmaxf(0.f, h[cj] + s[cj] * inv[j]);
            } else if (g + a.beta > 0.f) {
              hn = fmaxf(0.f, (fmaf(h[cj], g, s[cj]) - a.alpha) / (g + a.beta));
            }
            d = hn - h[cj];
            h[cj] = hn;
          }
          d = __shfl_sync(0xffffffffu, d, o, kGB);
#pragma unroll
          for (int c = 0; c < CB_; ++c)
            if (gb + kGB * c > j) s[c] = fmaf(-d, Gh[j * RPB + gb + kGB * c], s[c]);
          }
        }
      } else {
        float num[CB_], den[CB_];
#pragma unroll
        for (int c = 0; c < CB_; ++c) {
          num[c] = posp(s[c]);
          den[c] = negp(s[c]) + a.eps;
        }
#pragma unroll
        for (int cq = 0; cq < CB_; ++cq) {
#pragma unroll 1
          for (int o = 0; o < kGB; ++o) {
            const int q = kGB * cq + o;
            const float hq = __shfl_sync(0xffffffffu, h[cq], o, kGB);
#pragma unroll
            for (int c = 0; c < CB_; ++c) {
              const float gq = Gh[q * RPB + gb + kGB * c];
              num[c] = fmaf(negp(gq), hq, num[c]);
              den[c] = fmaf(posp(gq), hq, den[c]);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < CB_; ++c)
          h[c] = (gb + kGB * c < r) ? h[c] * sqrtf(num[c] / den[c]) : 0.f;
      }
      if (!has_col) {
#pragma unroll
        for (int c = 0; c < CB_; ++c) h[c] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < CB_; ++c) cross = fmaf(shc[c], h[c], cross);
    }
    stage_h();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cross += __shfl_xor_sync(0xffffffffu, cross, o);
    if ((t & 31) == 0) red[t >> 5] = cross;
    __syncthreads();
    float csum = 0.f;
    if (t == 0)
      for (int wI = 0; wI < kPT / 32; ++wI) csum += red[wI];
    add_b(accB_w, csum);
    if (!grid_sync(a.bar, G, a.status, a.abort_flag)) return;
  }
  // the last iteration's monitor terms: cross, and <W^T W, H H^T> for the normalised W
  if (blockIdx.x == 0 && a.iters > 0) {
    const int ph = (a.iters - 1) & 1;
    const float* accA_r = a.accA + ph * kCopies * EA;
    const float* accB_r = a.accB + ph * kCopies * EB;
    float q2 = 0.f;
    for (int e = t; e < r * r; e += kPT) {
      const int p = e / r, q = e - p * r;
      const float gww = acc_read(accA_r, EA, ell * r + e) / (sc[p] * sc[q]);
      q2 = fmaf(gww, acc_read(accB_r, EB, r * ell + e), q2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
    if ((t & 31) == 0) red[t >> 5] = q2;
    __syncthreads();
    if (t == 0) {
      float s = 0.f;
      for (int wI = 0; wI < kPT / 32; ++wI) s += red[wI];
      a.mon[0] = acc_read(accB_r, EB, r * ell + r * r);
      a.mon[1] = s;
    }
  }
  // write back: W normalised by the last s_j, H
  if (a.iters > 0) {
    if (has_row)
#pragma unroll
      for (int c = 0; c < CA; ++c) {
        const int j = ga + kGA * c;
        if (j < r) a.W[myrow * r + j] = normalize ? w[c] / sc[j] : w[c];
      }
    if (has_col)
#pragma unroll
      for (int c = 0; c < CB_; ++c) {
        const int j = gb + kGB * c;
        if (j < r) a.H[j * a.n + mycol] = h[c];
      }
  }
}

size_t smem_for(int RPB, int ell, int RB, int CB) {
  const int LS = ell | 1;
  return sizeof(float) * (2 * ell * RPB + 2 * RPB * RPB + 2 * RPB + kMaxRows * RPB +
                          static_cast<size_t>(2 * RB + 2 * CB) * LS);
}

template <int CA, int CB_, int RULE>
cudaError_t launch(const Launcher& L, PArgs& a, int grid) {
  auto k = iterate_persistent_kernel<CA, CB_, RULE>;
  const size_t smem = smem_for(kGB * CB_, a.ell, a.RB, a.CB);
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPT, smem)) != cudaSuccess)
    return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {&a};
  err = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k), dim3(grid), dim3(kPT), args, smem,
                                    L.stream);
  L.count();
  return err;
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

}  // namespace

size_t iterate_persistent_ws_bytes(int r, int ell) {
  const size_t ea = ea_size(r, ell), eb = eb_size(r, ell);
  return sizeof(float) * kCopies * 2 * (ea + eb) + sizeof(Barrier) + 2 * sizeof(int) + 1024;
}

bool iterate_persistent_supported(int64_t m, int64_t n, int r, int ell) {
  const int grid = num_sms();
  const int64_t rb = (m + grid - 1) / grid, cbk = (n + grid - 1) / grid;
  return r <= 32 && rb <= kMaxRows && cbk <= kMaxCols &&
         smem_for(32, ell, static_cast<int>(rb), static_cast<int>(cbk)) <= 220 * 1024;
}

cudaError_t launch_iterate_persistent(const Launcher& L, const IterArgs& ia, int iters, void* ws,
                                      size_t ws_bytes, int* status, float* mon, const int* done) {
  if (ws_bytes < iterate_persistent_ws_bytes(ia.r, ia.ell)) return cudaErrorInvalidValue;
  if (!iterate_persistent_supported(ia.m, ia.n, ia.r, ia.ell)) return cudaErrorInvalidValue;
  if (iters <= 0) return cudaSuccess;
  char* p = static_cast<char*>(ws);
  const size_t ea = ea_size(ia.r, ia.ell), eb = eb_size(ia.r, ia.ell);
  const int grid = num_sms();
  PArgs a;
  a.m = ia.m;
  a.n = ia.n;
  a.r = ia.r;
  a.ell = ia.ell;
  a.iters = iters;
  a.rule = ia.rule;
  a.alpha = ia.alpha;
  a.beta = ia.beta;
  a.eps = ia.eps;
  a.QL = ia.QL;
  a.QR = ia.QR;
  a.Xhat = ia.Xhat;
  a.Xchk = ia.Xchk;
  a.W = ia.W;
  a.H = ia.H;
  a.accA = reinterpret_cast<float*>(p);
  a.accB = a.accA + 2 * kCopies * ea;
  a.bar = reinterpret_cast<Barrier*>(a.accB + 2 * kCopies * eb);
  a.abort_flag = reinterpret_cast<int*>(a.bar + 1);
  a.status = status;
  a.mon = mon;
  a.done = done;
  const size_t clear = reinterpret_cast<char*>(a.abort_flag + 1) - p;
  cudaError_t err = cudaMemsetAsync(ws, 0, clear, L.stream);
  if (err != cudaSuccess) return err;
  a.RB = static_cast<int>((ia.m + grid - 1) / grid);
  a.CB = static_cast<int>((ia.n + grid - 1) / grid);
  const bool mu = ia.rule != 0;
  if (ia.r <= 8) return mu ? launch<2, 1, 1>(L, a, grid) : launch<2, 1, 0>(L, a, grid);
  if (ia.r <= 16) return mu ? launch<4, 1, 1>(L, a, grid) : launch<4, 1, 0>(L, a, grid);
  if (ia.r <= 24) return mu ? launch<6, 2, 1>(L, a, grid) : launch<6, 2, 0>(L, a, grid);
  return mu ? launch<8, 2, 1>(L, a, grid) : launch<8, 2, 0>(L, a, grid);
}

}  // namespace nmfrp
