// All iterations of FastHALS-RP / MU-RP in one cooperative (persistent) launch.
//
// The update rules are those of k_iterate.cu (Section 4, Eq. fastHALS_a with the Section 4.1
// terms; Section 3.1, Algorithm 3 with the semi-NMF rule). Each block owns a fixed slice of the
// rows of W and of the columns of H for the whole run; the slice's rows of X_chk and Q_L, its
// columns of X_hat and rows of Q_R, and its rows of W and columns of H live in shared memory
// across iterations. One iteration:
//
//   A  (rows of W)    H_tld from the cross-block sums; G_W = H_tld H_tld^T; per row: S_W row,
//                     Gauss-Seidel sweep over j; then the block's share of
//                     [Q_L | W]^T W  (W_tld_raw = Q_L^T W and W^T W, whose diagonal holds the
//                     squared column norms) is added into the cross-block sums.
//   -- grid barrier --
//   B  (columns of H) s_j = ||w_j||, W_tld = raw / s, G_H = W_tld^T W_tld; per column: h_j *= s_j
//                     (the normalisation moved to H), S_H column, sweep; then the block's share of
//                     H^T [Q_R | H]  (H_tld and H H^T) and of <S_H, H> is added.
//   -- grid barrier --
//
// A group of lanes handles one or more rows of W (columns of H); each lane owns a contiguous run
// of the components, so every shared-memory read of a Gram row or of H_tld / W_tld is a
// broadcast vector load that serves all the group's rows (Lanes<RP> below). The sweep is incremental: t_j = S_j - sum_q w_q
// G_qj is formed for every j; when w_j moves by d (computed by the lane owning j, broadcast in
// the group) every t_j' drops by d G_jj' (those with j' <= j are never read again, so they are
// updated too instead of being masked). These are the Gauss-Seidel values of the paper's
// component-by-component update.
//
// The per-element scalings use reciprocals formed once per phase (an IEEE division per element of
// a row cost as much as the row's whole S product).
//
// Block shares of the cross-block sums are register-tiled (4 x 4 outputs a thread, the rows of
// the slice split over thread groups) and summed in a fixed order in shared memory, then added
// with vector FP32 atomics into kCopies copies (block b into copy b % kCopies); readers sum the
// copies in a fixed order through L2. The order of the atomics within a copy varies from run to
// run, so results can differ in the last bits between runs.
//
// Error monitor (no read of X): after the last iteration the kernel leaves in mon[0] the cross
// term <W_tld^T X_hat, H> and in mon[1] the quadratic term <W^T W, H H^T>; with ||X||^2 they give
// ||X - W H||^2 ~ ||X||^2 - 2 mon[0] + mon[1] (X replaced by Q_L Q_L^T X in the cross term,
// Section 3 Eq. 3.4).
//
// If *done is set on entry (an earlier residual check reached the target) the kernel returns at
// once. Every wait is bounded: on time-out the kernel latches NMF_ERR_TIMEOUT and all blocks leave.
//
// Gated launches (the solve's loop): the launch continues from the iteration count left in
// solve[6] and runs until an exact residual check is due. At every residual_every-th iteration
// each block forms the monitor's estimate of the relative error from the sums (the same values
// in every block, so every block takes the same decision) and compares it with the target as
// the solve's gate does; the last iteration of the budget is always checked. The launch then
// stops, leaving the count in solve[6], the estimate in solve[4] and the gate flag set, for the
// exact residual and the decision that follow it in the stream. Checks the monitor rules out
// cost a few microseconds inside the kernel instead of a return to the host and a relaunch.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kNT = 512;          // threads per block (one block per SM)
constexpr int kCopies = 4;        // copies of each cross-block sum
constexpr long long kWaitCycles = 4000000000LL;   // about two seconds of polling

struct Barrier {
  unsigned int count;   // arrivals so far (never reset within a launch)
  unsigned int pad;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide barrier for a co-resident grid: the k-th barrier of the launch completes when the
// arrival counter reaches k * nblocks (one acquire-release add per block, acquire polling).
// The block barrier before the add orders the block's writes and atomics before it, and the
// release of the add is cumulative over them; the acquire of the last poll, followed by the
// block barrier, orders every thread's later reads after the other blocks' writes. No separate
// fence is needed (two full fences here cost 1.1 us an iteration). Returns false if the wait ran
// out.
__device__ bool grid_sync(Barrier* bar, unsigned nblocks, unsigned& epoch, int* status,
                          int* abort_flag, long long wait_cycles) {
  __syncthreads();
  __shared__ int ok;
  ++epoch;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned target = epoch * nblocks;
    const unsigned before = atom_add_acq_rel(&bar->count, 1u);
    if (before + 1 < target) {
      const long long t0 = clock64();
      while (static_cast<int>(ld_acquire(&bar->count) - target) < 0) {
        if (clock64() - t0 > wait_cycles || *reinterpret_cast<volatile int*>(abort_flag)) {
          ok = 0;
          break;
        }
      }
      if (!ok) {
        latch(status, kStTimeout);
        atomicExch(abort_flag, 1);
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ float posp(float v) { return v > 0.f ? v : 0.f; }
__device__ __forceinline__ float negp(float v) { return v < 0.f ? -v : 0.f; }

// ell padded to a multiple of 4, and the row stride of staged rows (a multiple of 4 whose
// quarter is odd: rows read as float4 by consecutive threads hit distinct banks).
__host__ __device__ __forceinline__ int lq_of(int ell) { return (ell + 3) & ~3; }
__host__ __device__ __forceinline__ int lsx_of(int ell) {
  const int s = lq_of(ell);
  return ((s / 4) % 2 == 0) ? s + 4 : s;
}
// cross-block sum sizes: phase A [LQ + RP][RP]; phase B [RP][LQ + RP] + cross (padded to 4)
__host__ __device__ __forceinline__ int ea_size(int RP, int LQ) { return (LQ + RP) * RP; }
__host__ __device__ __forceinline__ int eb_size(int RP, int LQ) { return RP * (LQ + RP) + 4; }

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
  float* accA;    // [2][kCopies][EA]
  float* accB;    // [2][kCopies][EB]
  float* mon;     // [2]: cross term and quadratic term of the last iteration
  const int* done;
  Barrier* bar;
  int* status;
  int* abort_flag;
  long long wait_cycles;   // polling budget of each grid barrier wait (SM clock cycles)
};

// Fixed-order sum of the kCopies copies of entry e, read through L2.
__device__ __forceinline__ float acc_read(const float* base, int E, int e) {
  float v[kCopies];
#pragma unroll
  for (int c = 0; c < kCopies; ++c) v[c] = __ldcg(base + c * E + e);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kCopies; ++c) s += v[c];
  return s;
}

// out[a][b] += sum_{i < K} A_i[a] B_i[b] (a < NA, b < NB, both multiples of 4), added with vector
// atomics into `dst` (row-major NA x NB). Row i of A is A1[i * lda1 + a] for a < NA1 and
// A2[i * lda2 + a - NA1] beyond; B likewise with NB1. `red` holds kNT * 16 floats.
__device__ void block_share(int K, int NA, int NB, const float* A1, int lda1, const float* A2,
                            int lda2, int NA1, const float* B1, int ldb1, const float* B2,
                            int ldb2, int NB1, float* red, float* dst) {
  const int t = threadIdx.x;
  const int tb = NB / 4, tiles = (NA / 4) * tb;
  int ks = kNT / tiles;
  if (ks < 1) ks = 1;
  const int chunk = (K + ks - 1) / ks;
  for (int u = t; u < tiles * ks; u += kNT) {
    const int tile = u % tiles, kk = u / tiles;
    const int a0 = 4 * (tile / tb), b0 = 4 * (tile % tb);
    const float* pa = a0 < NA1 ? A1 + a0 : A2 + (a0 - NA1);
    const float* pb = b0 < NB1 ? B1 + b0 : B2 + (b0 - NB1);
    const int lda = a0 < NA1 ? lda1 : lda2, ldb = b0 < NB1 ? ldb1 : ldb2;
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
    const int i1 = min(K, (kk + 1) * chunk);
#pragma unroll 2
    for (int i = kk * chunk; i < i1; ++i) {
      const float4 av = *reinterpret_cast<const float4*>(pa + i * lda);
      const float4 bv = *reinterpret_cast<const float4*>(pb + i * ldb);
      const float aa[4] = {av.x, av.y, av.z, av.w};
      const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(aa[x], bb[y], acc[x][y]);
    }
    float* rp = red + (static_cast<size_t>(kk) * NA + a0) * NB + b0;
#pragma unroll
    for (int x = 0; x < 4; ++x)
      *reinterpret_cast<float4*>(rp + x * NB) = make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
  }
  __syncthreads();
  const int q4 = NA * NB / 4;
  for (int q = t; q < q4; q += kNT) {
    float4 s = *reinterpret_cast<const float4*>(red + 4 * q);
    for (int kk = 1; kk < ks; ++kk) {
      const float4 v = *reinterpret_cast<const float4*>(red + static_cast<size_t>(kk) * NA * NB + 4 * q);
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    atomicAdd(reinterpret_cast<float4*>(dst + 4 * q), s);
  }
}

// G[p][q] = sum_k T[k][p] T[k][q] (RP x RP) from T (LQ x RP); inv[j] = 1 / G[j][j] where
// G[j][j] > 0, else 0. The 2 x 2 tiles of the upper triangle are computed over KS ranges of k
// by different threads (partials in `red`, at least kNT * 4 floats), summed in a fixed order,
// and mirrored. Ends with a block barrier.
template <int RP>
__device__ __forceinline__ void gram_rp(const float* T, int LQ, float* G, float* inv, float* red) {
  constexpr int T2 = RP / 2, NT = T2 * (T2 + 1) / 2;
  constexpr int KS0 = kNT / NT < 1 ? 1 : kNT / NT;
  const int ks_cap = (LQ + 3) / 4;   // at least four k a range
  const int KS = KS0 < ks_cap ? KS0 : ks_cap;
  const int chunk = (LQ + KS - 1) / KS;
  for (int u = threadIdx.x; u < NT * KS; u += kNT) {
    const int tile = u % NT, kk = u / NT;
    int P = 0, v = tile;
    while (v >= T2 - P) {
      v -= T2 - P;
      ++P;
    }
    const int p0 = 2 * P, q0 = 2 * (P + v);
    float g00 = 0.f, g01 = 0.f, g10 = 0.f, g11 = 0.f;
    const int k1 = min(LQ, (kk + 1) * chunk);
#pragma unroll 4
    for (int k = kk * chunk; k < k1; ++k) {
      const float2 a = *reinterpret_cast<const float2*>(T + k * RP + p0);
      const float2 b = *reinterpret_cast<const float2*>(T + k * RP + q0);
      g00 = fmaf(a.x, b.x, g00);
      g01 = fmaf(a.x, b.y, g01);
      g10 = fmaf(a.y, b.x, g10);
      g11 = fmaf(a.y, b.y, g11);
    }
    *reinterpret_cast<float4*>(red + 4 * u) = make_float4(g00, g01, g10, g11);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NT * 4; e += kNT) {
    const int tile = e >> 2, x = e & 3;
    float g = red[4 * tile + x];
    for (int kk = 1; kk < KS; ++kk) g += red[4 * (kk * NT + tile) + x];
    int P = 0, v = tile;
    while (v >= T2 - P) {
      v -= T2 - P;
      ++P;
    }
    if (v == 0 && x == 2) continue;   // the mirror of entry 1 of a diagonal tile
    const int p = 2 * P + (x >> 1), q = 2 * (P + v) + (x & 1);
    G[p * RP + q] = g;
    G[q * RP + p] = g;
    if (p == q) inv[p] = g > 0.f ? 1.f / g : 0.f;
  }
}

// gram_rp on threads [b0, b0 + nthr) of the block (whole warps; `tid` = threadIdx.x - b0), with
// the named barrier `bar` among them in place of the block barrier, so that the block's other
// warps can run the sweep's first half meanwhile. Same sums as gram_rp, split over fewer
// threads (so in another order). The caller ends with a block barrier.
template <int RP>
__device__ __forceinline__ void gram_rp_sub(const float* T, int LQ, float* G, float* inv,
                                            float* red, int tid, int nthr, int bar) {
  constexpr int T2 = RP / 2, NT = T2 * (T2 + 1) / 2;
  const int KS0 = nthr / NT < 1 ? 1 : nthr / NT;
  const int ks_cap = (LQ + 3) / 4;
  const int KS = KS0 < ks_cap ? KS0 : ks_cap;
  const int chunk = (LQ + KS - 1) / KS;
  for (int u = tid; u < NT * KS; u += nthr) {
    const int tile = u % NT, kk = u / NT;
    int P = 0, v = tile;
    while (v >= T2 - P) {
      v -= T2 - P;
      ++P;
    }
    const int p0 = 2 * P, q0 = 2 * (P + v);
    float g00 = 0.f, g01 = 0.f, g10 = 0.f, g11 = 0.f;
    const int k1 = min(LQ, (kk + 1) * chunk);
#pragma unroll 4
    for (int k = kk * chunk; k < k1; ++k) {
      const float2 a = *reinterpret_cast<const float2*>(T + k * RP + p0);
      const float2 b = *reinterpret_cast<const float2*>(T + k * RP + q0);
      g00 = fmaf(a.x, b.x, g00);
      g01 = fmaf(a.x, b.y, g01);
      g10 = fmaf(a.y, b.x, g10);
      g11 = fmaf(a.y, b.y, g11);
    }
    *reinterpret_cast<float4*>(red + 4 * u) = make_float4(g00, g01, g10, g11);
  }
  asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
  for (int e = tid; e < NT * 4; e += nthr) {
    const int tile = e >> 2, x = e & 3;
    float g = red[4 * tile + x];
    for (int kk = 1; kk < KS; ++kk) g += red[4 * (kk * NT + tile) + x];
    int P = 0, v = tile;
    while (v >= T2 - P) {
      v -= T2 - P;
      ++P;
    }
    if (v == 0 && x == 2) continue;   // the mirror of entry 1 of a diagonal tile
    const int p = 2 * P + (x >> 1), q = 2 * (P + v) + (x & 1);
    G[p * RP + q] = g;
    G[q * RP + p] = g;
    if (p == q) inv[p] = g > 0.f ? 1.f / g : 0.f;
  }
}

// C consecutive floats from shared memory (C a multiple of 2; float4 where it can).
template <int C>
__device__ __forceinline__ void ld_run(const float* p, float* v) {
  static_assert(C % 2 == 0, "runs are read as float2 / float4");
  if constexpr (C % 4 == 0) {
#pragma unroll
    for (int c = 0; c < C; c += 4) {
      const float4 x = *reinterpret_cast<const float4*>(p + c);
      v[c] = x.x;
      v[c + 1] = x.y;
      v[c + 2] = x.z;
      v[c + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < C; c += 2) {
      const float2 x = *reinterpret_cast<const float2*>(p + c);
      v[c] = x.x;
      v[c + 1] = x.y;
    }
  }
}

// One group of NG lanes updates R factor vectors at once (rows of W, or columns of H): vector rho
// has RP components, lane g owning [g C, g C + C), its cross products in s[rho] (S_j for the
// owned j). Every Gram row read from shared memory serves the R vectors. For FastHALS-RP on H
// (reg = true) the Section 4.1 alpha / beta form is used. Components j >= r are zero on entry
// and stay zero.
template <int RP, int NG, int R, int RULE>
__device__ __forceinline__ void update_rows(float (&v)[R][RP / NG], float (&s)[R][RP / NG],
                                            const float* G, const float* inv, int g, int r,
                                            bool reg, float alpha, float beta, float eps) {
  constexpr int C = RP / NG;
  const unsigned full = 0xffffffffu;
  if (RULE == 0 && NG == 2) {
    // Two lanes a vector (lane g owns components g C .. g C + C - 1). Each step's update is
    // formed by both lanes from their own component cj and kept by the owner only (no divergent
    // branch on the dependency chain: the diagonal loads do not wait for it), and one XOR
    // shuffle hands the partner's values over. Steps j >= r are skipped.
    // t_j = S_j - sum_q v_q G[q][j]: own q from registers, the partner's by one shuffle each
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {   // own component rows, then the partner's
      const int src = half ? (g ^ 1) : g;
#pragma unroll
      for (int q = 0; q < C; ++q) {
        float gr[C];
        ld_run<C>(G + (src * C + q) * RP + g * C, gr);
#pragma unroll
        for (int rho = 0; rho < R; ++rho) {
          const float vm = v[rho][q];
          const float vq = half ? __shfl_xor_sync(full, vm, 1) : vm;
#pragma unroll
          for (int c = 0; c < C; ++c) s[rho][c] = fmaf(-vq, gr[c], s[rho][c]);
        }
      }
    }
#pragma unroll 1
    for (int o = 0; o < 2; ++o) {
      const bool own = g == o;
#pragma unroll
      for (int cj = 0; cj < C; ++cj) {
        const int j = o * C + cj;
        if (j >= r) break;
        const int jm = g * C + cj;   // this lane's component at step position cj
        const float gjj = G[jm * RP + jm], ij = inv[jm];
        float gr[C];
        ld_run<C>(G + j * RP + g * C, gr);
#pragma unroll
        for (int rho = 0; rho < R; ++rho) {
          const float vo = v[rho][cj];
          float vn = vo;
          if (!reg) {
            if (gjj > 0.f) vn = fmaxf(0.f, fmaf(s[rho][cj], ij, vo));
          } else if (gjj + beta > 0.f) {
            vn = fmaxf(0.f, (fmaf(vo, gjj, s[rho][cj]) - alpha) / (gjj + beta));
          }
          const float dl = own ? vn - vo : 0.f;
          v[rho][cj] = own ? vn : vo;
          const float dd = dl + __shfl_xor_sync(full, dl, 1);
#pragma unroll
          for (int c = 0; c < C; ++c) s[rho][c] = fmaf(-dd, gr[c], s[rho][c]);
        }
      }
    }
  } else if (RULE == 0) {
    // t_j = S_j - sum_q v_q G[q][j]
#pragma unroll 1
    for (int o = 0; o < NG; ++o) {
#pragma unroll
      for (int cq = 0; cq < C; ++cq) {
        float gr[C];
        ld_run<C>(G + (o * C + cq) * RP + g * C, gr);
#pragma unroll
        for (int rho = 0; rho < R; ++rho) {
          const float vq = __shfl_sync(full, v[rho][cq], o, NG);
#pragma unroll
          for (int c = 0; c < C; ++c) s[rho][c] = fmaf(-vq, gr[c], s[rho][c]);
        }
      }
    }
#pragma unroll 1
    for (int o = 0; o < NG; ++o) {
#pragma unroll
      for (int cj = 0; cj < C; ++cj) {
        const int j = o * C + cj;
        float d[R];
#pragma unroll
        for (int rho = 0; rho < R; ++rho) d[rho] = 0.f;
        if (g == o && j < r) {
          const float gjj = G[j * RP + j], ij = inv[j];
#pragma unroll
          for (int rho = 0; rho < R; ++rho) {
            float vn = v[rho][cj];
            if (!reg) {
              if (gjj > 0.f) vn = fmaxf(0.f, fmaf(s[rho][cj], ij, v[rho][cj]));
            } else if (gjj + beta > 0.f) {
              vn = fmaxf(0.f, (fmaf(v[rho][cj], gjj, s[rho][cj]) - alpha) / (gjj + beta));
            }
            d[rho] = vn - v[rho][cj];
            v[rho][cj] = vn;
          }
        }
        float gr[C];
        ld_run<C>(G + j * RP + g * C, gr);
#pragma unroll
        for (int rho = 0; rho < R; ++rho) {
          const float dd = __shfl_sync(full, d[rho], o, NG);
#pragma unroll
          for (int c = 0; c < C; ++c) s[rho][c] = fmaf(-dd, gr[c], s[rho][c]);
        }
      }
    }
  } else {
    float num[R][C], den[R][C];
#pragma unroll
    for (int rho = 0; rho < R; ++rho)
#pragma unroll
      for (int c = 0; c < C; ++c) {
        num[rho][c] = posp(s[rho][c]);
        den[rho][c] = negp(s[rho][c]) + eps;
      }
#pragma unroll 1
    for (int o = 0; o < NG; ++o) {
#pragma unroll
      for (int cq = 0; cq < C; ++cq) {
        float gr[C];
        ld_run<C>(G + (o * C + cq) * RP + g * C, gr);
#pragma unroll
        for (int rho = 0; rho < R; ++rho) {
          const float vq = __shfl_sync(full, v[rho][cq], o, NG);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            num[rho][c] = fmaf(vq, negp(gr[c]), num[rho][c]);
            den[rho][c] = fmaf(vq, posp(gr[c]), den[rho][c]);
          }
        }
      }
    }
#pragma unroll
    for (int rho = 0; rho < R; ++rho)
#pragma unroll
      for (int c = 0; c < C; ++c)
        v[rho][c] = (g * C + c < r) ? v[rho][c] * sqrtf(num[rho][c] / den[rho][c]) : 0.f;
  }
}

// The whole run for one problem, executed by `G` co-resident blocks of which this is block
// `bid` (all blocks of a problem call it with the same arguments).
template <int RP, int RULE, int GA, int RA, int GB, int RC>
__device__ __forceinline__ void iterate_body(const PArgs& a, const SolveGate& g,
                                             const unsigned bid, const unsigned G, float* sh) {
  constexpr int CA = RP / GA, CBn = RP / GB;
  const int r = a.r, ell = a.ell, t = threadIdx.x;
  const int LQ = lq_of(ell), LS = lsx_of(ell);
  const int EA = ea_size(RP, LQ), EB = eb_size(RP, LQ);
  const int RB = a.RB, CB = a.CB;
  float* HtT = sh;                  // [LQ][RP]   H_tld^T
  float* Gw = HtT + LQ * RP;        // [RP][RP]
  float* WtS = Gw + RP * RP;        // [LQ][RP]   W_tld (normalised)
  float* Gh = WtS + LQ * RP;        // [RP][RP]
  float* sc = Gh + RP * RP;         // [RP]       s_j of the last W phase
  float* invs = sc + RP;            // [RP]       1 / G_jj of the current phase
  float* rsc = invs + RP;           // [RP]       1 / s_j
  float* Ws = rsc + RP;             // [RB][RP]   rows of W (unnormalised)
  float* Hs = Ws + RB * RP;         // [CB][RP]   columns of H
  float* Xc = Hs + CB * RP;         // [RB][LS]   rows of X_chk
  float* Ql = Xc + RB * LS;         // [RB][LS]   rows of Q_L
  float* Xh = Ql + RB * LS;         // [CB][LS]   columns of X_hat
  float* Qr = Xh + CB * LS;         // [CB][LS]   rows of Q_R
  float* red = Qr + CB * LS;        // [kNT * 16] block-share scratch
  __shared__ float wred[kNT / 32];
  const int64_t r0 = static_cast<int64_t>(bid) * RB, c0 = static_cast<int64_t>(bid) * CB;
  const int nrows = r0 < a.m ? static_cast<int>(a.m - r0 < RB ? a.m - r0 : RB) : 0;
  const int ncols = c0 < a.n ? static_cast<int>(a.n - c0 < CB ? a.n - c0 : CB) : 0;
  const bool normalize = (RULE == 0);
  const bool reg = !(a.alpha == 0.f && a.beta == 0.f);

  const bool gated = g.every > 0;
  // iterations of this launch: a.iters, or (gated) what the budget leaves after solve[6]
  const int start =
      gated ? static_cast<int>(*reinterpret_cast<const volatile double*>(g.solve + 6)) : 0;
  const int n_it = gated ? g.total - start : a.iters;
  if (*reinterpret_cast<const volatile int*>(a.done) || n_it <= 0) {   // converged, or done
    if (gated && bid == 0 && t == 0) g.flags[1] = 0;
    return;
  }
  unsigned epoch = 0;
  __shared__ int gate_sh;
  __shared__ double est_sh;
  // monitor terms of the iteration whose sums sit in buffers phm: the cross term and
  // <W^T W, H H^T> for the normalised W; every thread of the block gets both (fixed-order sums)
  auto monitor = [&](int phm, float& cross, float& quad) {
    const float* accA_r = a.accA + phm * kCopies * EA;
    const float* accB_r = a.accB + phm * kCopies * EB;
    float q2 = 0.f;
    for (int e = t; e < RP * RP; e += kNT) {
      const int p = e / RP, q = e - p * RP;
      const float gww = acc_read(accA_r, EA, (LQ + p) * RP + q) / (sc[p] * sc[q]);
      q2 = fmaf(gww, acc_read(accB_r, EB, p * (LQ + RP) + LQ + q), q2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
    if ((t & 31) == 0) wred[t >> 5] = q2;
    __syncthreads();
    float sum = 0.f;
    for (int wI = 0; wI < kNT / 32; ++wI) sum += wred[wI];
    __syncthreads();
    cross = acc_read(accB_r, EB, RP * (LQ + RP));
    quad = sum;
  };

  // ---- stage the slice (zero-padded) and the factors
  for (int j = t; j < RP; j += kNT) {
    sc[j] = 1.f;
    rsc[j] = 1.f;
  }
  for (int e = t; e < RB * RP; e += kNT) {
    const int i = e / RP, j = e - i * RP;
    Ws[e] = (i < nrows && j < r) ? a.W[(r0 + i) * r + j] : 0.f;
  }
  for (int e = t; e < CB * RP; e += kNT) {
    const int c = e / RP, j = e - c * RP;
    Hs[e] = (c < ncols && j < r) ? a.H[static_cast<int64_t>(j) * a.n + c0 + c] : 0.f;
  }
  for (int e = t; e < RB * LS; e += kNT) {
    const int i = e / LS, k = e - i * LS;
    const bool in = i < nrows && k < ell;
    Xc[e] = in ? a.Xchk[(r0 + i) * ell + k] : 0.f;
    Ql[e] = in ? a.QL[(r0 + i) * ell + k] : 0.f;
  }
  for (int e = t; e < CB * LS; e += kNT) {
    const int c = e / LS, k = e - c * LS;
    const bool in = c < ncols && k < ell;
    Xh[e] = in ? a.Xhat[static_cast<int64_t>(k) * a.n + c0 + c] : 0.f;
    Qr[e] = in ? a.QR[(c0 + c) * ell + k] : 0.f;
  }
  __syncthreads();
  // prologue: H_tld, H H^T of the initial H into accB[1]
  block_share(CB, RP, LQ + RP, Hs, RP, Hs, RP, RP, Qr, LS, Hs, RP, LQ, red,
              a.accB + (1 * kCopies + bid % kCopies) * EB);
  if (!grid_sync(a.bar, G, epoch, a.status, a.abort_flag, a.wait_cycles)) return;

  int ran = n_it;
  for (int step = 0; step < n_it; ++step) {
    const int ph = step & 1, pr = ph ^ 1;
    const int it = start + step;   // iterations before this one
    // ================= phase A: rows of W
    {
      const float* accB_r = a.accB + pr * kCopies * EB;
      for (int e = t; e < RP * LQ; e += kNT) {
        const int j = e / LQ, k = e - j * LQ;
        HtT[k * RP + j] = acc_read(accB_r, EB, j * (LQ + RP) + k);
      }
    }
    __syncthreads();
    {
      // group q of GA lanes takes the RA rows q, q + Q, q + 2Q, ... (Q = ceil(nrows / RA)), so
      // that neighbouring groups read neighbouring rows; whole warps run (shuffles), groups
      // past the slice compute on a valid row and store nothing. When the groups fit in one
      // pass with warps to spare, the spare warps form G_W while the others form their rows of
      // S_W (the first half of the sweep); otherwise G_W comes first.
      constexpr int GPW = 32 / GA;
      const int Q = (nrows + RA - 1) / RA;
      const int Qp = (Q + GPW - 1) / GPW * GPW;
      const int busy = Qp * GA;
      const bool overlap = RULE == 0 && Qp <= kNT / GA && busy + 64 <= kNT;
      const int g = t % GA;
      int idx[RA];
      bool live[RA];
      float w[RA][CA], sv[RA][CA];
      auto load_rows = [&](int q) {
#pragma unroll
        for (int rho = 0; rho < RA; ++rho) {
          const int row = q + rho * Q;
          live[rho] = q < Q && row < nrows;
          idx[rho] = live[rho] ? row : 0;
        }
#pragma unroll
        for (int rho = 0; rho < RA; ++rho) {
          ld_run<CA>(Ws + idx[rho] * RP + g * CA, w[rho]);
#pragma unroll
          for (int c = 0; c < CA; ++c) {
            w[rho][c] *= rsc[g * CA + c];   // normalisation of the previous W phase
            sv[rho][c] = 0.f;
          }
        }
        for (int k = 0; k < LQ; k += 4) {
          float xk[RA][4];
#pragma unroll
          for (int rho = 0; rho < RA; ++rho) {
            const float4 x4 = *reinterpret_cast<const float4*>(Xc + idx[rho] * LS + k);
            xk[rho][0] = x4.x;
            xk[rho][1] = x4.y;
            xk[rho][2] = x4.z;
            xk[rho][3] = x4.w;
          }
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            float hr[CA];
            ld_run<CA>(HtT + (k + q4) * RP + g * CA, hr);
#pragma unroll
            for (int rho = 0; rho < RA; ++rho)
#pragma unroll
              for (int c = 0; c < CA; ++c) sv[rho][c] = fmaf(xk[rho][q4], hr[c], sv[rho][c]);
          }
        }
      };
      auto update_store = [&]() {
        update_rows<RP, GA, RA, RULE>(w, sv, Gw, invs, g, r, false, 0.f, 0.f, a.eps);
#pragma unroll
        for (int rho = 0; rho < RA; ++rho)
          if (live[rho]) {
#pragma unroll
            for (int c = 0; c < CA; c += 2)
              *reinterpret_cast<float2*>(Ws + idx[rho] * RP + g * CA + c) =
                  make_float2(w[rho][c], w[rho][c + 1]);
          }
      };
      if (overlap) {
        if (t < busy) load_rows(t / GA);
        else gram_rp_sub<RP>(HtT, LQ, Gw, invs, red, t - busy, kNT - busy, 1);
        __syncthreads();
        if (t < busy) update_store();
      } else {
        gram_rp<RP>(HtT, LQ, Gw, invs, red);
        __syncthreads();
        for (int q = t / GA; q < Qp; q += kNT / GA) {
          load_rows(q);
          update_store();
        }
      }
    }
    __syncthreads();
    // [Q_L | W]^T W over the slice
    block_share(RB, LQ + RP, RP, Ql, LS, Ws, RP, LQ, Ws, RP, Ws, RP, RP, red,
                a.accA + (ph * kCopies + bid % kCopies) * EA);
    if (!grid_sync(a.bar, G, epoch, a.status, a.abort_flag, a.wait_cycles)) return;

    // ================= phase B: columns of H
    // the previous iteration's sums are read for the last time in phase A (and by a gated
    // launch's check after it): clear them for the next iteration
    for (int64_t e = static_cast<int64_t>(bid) * kNT + t; e < kCopies * EB;
         e += static_cast<int64_t>(G) * kNT)
      a.accB[pr * kCopies * EB + e] = 0.f;
    for (int64_t e = static_cast<int64_t>(bid) * kNT + t; e < kCopies * EA;
         e += static_cast<int64_t>(G) * kNT)
      a.accA[pr * kCopies * EA + e] = 0.f;
    {
      const float* accA_r = a.accA + ph * kCopies * EA;
      for (int j = t; j < RP; j += kNT) {
        const float c2 = acc_read(accA_r, EA, (LQ + j) * RP + j);
        const float sj = (normalize && j < r && c2 > 0.f) ? sqrtf(c2) : 1.f;
        sc[j] = sj;
        rsc[j] = 1.f / sj;
      }
      __syncthreads();
      for (int e = t; e < LQ * RP; e += kNT) WtS[e] = acc_read(accA_r, EA, e) * rsc[e % RP];
    }
    __syncthreads();
    float cross = 0.f;
    {
      // as in phase A: spare warps form G_H while the others form their columns of S_H
      constexpr int GPW = 32 / GB;
      const int Q = (ncols + RC - 1) / RC;
      const int Qp = (Q + GPW - 1) / GPW * GPW;
      const int busy = Qp * GB;
      const bool overlap = RULE == 0 && Qp <= kNT / GB && busy + 64 <= kNT;
      const int g = t % GB;
      int idx[RC];
      bool live[RC];
      float h[RC][CBn], sv[RC][CBn];
      auto load_cols = [&](int q) {
#pragma unroll
        for (int rho = 0; rho < RC; ++rho) {
          const int col = q + rho * Q;
          live[rho] = q < Q && col < ncols;
          idx[rho] = live[rho] ? col : 0;
        }
#pragma unroll
        for (int rho = 0; rho < RC; ++rho) {
          ld_run<CBn>(Hs + idx[rho] * RP + g * CBn, h[rho]);
#pragma unroll
          for (int z = 0; z < CBn; ++z) {
            h[rho][z] *= sc[g * CBn + z];
            sv[rho][z] = 0.f;
          }
        }
        for (int k = 0; k < LQ; k += 4) {
          float xk[RC][4];
#pragma unroll
          for (int rho = 0; rho < RC; ++rho) {
            const float4 x4 = *reinterpret_cast<const float4*>(Xh + idx[rho] * LS + k);
            xk[rho][0] = x4.x;
            xk[rho][1] = x4.y;
            xk[rho][2] = x4.z;
            xk[rho][3] = x4.w;
          }
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            float wr[CBn];
            ld_run<CBn>(WtS + (k + q4) * RP + g * CBn, wr);
#pragma unroll
            for (int rho = 0; rho < RC; ++rho)
#pragma unroll
              for (int z = 0; z < CBn; ++z) sv[rho][z] = fmaf(xk[rho][q4], wr[z], sv[rho][z]);
          }
        }
      };
      auto update_store = [&]() {
        float shc[RC][CBn];
#pragma unroll
        for (int rho = 0; rho < RC; ++rho)
#pragma unroll
          for (int z = 0; z < CBn; ++z) shc[rho][z] = sv[rho][z];   // S_H for the monitor
        update_rows<RP, GB, RC, RULE>(h, sv, Gh, invs, g, r, RULE == 0 && reg, a.alpha, a.beta,
                                      a.eps);
#pragma unroll
        for (int rho = 0; rho < RC; ++rho)
          if (live[rho]) {
#pragma unroll
            for (int z = 0; z < CBn; ++z) cross = fmaf(shc[rho][z], h[rho][z], cross);
#pragma unroll
            for (int z = 0; z < CBn; z += 2)
              *reinterpret_cast<float2*>(Hs + idx[rho] * RP + g * CBn + z) =
                  make_float2(h[rho][z], h[rho][z + 1]);
          }
      };
      if (overlap) {
        if (t < busy) load_cols(t / GB);
        else gram_rp_sub<RP>(WtS, LQ, Gh, invs, red, t - busy, kNT - busy, 1);
        __syncthreads();
        if (t < busy) update_store();
      } else {
        gram_rp<RP>(WtS, LQ, Gh, invs, red);
        __syncthreads();
        for (int q = t / GB; q < Qp; q += kNT / GB) {
          load_cols(q);
          update_store();
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cross += __shfl_xor_sync(0xffffffffu, cross, o);
    if ((t & 31) == 0) wred[t >> 5] = cross;
    __syncthreads();
    float* accB_w = a.accB + (ph * kCopies + bid % kCopies) * EB;
    block_share(CB, RP, LQ + RP, Hs, RP, Hs, RP, RP, Qr, LS, Hs, RP, LQ, red, accB_w);
    if (t == 0) {
      float csum = 0.f;
      for (int wI = 0; wI < kNT / 32; ++wI) csum += wred[wI];
      atomicAdd(&accB_w[RP * (LQ + RP)], csum);
    }
    if (!grid_sync(a.bar, G, epoch, a.status, a.abort_flag, a.wait_cycles)) return;
    if (gated && ((it + 1) % g.every == 0 || it + 1 == g.total)) {
      // the solve's gate on the monitor, in every block; the sums of buffers ph stay intact
      // until phase B of the next iteration, past a grid barrier
      float cross, quad;
      monitor(ph, cross, quad);
      if (t == 0) {
        const double x2 = g.solve[0];
        const double e2 =
            x2 - 2.0 * (static_cast<double>(cross) + g.solve[3]) + static_cast<double>(quad);
        const double est = x2 > 0.0 ? sqrt(fmax(e2, 0.0) / x2) : 0.0;
        int check = 1;
        if (it + 1 < g.total && g.target > 0.0) {
          const double cal = g.solve[5];
          check = cal > 0.0 ? (est * cal <= g.target * (1.0 + g.margin_cal))
                            : (est <= g.target * (1.0 + g.margin));
        }
        gate_sh = check;
        est_sh = est;
      }
      __syncthreads();
      if (gate_sh) {
        ran = step + 1;
        break;
      }
    }
  }
  // the last iteration's monitor terms: cross, and <W^T W, H H^T> for the normalised W
  if (bid == 0) {
    float cross, quad;
    monitor((ran - 1) & 1, cross, quad);
    if (t == 0) {
      a.mon[0] = cross;
      a.mon[1] = quad;
      if (gated) {
        g.solve[4] = est_sh;
        g.solve[6] = static_cast<double>(start + ran);
        g.flags[1] = 1;
      }
    }
  }
  // write back: W normalised by the last s_j, H
  {
    for (int e = t; e < nrows * r; e += kNT) {
      const int i = e / r, j = e - i * r;
      const float v = Ws[i * RP + j];
      a.W[(r0 + i) * r + j] = normalize ? v / sc[j] : v;
    }
    for (int e = t; e < ncols * r; e += kNT) {
      const int j = e / ncols, c = e - j * ncols;
      a.H[static_cast<int64_t>(j) * a.n + c0 + c] = Hs[c * RP + j];
    }
  }
}

// Lanes per row / rows per lane group of the W phase (GA, RA) and of the H phase (GB, RC) for
// each padded rank. Measured on the 20000 x 5000, r = 20 workload (W sweep per iteration):
// 2 lanes x 1 row 6.7 us, 4 x 2 7.1 us, 2 x 2 8.9 us, 4 x 4 9.4 us (register pressure), so one
// row per group; 4 lanes above RP = 32 keep the per-lane runs at 12 components.
template <int RP>
struct Lanes;
template <> struct Lanes<8> { static constexpr int GA = 2, RA = 1, GB = 2, RC = 1; };
template <> struct Lanes<16> { static constexpr int GA = 2, RA = 1, GB = 2, RC = 1; };
template <> struct Lanes<24> { static constexpr int GA = 2, RA = 1, GB = 2, RC = 1; };
template <> struct Lanes<32> { static constexpr int GA = 2, RA = 1, GB = 2, RC = 1; };
template <> struct Lanes<48> { static constexpr int GA = 4, RA = 1, GB = 4, RC = 1; };

template <int RP, int RULE, int GA, int RA, int GB, int RC>
__global__ void __launch_bounds__(kNT, 1) iterate_persistent_kernel(PArgs a, SolveGate g) {
  extern __shared__ __align__(16) float sh[];
  iterate_body<RP, RULE, GA, RA, GB, RC>(a, g, blockIdx.x, gridDim.x, sh);
}

// Several independent problems in one cooperative launch: blocks [start[p], start[p + 1]) run
// problem p with its own sums, barrier counter and abort flag.
constexpr int kMaxWave = 152;
struct MultiArgs {
  int nprob;
  int start[kMaxWave + 1];
  PArgs p[kMaxWave];
};

template <int RP, int RULE, int GA, int RA, int GB, int RC>
__global__ void __launch_bounds__(kNT, 1) iterate_multi_kernel(const __grid_constant__ MultiArgs M) {
  extern __shared__ __align__(16) float sh[];
  int lo = 0, hi = M.nprob;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (M.start[mid] <= static_cast<int>(blockIdx.x)) lo = mid;
    else hi = mid;
  }
  const PArgs a = M.p[lo];
  iterate_body<RP, RULE, GA, RA, GB, RC>(a, SolveGate{}, blockIdx.x - M.start[lo],
                                         M.start[lo + 1] - M.start[lo], sh);
}

size_t smem_floats(int RP, int ell, int RB, int CB) {
  const int LQ = lq_of(ell), LS = lsx_of(ell);
  return static_cast<size_t>(2 * LQ * RP + 2 * RP * RP + 3 * RP) + static_cast<size_t>(RB + CB) * RP +
         static_cast<size_t>(2 * RB + 2 * CB) * LS + kNT * 16;
}

int rp_of(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : r <= 24 ? 24 : r <= 32 ? 32 : 48; }

template <int RP, int RULE, int GA = Lanes<RP>::GA, int RA = Lanes<RP>::RA,
          int GB = Lanes<RP>::GB, int RC = Lanes<RP>::RC>
cudaError_t launch(const Launcher& L, PArgs& a, SolveGate& g, int grid) {
  auto k = iterate_persistent_kernel<RP, RULE, GA, RA, GB, RC>;
  const size_t smem = sizeof(float) * smem_floats(RP, a.ell, a.RB, a.CB);
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kNT, smem)) != cudaSuccess)
    return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {&a, &g};
  err = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k), dim3(grid), dim3(kNT), args, smem,
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
  const int RP = rp_of(r), LQ = lq_of(ell);
  const size_t ea = ea_size(RP, LQ), eb = eb_size(RP, LQ);
  return sizeof(float) * kCopies * 2 * (ea + eb) + sizeof(Barrier) + 2 * sizeof(int) + 1024;
}

bool iterate_persistent_supported(int64_t m, int64_t n, int r, int ell) {
  if (r < 1 || r > 48 || ell < 1 || ell > 128) return false;
  const int grid = num_sms();
  const int64_t rb = (m + grid - 1) / grid, cbk = (n + grid - 1) / grid;
  if (rb > 4096 || cbk > 4096) return false;
  return sizeof(float) * smem_floats(rp_of(r), ell, static_cast<int>(rb), static_cast<int>(cbk)) <=
         220 * 1024;
}

namespace {

// Arguments, cleared sums and the launch of one persistent run (iters, or the gate in a).
cudaError_t run_persistent(const Launcher& L, const IterArgs& ia, int iters, void* ws,
                           int* status, float* mon, const int* done, SolveGate g) {
  PArgs a;
  char* p = static_cast<char*>(ws);
  const int RP = rp_of(ia.r), LQ = lq_of(ia.ell);
  const size_t ea = ea_size(RP, LQ), eb = eb_size(RP, LQ);
  const int grid = num_sms();
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
  // 16-byte aligned sums (vector atomics)
  uintptr_t base = (reinterpret_cast<uintptr_t>(p) + 15) & ~static_cast<uintptr_t>(15);
  a.accA = reinterpret_cast<float*>(base);
  a.accB = a.accA + 2 * kCopies * ea;
  a.bar = reinterpret_cast<Barrier*>(a.accB + 2 * kCopies * eb);
  a.abort_flag = reinterpret_cast<int*>(a.bar + 1);
  a.status = status;
  a.mon = mon;
  a.done = done;
  a.wait_cycles = ia.wait_cycles > 0 ? ia.wait_cycles : kWaitCycles;
  const size_t clear = reinterpret_cast<char*>(a.abort_flag + 1) - reinterpret_cast<char*>(base);
  cudaError_t err = cudaMemsetAsync(a.accA, 0, clear, L.stream);
  if (err != cudaSuccess) return err;
  a.RB = static_cast<int>((ia.m + grid - 1) / grid);
  a.CB = static_cast<int>((ia.n + grid - 1) / grid);
  const bool mu = ia.rule != 0;
  switch (RP) {
    case 8: return mu ? launch<8, 1>(L, a, g, grid) : launch<8, 0>(L, a, g, grid);
    case 16: return mu ? launch<16, 1>(L, a, g, grid) : launch<16, 0>(L, a, g, grid);
    case 24: return mu ? launch<24, 1>(L, a, g, grid) : launch<24, 0>(L, a, g, grid);
    case 32: return mu ? launch<32, 1>(L, a, g, grid) : launch<32, 0>(L, a, g, grid);
    default: return mu ? launch<48, 1>(L, a, g, grid) : launch<48, 0>(L, a, g, grid);
  }
}

}  // namespace

cudaError_t launch_iterate_persistent(const Launcher& L, const IterArgs& ia, int iters, void* ws,
                                      size_t ws_bytes, int* status, float* mon, const int* done) {
  if (ws_bytes < iterate_persistent_ws_bytes(ia.r, ia.ell)) return cudaErrorInvalidValue;
  if (!iterate_persistent_supported(ia.m, ia.n, ia.r, ia.ell)) return cudaErrorInvalidValue;
  if (iters <= 0) return cudaSuccess;
  return run_persistent(L, ia, iters, ws, status, mon, done, SolveGate{});
}

cudaError_t launch_iterate_persistent_gated(const Launcher& L, const IterArgs& ia,
                                            const SolveGate& g, void* ws, size_t ws_bytes,
                                            int* status, float* mon) {
  if (ws_bytes < iterate_persistent_ws_bytes(ia.r, ia.ell)) return cudaErrorInvalidValue;
  if (!iterate_persistent_supported(ia.m, ia.n, ia.r, ia.ell)) return cudaErrorInvalidValue;
  if (g.total <= 0 || g.every <= 0 || !g.flags || !g.solve) return cudaErrorInvalidValue;
  return run_persistent(L, ia, 0, ws, status, mon, g.flags, g);
}

// ---------------------------------------------------------------- several problems at once

namespace {

template <int RP, int RULE>
cudaError_t launch_multi(const Launcher& L, const MultiArgs& M, int grid, size_t smem) {
  auto k = iterate_multi_kernel<RP, RULE, Lanes<RP>::GA, Lanes<RP>::RA, Lanes<RP>::GB,
                                Lanes<RP>::RC>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kNT, smem)) != cudaSuccess)
    return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {const_cast<MultiArgs*>(&M)};
  err = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k), dim3(grid), dim3(kNT), args, smem,
                                    L.stream);
  L.count();
  return err;
}

cudaError_t launch_multi_rp(int RP, bool mu, const Launcher& L, const MultiArgs& M, int grid,
                            size_t smem) {
  switch (RP) {
    case 8: return mu ? launch_multi<8, 1>(L, M, grid, smem) : launch_multi<8, 0>(L, M, grid, smem);
    case 16: return mu ? launch_multi<16, 1>(L, M, grid, smem) : launch_multi<16, 0>(L, M, grid, smem);
    case 24: return mu ? launch_multi<24, 1>(L, M, grid, smem) : launch_multi<24, 0>(L, M, grid, smem);
    case 32: return mu ? launch_multi<32, 1>(L, M, grid, smem) : launch_multi<32, 0>(L, M, grid, smem);
    default: return mu ? launch_multi<48, 1>(L, M, grid, smem) : launch_multi<48, 0>(L, M, grid, smem);
  }
}

}  // namespace

int iterate_multi_min_blocks(int64_t m, int64_t n, int r, int ell) {
  if (r < 1 || r > 48 || ell < 1 || ell > 128) return 0;
  const int sms = num_sms();
  for (int c = 1; c <= sms; ++c) {
    const int64_t rb = (m + c - 1) / c, cbk = (n + c - 1) / c;
    if (rb <= 4096 && cbk <= 4096 &&
        sizeof(float) * smem_floats(rp_of(r), ell, static_cast<int>(rb), static_cast<int>(cbk)) <=
            220 * 1024)
      return c;
  }
  return 0;
}

size_t iterate_multi_ws_bytes(const IterArgs* ia, int nprob) {
  size_t b = 1024;
  for (int i = 0; i < nprob; ++i) b += (iterate_persistent_ws_bytes(ia[i].r, ia[i].ell) + 255) / 256 * 256;
  return b;
}

cudaError_t launch_iterate_multi(const Launcher& L, const IterArgs* ia, const int* iters,
                                 const int* blocks, int nprob, void* ws, size_t ws_bytes,
                                 int* status, float* mon, const int* done_zero) {
  if (nprob < 1) return cudaSuccess;
  if (ws_bytes < iterate_multi_ws_bytes(ia, nprob)) return cudaErrorInvalidValue;
  const int sms = num_sms();
  // per-problem sums, barrier and abort flag (all zeroed here)
  std::vector<PArgs> pa(nprob);
  uintptr_t base = (reinterpret_cast<uintptr_t>(ws) + 255) & ~static_cast<uintptr_t>(255);
  const uintptr_t first = base;
  for (int i = 0; i < nprob; ++i) {
    if (ia[i].r < 1 || ia[i].r > 48 || blocks[i] < iterate_multi_min_blocks(ia[i].m, ia[i].n, ia[i].r, ia[i].ell) ||
        blocks[i] > sms)
      return cudaErrorInvalidValue;
    const int RP = rp_of(ia[i].r), LQ = lq_of(ia[i].ell);
    const size_t ea = ea_size(RP, LQ), eb = eb_size(RP, LQ);
    PArgs& a = pa[i];
    a.m = ia[i].m;
    a.n = ia[i].n;
    a.r = ia[i].r;
    a.ell = ia[i].ell;
    a.iters = iters[i];
    a.rule = ia[i].rule;
    a.alpha = ia[i].alpha;
    a.beta = ia[i].beta;
    a.eps = ia[i].eps;
    a.QL = ia[i].QL;
    a.QR = ia[i].QR;
    a.Xhat = ia[i].Xhat;
    a.Xchk = ia[i].Xchk;
    a.W = ia[i].W;
    a.H = ia[i].H;
    a.accA = reinterpret_cast<float*>(base);
    a.accB = a.accA + 2 * kCopies * ea;
    a.bar = reinterpret_cast<Barrier*>(a.accB + 2 * kCopies * eb);
    a.abort_flag = reinterpret_cast<int*>(a.bar + 1);
    a.status = status;
    a.mon = mon + 2 * i;
    a.done = done_zero;
    a.wait_cycles = ia[i].wait_cycles > 0 ? ia[i].wait_cycles : kWaitCycles;
    a.RB = static_cast<int>((ia[i].m + blocks[i] - 1) / blocks[i]);
    a.CB = static_cast<int>((ia[i].n + blocks[i] - 1) / blocks[i]);
    base += (iterate_persistent_ws_bytes(ia[i].r, ia[i].ell) + 255) / 256 * 256;
  }
  cudaError_t err = cudaMemsetAsync(reinterpret_cast<void*>(first), 0, base - first, L.stream);
  if (err != cudaSuccess) return err;
  // waves: problems of one (RP, rule) class, largest first, first-fit into the SMs
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    const int kx = rp_of(ia[x].r) * 2 + ia[x].rule, ky = rp_of(ia[y].r) * 2 + ia[y].rule;
    if (kx != ky) return kx < ky;
    return blocks[x] > blocks[y];
  });
  size_t at = 0;
  while (at < order.size()) {
    const int cls = rp_of(ia[order[at]].r) * 2 + ia[order[at]].rule;
    size_t end = at;
    while (end < order.size() && rp_of(ia[order[end]].r) * 2 + ia[order[end]].rule == cls) ++end;
    // first-fit decreasing over the class
    std::vector<std::vector<int>> waves;
    std::vector<int> used;
    for (size_t q = at; q < end; ++q) {
      const int i = order[q];
      size_t w = 0;
      while (w < waves.size() && (used[w] + blocks[i] > sms || waves[w].size() >= kMaxWave)) ++w;
      if (w == waves.size()) {
        waves.emplace_back();
        used.push_back(0);
      }
      waves[w].push_back(i);
      used[w] += blocks[i];
    }
    for (size_t w = 0; w < waves.size(); ++w) {
      MultiArgs M;
      M.nprob = static_cast<int>(waves[w].size());
      int grid = 0;
      size_t smem = 0;
      for (int k = 0; k < M.nprob; ++k) {
        const int i = waves[w][k];
        M.start[k] = grid;
        M.p[k] = pa[i];
        grid += blocks[i];
        const size_t sm = sizeof(float) * smem_floats(rp_of(ia[i].r), ia[i].ell, pa[i].RB, pa[i].CB);
        smem = sm > smem ? sm : smem;
      }
      M.start[M.nprob] = grid;
      const int RP = rp_of(ia[waves[w][0]].r);
      if ((err = launch_multi_rp(RP, ia[waves[w][0]].rule != 0, L, M, grid, smem)) != cudaSuccess)
        return err;
    }
    at = end;
  }
  return cudaSuccess;
}

}  // namespace nmfrp
