// Fused dual pass over a BF16 X on the 5th-generation tensor cores:
//   Y = X V (m x l) and Z = X^T U (n x l) from one TMA stream of X.
// This is every sketch pass (Section 3, Eq. 3.5: X applied to one chain's basis and X^T to the
// other's) and the compression (Section 4: X_chk = X Q_R, X_hat = Q_L^T X).
//
// Tiling. A CTA owns a rectangle of row blocks (128 rows) x column tiles (128 columns). For each
// 128 x 128 tile of X, staged in shared memory by TMA as two 128B-swizzled 128 x 64 halves:
//   Y block (128 x LP) += X_tile (K-major A, K = columns)         . V_tile^T  (B: LP x 128)
//   Z tile  (128 x LP) += X_tile viewed MN-major (A, K = rows)    . U_block^T (B: LP x 128)
// (tcgen05.mma kind::f16, M = 128, N = LP = l rounded up to 16, BF16 inputs, FP32 accumulation
// in tensor memory). The Y accumulator of the current row block is double-buffered in TMEM; the
// Z accumulators of all the CTA's column tiles stay in TMEM for the whole rectangle. V^T and U^T
// are BF16 copies made by a small preparation kernel (rows l..LP-1 zero).
//
// Warp roles (192 threads): warps 0-3 drain TMEM (each its 32-lane sub-partition) and write the
// partial sums, warp 4 issues the TMA loads, warp 5 allocates TMEM and issues the MMAs.
// FP8 X (E4M3 codes, one E8M0 scale a 32 x 32 tile): TMA brings each 128 x 128 tile of codes
// (16 KB, 128B-swizzled) into its own ring, and warps 6-13 rewrite it as the BF16 tile the MMAs
// read, code times 2^k (exact in BF16), in the same swizzled layout, before signalling the MMA
// issuer; the HBM stream is half that of BF16 X.
// FP32 X: TMA brings each tile into a 64 KB stage as four 32-row x 128-column boxes (512-byte
// rows, no swizzle); warps 6-13 read it into registers, meet at a barrier, and rewrite the stage
// in place as a BF16 hi tile and a BF16 lo tile (hi = bf16(x), lo = bf16(x - hi): x to about
// 2^-18 relative), which is the same 64 KB. Two stages let one tile convert while the previous
// one's MMAs run. With V and U also entering as hi + lo pairs, each product accumulates
// x_hi v_hi + x_hi v_lo + x_lo v_hi: FP32-grade sums on the BF16 tensor cores from one FP32
// stream of X. Partial
// sums of Y (one per column group) and Z (one per row group) are summed in a fixed slot order
// by one slot-sum launch for both. Every mbarrier wait is bounded; on time-out the kernel
// latches NMF_ERR_TIMEOUT, drains what it issued and frees its tensor memory.
#include <cuda.h>

#include <algorithm>
#include <vector>
#include <cuda_fp8.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nmfrp {
namespace {

using namespace tc;

constexpr int kRows = 128;          // rows per block (MMA M for Y)
constexpr int kCols = 128;          // columns per tile (MMA M for Z)
constexpr int kHalfCols = 64;       // 128-byte swizzle atom: 64 BF16 columns
constexpr int kThreads = 192;
constexpr int kThreadsF8 = 448;     // + warps 6-13: FP8 -> BF16 converters (two a row)
constexpr int kConv = kThreadsF8 - kThreads;
constexpr int kF8Stages = 4;        // ring of FP8 tiles
constexpr uint32_t kX8Stage = 128 * 128;   // one 128 x 128 E4M3 tile (16 KB)
constexpr uint32_t kF32Box = 32 * 128 * 4;   // one 32-row x 128-column FP32 box (16 KB)

// Element type of X inside the kernel: BF16 read by the MMAs directly, or FP8 / FP32 converted
// to BF16 in shared memory first.
enum : int { kXkBf16 = 0, kXkF8 = 1, kXkF32 = 2 };

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, M = 128, N = LP.
__host__ __device__ constexpr uint32_t idesc_bf16(int N, int a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(a_mn_major) << 15) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(kRows >> 4) << 24);
}

// ------------------------------------------------------------------ kernel

constexpr int kMaxGroups = 160;    // column groups whose row-group counts a table holds

// Row groups of each column group: CTAs [cta0[g], cta0[g + 1]) take column group g, each a
// contiguous share of the row blocks. Narrower groups get fewer row groups, so every CTA streams
// about the same number of bytes. Without a table (more column groups than it holds) every
// group has n_rowgroups row groups.
struct GroupTable {
  int table;                      // 1: cta0 is valid
  int cta0[kMaxGroups + 1];
};

struct TcArgs {
  int64_t m, n;
  int ell;
  int n_rowgroups, n_colgroups;   // n_rowgroups: the most row groups of any column group
  int64_t n_rowblocks;            // ceil(m / 128)
  int tiles_per_group;            // column tiles per column group (<= the kernel's NCT)
  int stages;                     // X stages in shared memory (<= kMaxStages)
  int64_t n_coltiles;             // ceil(n / 128)
  float* Ypart;                   // [n_colgroups][ell][m]   (k-major: rows contiguous)
  float* Zpart;                   // [n_rowgroups][ell][n]
  GroupTable gt;
  int* status;
  const uint8_t* S;               // FP8 X: E8M0 tile scales (row-major, tn a row)
  int64_t tn;
  int nub;                        // U buffers (2, or 1 where shared memory is short)
};

// Two E4M3 codes (low byte = first element) times 2^k (exact) as a BF16 pair (low half first).
__device__ __forceinline__ uint32_t e4m3x2_to_bf16x2(uint32_t pair, float sc) {
  const __half2_raw h =
      __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(pair & 0xFFFFu), __NV_E4M3);
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h));
  const __nv_bfloat162 b = __floats2bfloat162_rn(f.x * sc, f.y * sc);
  return *reinterpret_cast<const uint32_t*>(&b);
}

constexpr int kMaxStages = 4;
constexpr uint32_t kXStage = 2 * kRows * kHalfCols * 2;   // 32 KB: two 128 x 64 BF16 halves
constexpr int kSmemCap = 232448 - 1024;   // opt-in shared memory per block, less the static part

// tensor-memory columns of one accumulator and the most column tiles whose Z accumulators fit
__host__ __device__ constexpr int acc_stride(int LP) { return (LP + 31) / 32 * 32; }
__host__ __device__ constexpr int nct_max(int LP) {
  return (512 / acc_stride(LP) - 2) > 14 ? 14 : (512 / acc_stride(LP) - 2);
}
// FP32 X: each row block's Z contribution is drained from tensor memory into FP32 registers of
// the epilogue (double-buffered with Y), so the resident column tiles are bounded by the
// registers (96 sums a thread) and by two Z buffers in tensor memory.
constexpr int kZRegs = 96;
__host__ __device__ constexpr int nct_f32_max(int LP) {
  return kZRegs / LP < 1 ? 1 : kZRegs / LP;
}

// SPLIT = 2: V and U enter as hi + lo BF16 pairs (v = hi + lo to about 2^-16 relative), each
// product is accumulated from both, so only X is rounded to BF16 (FP32 X: split too).
template <int LP, int SPLIT, int XK>
__global__ void __launch_bounds__(XK != kXkBf16 ? kThreadsF8 : kThreads, 1) dual_pass_tc_kernel(
    const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapV,
    const __grid_constant__ CUtensorMap mapU, TcArgs a) {
  constexpr bool F8 = XK == kXkF8, F32 = XK == kXkF32, CONV = F8 || F32;
  static_assert(!F32 || SPLIT == 2, "FP32 X takes split bases");
  constexpr int NCT = F32 ? nct_f32_max(LP) : nct_max(LP);
  constexpr uint32_t kXHalf = kRows * kHalfCols * 2;   // 16 KB
  constexpr uint32_t kXStg = F32 ? 2 * kXStage : kXStage;   // FP32: hi tile, then lo tile
  constexpr uint32_t kBBox = LP * kHalfCols * 2;        // LP rows x 128 B
  constexpr uint32_t kBTile = SPLIT * 2 * kBBox;        // one column tile (or row block) of V (U)
  constexpr int AS = acc_stride(LP);
  constexpr int kTmemNeed = (2 + (F32 ? 2 : 1) * NCT) * AS;
  constexpr uint32_t kTmemCols = kTmemNeed <= 32 ? 32 : kTmemNeed <= 64 ? 64 : kTmemNeed <= 128
                                                                                ? 128
                                                                                : kTmemNeed <= 256
                                                                                      ? 256
                                                                                      : 512;
  static_assert(kTmemNeed <= 512, "tensor memory budget");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int stages = a.stages, nub = a.nub;
  unsigned char* Xs = smem;                              // [stages][kXStg]
  unsigned char* X8 = Xs + stages * kXStg;               // [kF8Stages][16 KB] (F8 only)
  unsigned char* Us = X8 + (F8 ? kF8Stages * kX8Stage : 0u);   // [nub][SPLIT][2 halves][kBBox]
  unsigned char* Vs = Us + nub * kBTile;                 // [nct][SPLIT][2 halves][kBBox]
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t u_full[2], u_empty[2], v_full;
  __shared__ __align__(8) uint64_t ydone_bar[2], yfree_bar[2], zdone_bar, drain_bar;
  __shared__ __align__(8) uint64_t conv_bar;   // FP32: the converters' read-before-write barrier
  // FP8: the ring of code tiles; FP32: f8_full[s] = the FP32 tile of stage s has landed
  __shared__ __align__(8) uint64_t f8_full[kF8Stages], f8_empty[kF8Stages];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_f;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int cg, rg, nrg;
  if (a.gt.table) {
    cg = 0;
    while (cg + 1 < a.n_colgroups && a.gt.cta0[cg + 1] <= static_cast<int>(blockIdx.x)) ++cg;
    rg = blockIdx.x - a.gt.cta0[cg];
    nrg = a.gt.cta0[cg + 1] - a.gt.cta0[cg];
  } else {
    cg = blockIdx.x / a.n_rowgroups;
    rg = blockIdx.x - cg * a.n_rowgroups;
    nrg = a.n_rowgroups;
  }
  // this CTA's row blocks [rb0, rb1) and column tiles [ct0, ct1)
  const int64_t rb0 = rg * a.n_rowblocks / nrg;
  const int64_t rb1 = (rg + 1) * a.n_rowblocks / nrg;
  const int64_t ct0 = static_cast<int64_t>(cg) * a.tiles_per_group;
  const int64_t ct1 = min(a.n_coltiles, ct0 + a.tiles_per_group);
  const int nrb = static_cast<int>(rb1 - rb0), nct = static_cast<int>(ct1 - ct0);
  const int ntiles = nrb * nct;

  if (threadIdx.x == 0) {
    abort_f = 0;
    for (int s = 0; s < kMaxStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), CONV ? kConv : 1);   // FP8 / FP32: the converters
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int s = 0; s < kF8Stages; ++s) {
      mbar_init(smem_u32(&f8_full[s]), 1);
      mbar_init(smem_u32(&f8_empty[s]), kConv);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&u_full[b]), 1);
      mbar_init(smem_u32(&u_empty[b]), 1);
      mbar_init(smem_u32(&ydone_bar[b]), 1);
      mbar_init(smem_u32(&yfree_bar[b]), 128);
    }
    mbar_init(smem_u32(&v_full), 1);
    mbar_init(smem_u32(&zdone_bar), 1);
    mbar_init(smem_u32(&drain_bar), 1);
    mbar_init(smem_u32(&conv_bar), kConv);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) tmem_alloc(smem_u32(&tmem_base), kTmemCols);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 4) {
    // ---------------- TMA producer
    if (lane == 0 && ntiles > 0) {
      const uint64_t pol_x = policy_evict_first(), pol_b = policy_evict_last();
      // the CTA's column tiles of V stay resident for the whole rectangle
      const uint32_t vb = smem_u32(&v_full);
      mbar_expect_tx(vb, static_cast<uint32_t>(nct) * kBTile);
      for (int lc = 0; lc < nct; ++lc)
        for (int sp = 0; sp < SPLIT; ++sp)
          for (int hf = 0; hf < 2; ++hf)
            tma_load_2d(smem_u32(Vs + lc * kBTile + (sp * 2 + hf) * kBBox), &mapV,
                        static_cast<int>((ct0 + lc) * kCols) + hf * kHalfCols, sp * LP, vb, pol_b);
      int issued = 0, u_issued = 0;
      bool ok = true;
      for (int lr = 0; lr < nrb && ok; ++lr) {
        const int ub = lr % nub;
        const int row0 = static_cast<int>((rb0 + lr) * kRows);
        if (!mbar_wait(smem_u32(&u_empty[ub]), ((lr / nub) & 1) ^ 1, &abort_f)) break;
        const uint32_t ubar = smem_u32(&u_full[ub]);
        mbar_expect_tx(ubar, kBTile);
        for (int sp = 0; sp < SPLIT; ++sp)
          for (int hf = 0; hf < 2; ++hf)
            tma_load_2d(smem_u32(Us + ub * kBTile + (sp * 2 + hf) * kBBox), &mapU,
                        row0 + hf * kHalfCols, sp * LP, ubar, pol_b);
        u_issued = lr + 1;
        for (int lc = 0; lc < nct; ++lc) {
          const int tI = lr * nct + lc;
          const int col0 = static_cast<int>((ct0 + lc) * kCols);
          if constexpr (F8) {
            const int s8 = tI % kF8Stages;
            if (!mbar_wait(smem_u32(&f8_empty[s8]), ((tI / kF8Stages) & 1) ^ 1, &abort_f)) {
              ok = false;
              break;
            }
            const uint32_t fb = smem_u32(&f8_full[s8]);
            mbar_expect_tx(fb, kX8Stage);
            tma_load_2d(smem_u32(X8 + s8 * kX8Stage), &mapX, col0, row0, fb, pol_x);
          } else if constexpr (F32) {
            // the FP32 tile straight into its stage: four boxes of 32 rows
            const int s = tI % stages;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ((tI / stages) & 1) ^ 1, &abort_f)) {
              ok = false;
              break;
            }
            unsigned char* st = Xs + s * kXStg;
            const uint32_t fb = smem_u32(&f8_full[s]);
            mbar_expect_tx(fb, 4 * kF32Box);
            for (int q = 0; q < 4; ++q)
              tma_load_2d(smem_u32(st + q * kF32Box), &mapX, col0, row0 + 32 * q, fb, pol_x);
          } else {
            const int s = tI % stages;
            const uint32_t ph = (tI / stages) & 1;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1, &abort_f)) {
              ok = false;
              break;
            }
            unsigned char* st = Xs + s * kXStg;
            const uint32_t fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, kXStage);
            tma_load_2d(smem_u32(st), &mapX, col0, row0, fb, pol_x);
            tma_load_2d(smem_u32(st + kXHalf), &mapX, col0 + kHalfCols, row0, fb, pol_x);
          }
          issued = tI + 1;
        }
      }
      // every copy issued has landed before the CTA may leave
      mbar_drain(vb, 0);
      for (int lr = u_issued - nub > 0 ? u_issued - nub : 0; lr < u_issued; ++lr)
        mbar_drain(smem_u32(&u_full[lr % nub]), (lr / nub) & 1);
      const int rn = F8 ? kF8Stages : stages;   // units: FP8 ring tiles, else stage tiles
      for (int tI = issued - rn > 0 ? issued - rn : 0; tI < issued; ++tI)
        mbar_drain(smem_u32(CONV ? &f8_full[tI % rn] : &full_bar[tI % rn]), (tI / rn) & 1);
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer
    if (lane == 0 && ntiles > 0) {
      constexpr uint32_t idY = idesc_bf16(LP, 0);   // A = X tile, K-major
      constexpr uint32_t idZ = idesc_bf16(LP, 1);   // A = X tile, MN-major
      bool ok = mbar_wait(smem_u32(&v_full), 0, &abort_f);
      for (int lr = 0; lr < nrb && ok; ++lr) {
        const int yb = lr & 1, ub = lr % nub;
        if (!mbar_wait(smem_u32(&yfree_bar[yb]), ((lr >> 1) & 1) ^ 1, &abort_f) ||
            !mbar_wait(smem_u32(&u_full[ub]), (lr / nub) & 1, &abort_f)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dY = tmem + static_cast<uint32_t>(yb * AS);
        const uint32_t ubase = smem_u32(Us + ub * kBTile);
        for (int lc = 0; lc < nct; ++lc) {
          const int tI = lr * nct + lc;
          const int s = tI % stages;
          const uint32_t ph = (tI / stages) & 1;
          if (!mbar_wait(smem_u32(&full_bar[s]), ph, &abort_f)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t xa = smem_u32(Xs + s * kXStg), xb = xa + kXHalf;
          const uint32_t vbase = smem_u32(Vs + lc * kBTile);
          // FP32 X: Z of this row block in buffer yb (drained with Y), else resident per tile
          const uint32_t dZ = tmem + static_cast<uint32_t>((2 + (F32 ? yb * NCT : 0) + lc) * AS);
          const bool zacc = !F32 && lr > 0;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint32_t off = (kk & 3) * 32;
            const uint32_t hf = kk < 4 ? 0u : 1u;
            // Y: K = columns of the tile
            const uint64_t aY = sdesc((kk < 4 ? xa : xb) + off, 16, 1024);
            // Z: K = rows of the tile; MN-major A spans both halves (LBO = 16 KB)
            const uint64_t aZ = sdesc(xa + kk * 2048, kXHalf, 1024);
#pragma unroll
            for (int sp = 0; sp < SPLIT; ++sp) {
              const uint64_t bY = sdesc(vbase + (sp * 2 + hf) * kBBox + off, 16, 1024);
              mma_bf16(dY, aY, bY, idY, (lc > 0 || kk > 0 || sp > 0) ? 1u : 0u);
              const uint64_t bZ = sdesc(ubase + (sp * 2 + hf) * kBBox + off, 16, 1024);
              mma_bf16(dZ, aZ, bZ, idZ, (zacc || kk > 0 || sp > 0) ? 1u : 0u);
            }
            if constexpr (F32) {
              // x_lo times the hi parts of V and U (the lo tile sits kXStage past the hi tile)
              const uint64_t aYl = sdesc((kk < 4 ? xa : xb) + kXStage + off, 16, 1024);
              const uint64_t aZl = sdesc(xa + kXStage + kk * 2048, kXHalf, 1024);
              mma_bf16(dY, aYl, sdesc(vbase + hf * kBBox + off, 16, 1024), idY, 1u);
              mma_bf16(dZ, aZl, sdesc(ubase + hf * kBBox + off, 16, 1024), idZ, 1u);
            }
          }
          mma_commit(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&u_empty[ub]));
        mma_commit(smem_u32(&ydone_bar[yb]));
      }
      if (ok) mma_commit(smem_u32(&zdone_bar));
      // drain: all MMAs issued by this thread complete before tensor memory is freed
      mma_commit(smem_u32(&drain_bar));
      mbar_drain(smem_u32(&drain_bar), 0);
    }
  } else if (warp >= 6) {
    // ---------------- FP8 converters (warps 6-13): thread t rewrites half `part` of row ct
    if constexpr (F8) {
      const int ct = (threadIdx.x - kThreads) & 127, part = (threadIdx.x - kThreads) >> 7;
      const int sw = ct & 7;
      bool ok = true;
      for (int lr = 0; lr < nrb && ok; ++lr) {
        const int64_t row = (rb0 + lr) * kRows + ct;
        for (int lc = 0; lc < nct; ++lc) {
          const int tI = lr * nct + lc;
          const int s8 = tI % kF8Stages, s = tI % stages;
          if (!mbar_wait(smem_u32(&f8_full[s8]), (tI / kF8Stages) & 1, &abort_f) ||
              !mbar_wait(smem_u32(&empty_bar[s]), ((tI / stages) & 1) ^ 1, &abort_f)) {
            ok = false;
            break;
          }
          const int64_t col0 = (ct0 + lc) * kCols;
          const unsigned char* src = X8 + s8 * kX8Stage + ct * 128;
          unsigned char* dst = Xs + s * kXStage + ct * 128;
          // scale bytes of this row's tiles from column col0 on (rows / columns past the
          // matrix hold zero codes from the TMA fill: any scale serves)
          const bool rin = row < a.m;
          const uint8_t* srow = a.S + (rin ? (row >> 5) * a.tn : 0) + (col0 >> 5);
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int c = 4 * part + cc;
            // codes of columns col0 + 16 c .. + 15 (chunk c of the row, swizzled)
            const uint4 w = *reinterpret_cast<const uint4*>(src + ((c ^ sw) << 4));
            // the E8M0 byte is the biased exponent of 2^k (byte 0: 2^-127, a subnormal)
            const uint32_t eb = (rin && col0 + 16 * c < a.n) ? srow[c >> 1] : 127u;
            const float sc = eb ? __uint_as_float(eb << 23) : __uint_as_float(0x00400000u);
            const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
            uint32_t o[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              o[2 * h] = e4m3x2_to_bf16x2(wv[h], sc);
              o[2 * h + 1] = e4m3x2_to_bf16x2(wv[h] >> 16, sc);
            }
            // BF16 columns 16 c .. 16 c + 15: half c / 4, 16-byte chunks 2 (c % 4) and + 1
            unsigned char* hb = dst + (c >> 2) * kXHalf;
            const int j0 = (c & 3) * 2;
            *reinterpret_cast<uint4*>(hb + ((j0 ^ sw) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<uint4*>(hb + (((j0 + 1) ^ sw) << 4)) =
                make_uint4(o[4], o[5], o[6], o[7]);
          }
          // the MMAs read the tile through the async proxy
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(smem_u32(&full_bar[s]));
          mbar_arrive(smem_u32(&f8_empty[s8]));
        }
      }
    } else if constexpr (F32) {
      // Thread (converter warp cw, lane) takes row rb of every box (tile rows rb + 32 q) and the
      // 16-byte chunks j, j + 8, j + 16, j + 24 of its 512-byte rows (j = lane % 8). The four
      // rows of a warp are b, b + 4, b + 2, b + 6 (b = 8 (cw / 2) + cw % 2): a quarter-warp
      // reads 128 contiguous bytes, and a half-warp's 8-byte stores fall in two rows whose
      // swizzles differ by 4, so neither side has bank conflicts.
      const int cw = warp - 6, j = lane & 7, k = lane >> 3;
      const int rb = 8 * (cw >> 1) + (cw & 1) + (((k & 1) << 2) | (k & 2));
      const int sw = rb & 7;   // tile row 32 q + rb has the same swizzle phase
      for (int tI = 0; tI < ntiles; ++tI) {
        const int s = tI % stages;
        if (!mbar_wait(smem_u32(&f8_full[s]), (tI / stages) & 1, &abort_f)) break;
        unsigned char* st = Xs + s * kXStg;
        float4 x[4][4];   // [box q][chunk cc]
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
            x[q][cc] = *reinterpret_cast<const float4*>(st + q * kF32Box + rb * 512 +
                                                        (8 * cc + j) * 16);
        // every converter has its FP32 values before any of the stage is overwritten (an
        // mbarrier with a bounded wait, so that an abort cannot leave threads at the barrier)
        mbar_arrive(smem_u32(&conv_bar));
        if (!mbar_wait(smem_u32(&conv_bar), tI & 1, &abort_f)) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          unsigned char* rowp = st + (32 * q + rb) * 128;
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const float4 v = x[q][cc];
            const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y);
            const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.z, v.w);
            const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
            const __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y);
            const __nv_bfloat162 l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
            // columns 4 (8 cc + j) .. + 3: half cc / 2, BF16 chunk 4 (cc % 2) + j / 2, bytes
            // 8 (j % 2) .. + 7 of it; the lo tile sits kXStage past the hi tile
            unsigned char* d = rowp + (cc >> 1) * kXHalf +
                               (((4 * (cc & 1) + (j >> 1)) ^ sw) << 4) + ((j & 1) << 3);
            *reinterpret_cast<uint2*>(d) = make_uint2(*reinterpret_cast<const uint32_t*>(&h0),
                                                      *reinterpret_cast<const uint32_t*>(&h1));
            *reinterpret_cast<uint2*>(d + kXStage) =
                make_uint2(*reinterpret_cast<const uint32_t*>(&l0),
                           *reinterpret_cast<const uint32_t*>(&l1));
          }
        }
        // the MMAs read the tiles through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_bar[s]));
      }
    }
  } else {
    // ---------------- epilogue: warps 0-3, TMEM lanes 32 warp .. 32 warp + 31
    // partial sums are k-major, so each store of a warp covers 32 consecutive floats
    const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
    float v[16];
    // FP32 X: this thread's column (one a tile) summed over the row blocks, round-to-nearest
    float zsum[F32 ? NCT * LP : 1];
#pragma unroll
    for (int i = 0; i < (F32 ? NCT * LP : 1); ++i) zsum[i] = 0.f;
    for (int lr = 0; lr < (ntiles > 0 ? nrb : 0); ++lr) {
      const int yb = lr & 1;
      if (!mbar_wait(smem_u32(&ydone_bar[yb]), (lr >> 1) & 1, &abort_f)) break;
      tc_fence_after();
      const int64_t row = (rb0 + lr) * kRows + warp * 32 + lane;
      float* dst = a.Ypart + static_cast<int64_t>(cg) * a.ell * a.m + row;
#pragma unroll 1
      for (int c = 0; c < LP; c += 16) {
        tmem_ld16(tmem + lane_base + yb * AS + c, v);
        if (row < a.m) {
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (c + k < a.ell) __stcg(dst + static_cast<int64_t>(c + k) * a.m, v[k]);
        }
      }
      if constexpr (F32) {
#pragma unroll
        for (int lc = 0; lc < NCT; ++lc) {
          if (lc < nct) {
#pragma unroll
            for (int c = 0; c < LP; c += 16) {
              tmem_ld16(tmem + lane_base + (2 + yb * NCT + lc) * AS + c, v);
#pragma unroll
              for (int k = 0; k < 16; ++k) zsum[lc * LP + c + k] += v[k];
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&yfree_bar[yb]));
    }
    if constexpr (F32) {
#pragma unroll
      for (int lc = 0; lc < NCT; ++lc) {
        const int64_t col = (ct0 + lc) * kCols + warp * 32 + lane;
        if (lc < nct && ntiles > 0 && col < a.n) {
          float* dst = a.Zpart + static_cast<int64_t>(rg) * a.ell * a.n + col;
#pragma unroll
          for (int c = 0; c < LP; ++c)
            if (c < a.ell) __stcg(dst + static_cast<int64_t>(c) * a.n, zsum[lc * LP + c]);
        }
      }
    } else if (ntiles > 0 && mbar_wait(smem_u32(&zdone_bar), 0, &abort_f)) {
      tc_fence_after();
      for (int lc = 0; lc < nct; ++lc) {
        const int64_t col = (ct0 + lc) * kCols + warp * 32 + lane;
        float* dst = a.Zpart + static_cast<int64_t>(rg) * a.ell * a.n + col;
#pragma unroll 1
        for (int c = 0; c < LP; c += 16) {
          tmem_ld16(tmem + lane_base + (2 + lc) * AS + c, v);
          if (col < a.n) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (c + k < a.ell) __stcg(dst + static_cast<int64_t>(c + k) * a.n, v[k]);
          }
        }
      }
      tc_fence_before();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && abort_f) latch(a.status, kStTimeout);
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Operand preparation of one pass in one launch: V (n x ell, FP32) -> Vt and U (m x ell) -> Ut
// (SPLIT*LP x ld, BF16): rows [0, LP) hold hi = bf16(v), rows [LP, 2 LP) (SPLIT = 2) hold
// lo = bf16(v - hi); rows ell..LP-1 of each part and columns rows..ld-1 are zero. Blocks
// [0, nbv) of grid.x take V, the rest U.
__global__ void prep_operands_kernel(const float* __restrict__ V, int64_t n, int64_t ldv,
                                     __nv_bfloat16* __restrict__ Vt, const float* __restrict__ U,
                                     int64_t m, int64_t ldu, __nv_bfloat16* __restrict__ Ut,
                                     int ell, int LP, int split, int nbv) {
  __shared__ float tile[32][33];
  const bool isv = static_cast<int>(blockIdx.x) < nbv;
  const float* src = isv ? V : U;
  const int64_t rows = isv ? n : m, ld = isv ? ldv : ldu;
  __nv_bfloat16* dst = isv ? Vt : Ut;
  const int64_t r0 = static_cast<int64_t>(isv ? blockIdx.x : blockIdx.x - nbv) * 32;
  const int k0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i;
    const int k = k0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && k < ell) ? src[r * ell + k] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i;
    const int64_t r = r0 + threadIdx.x;
    if (k < LP && r < ld) {
      const float x = tile[threadIdx.x][i];
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      dst[static_cast<int64_t>(k) * ld + r] = hi;
      if (split == 2)
        dst[static_cast<int64_t>(LP + k) * ld + r] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
  }
}

// Slot sums of one pass in one launch: Y[row][k] = sum over ys slots of Yp[slot][k][row] and
// Z[col][k] (or Z[k][col] when z_kmajor) = sum over zs slots of Zp[slot][k][col], in slot order.
// A block takes 128 rows (or columns) x 8 values of k: a thread sums four consecutive rows of
// one k with 16-byte loads, eight slots in flight, and the block writes its tile transposed
// through shared memory (or straight, k-major). Blocks [0, by) of grid.x take Y, the rest Z.
constexpr int kRedRows = 128;
__global__ void __launch_bounds__(256) reduce_pass_kernel(const float* __restrict__ Yp, int ys,
                                                          int64_t m, float* __restrict__ Y,
                                                          const float* __restrict__ Zp, int zs,
                                                          int64_t n, float* __restrict__ Z,
                                                          int ell, int z_kmajor, int by, int tpg,
                                                          const __grid_constant__ GroupTable gt) {
  __shared__ float tile[8][kRedRows + 4];
  const bool isy = static_cast<int>(blockIdx.x) < by;
  const float* part = isy ? Yp : Zp;
  // a block of Z is one column tile: its slots are the row groups of its column group
  int slots = isy ? ys : zs;
  if (!isy && gt.table) {
    const int g = static_cast<int>(blockIdx.x - by) / tpg;
    slots = gt.cta0[g + 1] - gt.cta0[g];
  }
  const int64_t rows = isy ? m : n;
  float* out = isy ? Y : Z;
  const bool kmajor = !isy && z_kmajor;
  const int64_t row0 = static_cast<int64_t>(isy ? blockIdx.x : blockIdx.x - by) * kRedRows;
  const int k0 = blockIdx.y * 8;
  const int t = threadIdx.x, kq = t >> 5, q = t & 31;   // k = k0 + kq, rows row0 + 4q .. + 3
  const int k = k0 + kq;
  const int64_t r = row0 + 4 * q;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k < ell && r < rows) {
    const int64_t sstride = static_cast<int64_t>(ell) * rows;
    const float* pp = part + static_cast<int64_t>(k) * rows + r;
    if (r + 4 <= rows && (rows & 3) == 0) {
      int c = 0;
      for (; c + 8 <= slots; c += 8) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(reinterpret_cast<const float4*>(pp + (c + u) * sstride));
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          acc.x += v[u].x;
          acc.y += v[u].y;
          acc.z += v[u].z;
          acc.w += v[u].w;
        }
      }
      for (; c < slots; ++c) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(pp + c * sstride));
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
      }
    } else {
      // ragged tail (or rows not a multiple of 4: no 16-byte alignment): element loads
      float a4[4] = {0.f, 0.f, 0.f, 0.f};
      for (int c = 0; c < slots; ++c)
        for (int e = 0; e < 4; ++e)
          if (r + e < rows) a4[e] += __ldcg(pp + c * sstride + e);
      acc = make_float4(a4[0], a4[1], a4[2], a4[3]);
    }
  }
  if (kmajor) {
    if (k < ell)
      for (int e = 0; e < 4; ++e)
        if (r + e < rows) out[static_cast<int64_t>(k) * rows + r + e] = (&acc.x)[e];
    return;
  }
  tile[kq][4 * q] = acc.x;
  tile[kq][4 * q + 1] = acc.y;
  tile[kq][4 * q + 2] = acc.z;
  tile[kq][4 * q + 3] = acc.w;
  __syncthreads();
  // out rows row0 .. row0 + 127, columns k0 .. k0 + 7: thread t writes (row t / 8 * 4 + i ...)
  for (int e = t; e < kRedRows * 8; e += 256) {
    const int i = e >> 3, j = e & 7;
    if (row0 + i < rows && k0 + j < ell) out[(row0 + i) * ell + k0 + j] = tile[j][i];
  }
}

// ------------------------------------------------------------------ host side

// 2-D map of E4M3 codes: `inner` columns (row pitch `pitch` bytes, a multiple of 16), `outer`
// rows, box 128 x 128 (128-byte rows: the 128B swizzle atom); reads past the edges give zero.
bool make_map8(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {pitch};
  const cuuint32_t box[2] = {128, 128};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

int lp16(int ell) { return (ell + 15) / 16 * 16; }

struct Plan {
  int LP, split, stages, nct, nub;
  size_t smem;
  int rowgroups, colgroups, tiles_per_group;   // rowgroups: the most of any column group
  int ctas;
  int64_t rowblocks, coltiles;
  GroupTable gt;
};

// nub: U buffers (two unless shared memory is short)
size_t smem_bytes(int LP, int split, int stages, int nct, int xk = kXkBf16, int nub = 2) {
  const size_t btile = static_cast<size_t>(split) * 2 * LP * kHalfCols * 2;
  const size_t xin = xk == kXkF8 ? kF8Stages * kX8Stage : 0;
  return static_cast<size_t>(stages) * (xk == kXkF32 ? 2 : 1) * kXStage + xin +
         static_cast<size_t>(nub) * btile + static_cast<size_t>(nct) * btile + 1024;
}

// Deepest X pipeline that still keeps enough resident column tiles (4 stages with
// min(4, NCT) tiles, else 3 stages with min(2, NCT), else 2 stages with one), then as many
// resident column tiles as fit. nct = 0 means the configuration does not fit.
// FP32 X: two 64 KB stages (FP32 tile, converted in place to hi + lo), two U buffers, or one
// where the split bases leave no room for two (LP = 80).
void pick_stages(int LP, int split, int* stages, int* nct, int xk = kXkBf16, int* nub = nullptr) {
  const int cap = xk == kXkF32 ? nct_f32_max(LP) : nct_max(LP);
  if (nub) *nub = 2;
  if (xk == kXkF32) {
    *stages = 2;
    for (int u = 2; u >= 1; --u) {
      int k = cap;
      while (k > 0 && smem_bytes(LP, split, 2, k, xk, u) > static_cast<size_t>(kSmemCap)) --k;
      if (k > 0) {
        *nct = k;
        if (nub) *nub = u;
        return;
      }
    }
    *nct = 0;
    return;
  }
  for (int s = kMaxStages; s >= 2; --s) {
    int k = cap;
    while (k > 0 && smem_bytes(LP, split, s, k, xk) > static_cast<size_t>(kSmemCap)) --k;
    const int want = s == 4 ? (cap < 4 ? cap : 4) : s == 3 ? (cap < 2 ? cap : 2) : 1;
    if (k >= want && k > 0) {
      *stages = s;
      *nct = k;
      return;
    }
  }
  *stages = 2;
  *nct = 0;
}

Plan plan_for(int64_t m, int64_t n, int ell, int split, int xk = kXkBf16) {
  Plan p;
  p.LP = lp16(ell);
  p.split = split;
  pick_stages(p.LP, split, &p.stages, &p.nct, xk, &p.nub);
  p.smem = smem_bytes(p.LP, split, p.stages, p.nct > 0 ? p.nct : 1, xk, p.nub);
  p.rowblocks = cdiv(m, kRows);
  p.coltiles = cdiv(n, kCols);
  const int nct = p.nct > 0 ? p.nct : 1;
  p.colgroups = static_cast<int>(cdiv(p.coltiles, nct));
  p.tiles_per_group = static_cast<int>(cdiv(p.coltiles, p.colgroups));
  const int sms = num_sms();
  p.gt.table = 0;
  if (p.colgroups > sms || p.colgroups > kMaxGroups) {
    // more column groups than CTAs at a time: one row group each
    p.rowgroups = 1;
    p.ctas = p.colgroups;
    return p;
  }
  // row groups in proportion to each column group's tiles, then one more at a time to the group
  // whose CTAs carry the most tiles, while CTAs are left. Every tile counts in full, the partial
  // last one too: measured, its MMAs, FP8 conversion and barriers cost about as much as a full
  // tile's (weighting it by its bytes left one CTA with 79 such tiles and doubled the FP8 pass)
  std::vector<int64_t> width(p.colgroups);
  std::vector<int> R(p.colgroups);
  int used = 0;
  for (int g = 0; g < p.colgroups; ++g) {
    width[g] = std::min<int64_t>(p.coltiles, (g + 1) * p.tiles_per_group) - g * p.tiles_per_group;
    int r = static_cast<int>(static_cast<double>(sms) * width[g] / p.coltiles);
    r = std::max(1, std::min<int>(r, static_cast<int>(p.rowblocks)));
    R[g] = r;
    used += r;
  }
  while (used > sms) {   // rounding can only overshoot through the max(1, .)
    int g = static_cast<int>(std::max_element(R.begin(), R.end()) - R.begin());
    if (R[g] <= 1) break;
    --R[g];
    --used;
  }
  auto load = [&](int g) { return cdiv(p.rowblocks, R[g]) * width[g]; };
  while (used < sms) {
    int best = -1;
    for (int g = 0; g < p.colgroups; ++g)
      if (R[g] < p.rowblocks && (best < 0 || load(g) > load(best))) best = g;
    if (best < 0) break;
    ++R[best];
    ++used;
  }
  p.gt.table = 1;
  p.gt.cta0[0] = 0;
  p.rowgroups = 0;
  for (int g = 0; g < p.colgroups; ++g) {
    p.gt.cta0[g + 1] = p.gt.cta0[g] + R[g];
    p.rowgroups = std::max(p.rowgroups, R[g]);
  }
  p.ctas = p.gt.cta0[p.colgroups];
  return p;
}

template <int LP, int SPLIT, int XK>
cudaError_t launch_t(const Launcher& L, const CUtensorMap& mx, const CUtensorMap& mv,
                     const CUtensorMap& mu, const TcArgs& a, size_t smem) {
  auto k = dual_pass_tc_kernel<LP, SPLIT, XK>;
  if (smem < 120 * 1024) smem = 120 * 1024;   // one CTA per SM: it owns the tensor memory
  cudaError_t err =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  dim3 grid(a.gt.table ? a.gt.cta0[a.n_colgroups] : a.n_colgroups * a.n_rowgroups);
  k<<<grid, XK != kXkBf16 ? kThreadsF8 : kThreads, smem, L.stream>>>(mx, mv, mu, a);
  L.count();
  return cudaGetLastError();
}

template <int SPLIT, int XK>
cudaError_t launch_lp(int LP, const Launcher& L, const CUtensorMap& mx, const CUtensorMap& mv,
                      const CUtensorMap& mu, const TcArgs& a, size_t smem) {
  switch (LP) {
    case 16: return launch_t<16, SPLIT, XK>(L, mx, mv, mu, a, smem);
    case 32: return launch_t<32, SPLIT, XK>(L, mx, mv, mu, a, smem);
    case 48: return launch_t<48, SPLIT, XK>(L, mx, mv, mu, a, smem);
    case 64: return launch_t<64, SPLIT, XK>(L, mx, mv, mu, a, smem);
    case 80: return launch_t<80, SPLIT, XK>(L, mx, mv, mu, a, smem);
    case 96: return launch_t<96, SPLIT, XK>(L, mx, mv, mu, a, smem);
    case 112: return launch_t<112, SPLIT, XK>(L, mx, mv, mu, a, smem);
    case 128: return launch_t<128, SPLIT, XK>(L, mx, mv, mu, a, smem);
    default: return cudaErrorInvalidValue;
  }
}

// FP32 X: the split bases fit shared memory up to LP = 80
cudaError_t launch_lp_f32(int LP, const Launcher& L, const CUtensorMap& mx, const CUtensorMap& mv,
                          const CUtensorMap& mu, const TcArgs& a, size_t smem) {
  switch (LP) {
    case 16: return launch_t<16, 2, kXkF32>(L, mx, mv, mu, a, smem);
    case 32: return launch_t<32, 2, kXkF32>(L, mx, mv, mu, a, smem);
    case 48: return launch_t<48, 2, kXkF32>(L, mx, mv, mu, a, smem);
    case 64: return launch_t<64, 2, kXkF32>(L, mx, mv, mu, a, smem);
    case 80: return launch_t<80, 2, kXkF32>(L, mx, mv, mu, a, smem);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool dual_pass_tc_supported(int64_t m, int64_t n, int64_t ldx, int ell, const void* X) {
  if (ell < 1 || ell > 128) return false;
  if (ldx % 8 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return false;
  if (m > (int64_t(1) << 31) - kRows || n > (int64_t(1) << 31) - kCols) return false;
  return encode_fn() != nullptr;
}

bool dual_pass_tc_split_supported(int ell) {
  int s = 0, k = 0;
  pick_stages(lp16(ell), 2, &s, &k);
  return ell >= 1 && ell <= 128 && k > 0;
}

bool dual_pass_tc_f32_supported(int64_t m, int64_t n, int64_t ldx, int ell, const void* X) {
  if (ell < 1 || ell > 80) return false;
  // TMA: 16-byte aligned base and row pitch; every box starts at a column multiple of 32
  if (ldx % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return false;
  if (m > (int64_t(1) << 31) - kRows || n > (int64_t(1) << 31) - kCols) return false;
  int s = 0, k = 0, u = 0;
  pick_stages(lp16(ell), 2, &s, &k, kXkF32, &u);
  return k > 0 && encode_fn() != nullptr;
}

size_t dual_pass_tc_ws_bytes(int64_t m, int64_t n, int ell) {
  // the largest of the layouts (plain and split operands, BF16, FP8 and FP32 X)
  size_t best = 0;
  for (int v = 0; v < 4; ++v) {
    const int split = (v == 1 || v == 3) ? 2 : 1;
    const int xk = v == 2 ? kXkF8 : v == 3 ? kXkF32 : kXkBf16;
    if (v == 3 && ell > 80) continue;
    const Plan p = plan_for(m, n, ell, split, xk);
    const int64_t ldv = (n + 7) / 8 * 8, ldu = (m + 7) / 8 * 8;
    const size_t b =
        sizeof(float) * static_cast<size_t>(p.colgroups * m * ell + p.rowgroups * n * ell) +
        2 * static_cast<size_t>(split * p.LP) * (ldv + ldu) + 4096;
    if (b > best) best = b;
  }
  return best;
}

namespace {

// Operand preparation, the kernel and the slot sums for one dual pass; mx maps X (BF16 halves of
// 128 x 64, FP8 tiles of 128 x 128, or FP32 boxes of 128 x 32), S / tn the FP8 tile scales.
cudaError_t run_tc(const Launcher& L, const CUtensorMap& mx, int xk, const uint8_t* S, int64_t tn,
                   int64_t m, int64_t n, int ell, const float* V, const float* U, float* Y,
                   float* Z, void* ws, int* status, int sp, bool z_kmajor) {
  const Plan p = plan_for(m, n, ell, sp, xk);
  if (p.nct < 1) return cudaErrorInvalidValue;
  const int64_t ldv = (n + 7) / 8 * 8, ldu = (m + 7) / 8 * 8;
  char* w = static_cast<char*>(ws);
  float* Ypart = reinterpret_cast<float*>(w);
  uintptr_t q = reinterpret_cast<uintptr_t>(Ypart + p.colgroups * m * ell);
  q = (q + 255) & ~uintptr_t(255);   // 16-byte loads of the slot sums
  float* Zpart = reinterpret_cast<float*>(q);
  q = reinterpret_cast<uintptr_t>(Zpart + p.rowgroups * n * ell);
  q = (q + 255) & ~uintptr_t(255);
  __nv_bfloat16* Vt = reinterpret_cast<__nv_bfloat16*>(q);
  q += 2 * static_cast<size_t>(sp * p.LP) * ldv;
  q = (q + 255) & ~uintptr_t(255);
  __nv_bfloat16* Ut = reinterpret_cast<__nv_bfloat16*>(q);
  {
    const int nbv = static_cast<int>(cdiv(ldv, 32));
    dim3 g(static_cast<unsigned>(nbv + cdiv(ldu, 32)), static_cast<unsigned>(cdiv(p.LP, 32)));
    prep_operands_kernel<<<g, dim3(32, 8), 0, L.stream>>>(V, n, ldv, Vt, U, m, ldu, Ut, ell, p.LP,
                                                          sp, nbv);
    L.count();
  }
  CUtensorMap mv, mu;
  if (!make_map(&mv, Vt, static_cast<uint64_t>(ldv), static_cast<uint64_t>(sp * p.LP),
                static_cast<uint64_t>(ldv), kHalfCols, static_cast<uint32_t>(p.LP)) ||
      !make_map(&mu, Ut, static_cast<uint64_t>(ldu), static_cast<uint64_t>(sp * p.LP),
                static_cast<uint64_t>(ldu), kHalfCols, static_cast<uint32_t>(p.LP)))
    return cudaErrorInvalidValue;
  TcArgs a;
  a.m = m;
  a.n = n;
  a.ell = ell;
  a.n_rowgroups = p.rowgroups;
  a.n_colgroups = p.colgroups;
  a.n_rowblocks = p.rowblocks;
  a.tiles_per_group = p.tiles_per_group;
  a.stages = p.stages;
  a.n_coltiles = p.coltiles;
  a.Ypart = Ypart;
  a.Zpart = Zpart;
  a.gt = p.gt;
  a.status = status;
  a.S = S;
  a.tn = tn;
  a.nub = p.nub;
  const size_t smem = smem_bytes(p.LP, sp, p.stages, p.tiles_per_group, xk, p.nub);
  cudaError_t err = xk == kXkF8 ? launch_lp<1, kXkF8>(p.LP, L, mx, mv, mu, a, smem)
                    : xk == kXkF32 ? launch_lp_f32(p.LP, L, mx, mv, mu, a, smem)
                    : sp == 2      ? launch_lp<2, kXkBf16>(p.LP, L, mx, mv, mu, a, smem)
                                   : launch_lp<1, kXkBf16>(p.LP, L, mx, mv, mu, a, smem);
  if (err != cudaSuccess) return err;
  const int by = static_cast<int>(cdiv(m, kRedRows));
  dim3 gr(static_cast<unsigned>(by + cdiv(n, kRedRows)), static_cast<unsigned>(cdiv(ell, 8)));
  reduce_pass_kernel<<<gr, 256, 0, L.stream>>>(Ypart, p.colgroups, m, Y, Zpart, p.rowgroups, n, Z,
                                               ell, z_kmajor ? 1 : 0, by, p.tiles_per_group, p.gt);
  L.count();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dual_pass_tc(const Launcher& L, const __nv_bfloat16* X, int64_t m, int64_t n,
                                int64_t ldx, int ell, const float* V, const float* U, float* Y,
                                float* Z, void* ws, size_t ws_bytes, int* status, bool split,
                                bool z_kmajor) {
  if (ws_bytes < dual_pass_tc_ws_bytes(m, n, ell)) return cudaErrorInvalidValue;
  const int sp = (split && dual_pass_tc_split_supported(ell)) ? 2 : 1;
  CUtensorMap mx;
  if (!make_map(&mx, X, static_cast<uint64_t>(n), static_cast<uint64_t>(m),
                static_cast<uint64_t>(ldx), kHalfCols, kRows))
    return cudaErrorInvalidValue;
  return run_tc(L, mx, kXkBf16, nullptr, 0, m, n, ell, V, U, Y, Z, ws, status, sp, z_kmajor);
}

cudaError_t launch_dual_pass_tc_f32(const Launcher& L, const float* X, int64_t m, int64_t n,
                                    int64_t ldx, int ell, const float* V, const float* U, float* Y,
                                    float* Z, void* ws, size_t ws_bytes, int* status,
                                    bool z_kmajor) {
  if (ws_bytes < dual_pass_tc_ws_bytes(m, n, ell) || !dual_pass_tc_f32_supported(m, n, ldx, ell, X))
    return cudaErrorInvalidValue;
  CUtensorMap mx;
  if (!make_map_f32(&mx, X, static_cast<uint64_t>(n), static_cast<uint64_t>(m),
                    static_cast<uint64_t>(ldx), kCols, 32, CU_TENSOR_MAP_L2_PROMOTION_L2_256B))
    return cudaErrorInvalidValue;
  return run_tc(L, mx, kXkF32, nullptr, 0, m, n, ell, V, U, Y, Z, ws, status, 2, z_kmajor);
}

bool dual_pass_tc_fp8_supported(int64_t m, int64_t n, int ell, const void* Xq) {
  if (ell < 1 || ell > 128 || (reinterpret_cast<uintptr_t>(Xq) & 15) != 0) return false;
  if (m < kRows || n < kCols) return false;   // the 128 x 128 box stays within the tensor
  if (m > (int64_t(1) << 31) - kRows || n > (int64_t(1) << 31) - kCols) return false;
  int s = 0, k = 0;
  pick_stages(lp16(ell), 1, &s, &k, kXkF8);
  return k > 0 && encode_fn() != nullptr;
}

cudaError_t launch_dual_pass_tc_fp8(const Launcher& L, const uint8_t* Xq, int64_t m, int64_t n,
                                    int ell, const float* V, const float* U, float* Y, float* Z,
                                    void* ws, size_t ws_bytes, int* status, bool z_kmajor) {
  if (ws_bytes < dual_pass_tc_ws_bytes(m, n, ell)) return cudaErrorInvalidValue;
  int64_t ldq = 0, off = 0;
  fp8_copy_bytes(m, n, &ldq, &off);
  CUtensorMap mx;
  if (!make_map8(&mx, Xq, static_cast<uint64_t>(n), static_cast<uint64_t>(m),
                 static_cast<uint64_t>(ldq)))
    return cudaErrorInvalidValue;
  return run_tc(L, mx, kXkF8, Xq + off, (n + 31) / 32, m, n, ell, V, U, Y, Z, ws, status, 1,
                z_kmajor);
}

}  // namespace nmfrp
