// Full-size residual of Eq. 2.2, ||X - W H||_F^2 and ||X||_F^2, with the W H rebuild on the
// 5th-generation tensor cores: FP32 X (rows 16-byte aligned), r <= 32.
//
// A tile of X (64 rows i0 .., 128 columns c0 ..) is compared with the transposed product tile
//   D = (W H)^T [c0 .., i0 ..] = H_tile^T W_tile^T   (M = 128 columns, N = 64 rows, K = r)
// accumulated in tensor memory from three-term BF16 splits of W and H: v = v1 + v2 + v3 with
// v1 = bf16(v), v2 = bf16(v - v1), v3 = bf16(v - v1 - v2) (the differences are exact in FP32),
// so v is represented to about 2^-25; the six products of significance >= 2^-16 (11, 12, 21,
// 13, 22, 31) are accumulated in FP32, leaving each entry of W H within a few units of 2^-24 of
// its value, the accuracy of an FP32 rebuild. Each column of H and row of W holds two 128-byte
// rows of BF16 K entries: [v1 | v2] (32 entries each, r used, zeros after) and [v3 | 0].
//
// TMA stages the X tile (one 128-column box, 32 KB, rows of 512 B) with the two halves of the H
// tile of its 128 columns (32 KB) and, once per row block, the two halves of the W tile (16 KB).
// An epilogue warp reads TMEM lanes 32 q .. 32 q + 31 of its quarter q, i.e. columns c0 + 32 q +
// lane: each 32x32b.x16 load gives a thread 16 consecutive rows of D for its column, and the
// warp reads the matching x of one row from shared memory as 32 consecutive floats
// (conflict-free). Per tile, (x - wh)^2 and x^2 are summed in FP32 (64 terms a thread), carried
// across tiles in float-float, and summed over the block in FP64 (fixed order).
//
// Warp roles (192 threads): warps 0-3 epilogue, warp 4 TMA, warp 5 TMEM allocation and MMAs.
// A CTA takes a contiguous range of tiles ordered row block by row block, so consecutive tiles
// continue the same 64 rows of X (DRAM locality) and the W tile stays resident while the column
// tiles of one row block pass. Every wait is bounded; on time-out
// the kernel latches NMF_ERR_TIMEOUT, drains what it issued and frees its tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nmfrp {
namespace {

using namespace tc;

constexpr int kRC = 128;                   // tile columns (MMA M, TMEM lanes)
constexpr int kRR = 64;                    // tile rows (MMA N, TMEM columns)
constexpr int kEpiWarps = 4;               // epilogue warps: kEpiWarps / 4 a TMEM lane quarter
constexpr int kRThreads = 32 * (kEpiWarps + 2);
constexpr int kProdWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kRStagesUsed = 3;
constexpr int kWBufs = 1;                  // W tiles resident at a time (a new row block waits)
constexpr uint32_t kXTile = kRC * kRR * 4;   // the X tile, one 128-column box: 32 KB
constexpr uint32_t kWHalf = kRR * 128;     // 64 rows x 128 B of BF16 K entries: 8 KB
constexpr uint32_t kHHalf = kRC * 128;     // 128 rows x 128 B: 16 KB
constexpr uint32_t kTmemCols = 128;        // two 64-column D buffers

struct RtArgs {
  int64_t m, n;
  int nk;                // K steps of 16 (1 for r <= 16, else 2)
  int64_t nct, tiles;    // column tiles, all tiles
  double* part;          // 2 doubles a block
  int* status;
  const int* gate;
};

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 64.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            (static_cast<uint32_t>(kRR >> 3) << 17) |
                            (static_cast<uint32_t>(kRC >> 4) << 24);

__global__ void __launch_bounds__(kRThreads, 1) residual_tc_kernel(
    const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapW,
    const __grid_constant__ CUtensorMap mapH, RtArgs a) {
  if (a.gate && !*reinterpret_cast<const volatile int*>(a.gate)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* Xs = smem;                                  // [stages][32 KB]
  unsigned char* Hs = Xs + kRStagesUsed * kXTile;            // [stages][2 halves][16 KB]
  unsigned char* Ws = Hs + kRStagesUsed * 2 * kHHalf;        // [kWBufs][2 halves][8 KB]
  __shared__ __align__(8) uint64_t full_bar[kRStagesUsed], empty_bar[kRStagesUsed];
  __shared__ __align__(8) uint64_t wfull[kWBufs], wempty[kWBufs], dfull[2], dfree[2], drain_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_f;
  __shared__ double red[2][kRThreads / 32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t t0 = blockIdx.x * a.tiles / G, t1 = (blockIdx.x + 1) * a.tiles / G;
  const int T = static_cast<int>(t1 - t0);

  if (threadIdx.x == 0) {
    abort_f = 0;
    for (int s = 0; s < kRStagesUsed; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1 + kEpiWarps);   // the MMAs (H) and the epilogue (X)
    }
    for (int b = 0; b < kWBufs; ++b) {
      mbar_init(smem_u32(&wfull[b]), 1);
      mbar_init(smem_u32(&wempty[b]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&dfull[b]), 1);
      mbar_init(smem_u32(&dfree[b]), kEpiWarps);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&tmem_base), kTmemCols);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  FSum se2, sx2;

  if (warp == kProdWarp) {
    // ---------------- TMA producer
    if (lane == 0 && T > 0) {
      const uint64_t pol_x = policy_evict_first(), pol_b = policy_evict_last();
      int issued = 0, wloads = 0;
      int64_t prev_rb = -1;
      for (int k = 0; k < T; ++k) {
        const int64_t g = t0 + k, rb = g / a.nct, ct = g - rb * a.nct;
        if (rb != prev_rb) {
          const int wb = wloads % kWBufs;
          if (!mbar_wait(smem_u32(&wempty[wb]), ((wloads / kWBufs) & 1) ^ 1, &abort_f)) break;
          const uint32_t wbar = smem_u32(&wfull[wb]);
          mbar_expect_tx(wbar, 2 * kWHalf);
          for (int hf = 0; hf < 2; ++hf)
            tma_load_2d(smem_u32(Ws + (2 * wb + hf) * kWHalf), &mapW, 64 * hf,
                        static_cast<int>(rb * kRR), wbar, pol_b);
          ++wloads;
          prev_rb = rb;
        }
        const int s = k % kRStagesUsed;
        if (!mbar_wait(smem_u32(&empty_bar[s]), ((k / kRStagesUsed) & 1) ^ 1, &abort_f)) break;
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, kXTile + 2 * kHHalf);
        tma_load_2d(smem_u32(Xs + s * kXTile), &mapX, static_cast<int>(ct * kRC),
                    static_cast<int>(rb * kRR), fb, pol_x);
        for (int hf = 0; hf < 2; ++hf)
          tma_load_2d(smem_u32(Hs + (2 * s + hf) * kHHalf), &mapH, 64 * hf,
                      static_cast<int>(ct * kRC), fb, pol_b);
        issued = k + 1;
      }
      // every copy issued has landed before the CTA may leave
      for (int w = wloads - kWBufs > 0 ? wloads - kWBufs : 0; w < wloads; ++w)
        mbar_drain(smem_u32(&wfull[w % kWBufs]), (w / kWBufs) & 1);
      for (int k = issued - kRStagesUsed > 0 ? issued - kRStagesUsed : 0; k < issued; ++k)
        mbar_drain(smem_u32(&full_bar[k % kRStagesUsed]), (k / kRStagesUsed) & 1);
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer
    if (lane == 0 && T > 0) {
      bool ok = true;
      int wloads = 0, wb = 0;
      int64_t prev_rb = -1;
      for (int k = 0; k < T && ok; ++k) {
        const int64_t g = t0 + k, rb = g / a.nct;
        if (rb != prev_rb) {
          wb = wloads % kWBufs;
          if (!mbar_wait(smem_u32(&wfull[wb]), (wloads / kWBufs) & 1, &abort_f)) {
            ok = false;
            break;
          }
          ++wloads;
          prev_rb = rb;
        }
        const int s = k % kRStagesUsed, db = k & 1;
        if (!mbar_wait(smem_u32(&full_bar[s]), (k / kRStagesUsed) & 1, &abort_f) ||
            !mbar_wait(smem_u32(&dfree[db]), ((k >> 1) & 1) ^ 1, &abort_f)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // the three terms of each split: term 1 at byte 0 and term 2 at byte 64 of the first
        // half's 128-byte rows, term 3 at byte 0 of the second half's
        const uint32_t ah = smem_u32(Hs + 2 * s * kHHalf), bw = smem_u32(Ws + 2 * wb * kWHalf);
        const uint32_t at[3] = {ah, ah + 64, ah + kHHalf};
        const uint32_t bt[3] = {bw, bw + 64, bw + kWHalf};
        const uint32_t d = tmem + static_cast<uint32_t>(db * kRR);
        // (A term, B term) pairs of significance >= 2^-16
        const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
        for (int kk = 0; kk < a.nk; ++kk) {
          const uint32_t o = 32u * kk;   // bytes of 16 BF16 K entries
#pragma unroll
          for (int u = 0; u < 6; ++u)
            mma_bf16(d, sdesc(at[pa[u]] + o, 16, 1024), sdesc(bt[pb[u]] + o, 16, 1024), kIdesc,
                     (kk > 0 || u > 0) ? 1u : 0u);
        }
        mma_commit(smem_u32(&empty_bar[s]));
        mma_commit(smem_u32(&dfull[db]));
        const bool last_of_rb = (k + 1 == T) || ((t0 + k + 1) / a.nct != rb);
        if (last_of_rb) mma_commit(smem_u32(&wempty[wb]));
      }
      // all MMAs issued by this thread complete before tensor memory is freed
      mma_commit(smem_u32(&drain_bar));
      mbar_drain(smem_u32(&drain_bar), 0);
    }
  } else {
    // ---------------- epilogue: warp w reads TMEM lanes (columns) 32 (w % 4) .. + 31 (a warp may
    // only touch its sub-partition's lanes) and its share of the tile's rows
    constexpr int kChunks = kRR / 16 / (kEpiWarps / 4);   // 16-row TMEM loads a warp
    const int quarter = warp & 3, part = warp >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    float v[16];
    for (int k = 0; k < T; ++k) {
      const int s = k % kRStagesUsed, db = k & 1;
      // the whole warp leaves together (the TMEM loads below need all 32 lanes)
      const bool ok = mbar_wait(smem_u32(&dfull[db]), (k >> 1) & 1, &abort_f) &&
                      mbar_wait(smem_u32(&full_bar[s]), (k / kRStagesUsed) & 1, &abort_f);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const float* xs = reinterpret_cast<const float*>(Xs + s * kXTile) + 32 * quarter;
      float te = 0.f, tx = 0.f;
#pragma unroll 1
      for (int q = kChunks * part; q < kChunks * (part + 1); ++q) {
        tmem_ld16(tmem + lane_base + static_cast<uint32_t>(db * kRR + 16 * q), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float x = xs[(16 * q + j) * kRC + lane];
          const float dd = x - v[j];
          te = fmaf(dd, dd, te);
          tx = fmaf(x, x, tx);
        }
      }
      se2.add(te);
      sx2.add(tx);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&dfree[db]));
        mbar_arrive(smem_u32(&empty_bar[s]));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && abort_f) latch(a.status, kStTimeout);
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
  // block sums in FP64, fixed order
  double e2 = se2.value(), x2 = sx2.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
  }
  if (lane == 0) {
    red[0][warp] = e2;
    red[1][warp] = x2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double se = 0.0, sx = 0.0;
    for (int w = 0; w < kRThreads / 32; ++w) {
      se += red[0][w];
      sx += red[1][w];
    }
    a.part[2 * blockIdx.x] = se;
    a.part[2 * blockIdx.x + 1] = sx;
  }
}

// Rows of the split operands, 128 BF16 K entries each: [v1 | v2] in entries [0, 64) (32 each),
// [v3 | 0] in [64, 128), for the rows of W (rows < m) and the columns of H (row m + c = column c).
__global__ void split_rows_kernel(const float* __restrict__ W, int64_t m, const float* __restrict__ H,
                                  int64_t n, int r, __nv_bfloat16* __restrict__ Wsp,
                                  __nv_bfloat16* __restrict__ Hsp, const int* gate) {
  if (gate && !*reinterpret_cast<const volatile int*>(gate)) return;
  const int64_t total = (m + n) * 128;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = e >> 7;
    const int k = static_cast<int>(e & 127);
    const int j = k & 31, term = k >> 5;   // term 3 (k in [96, 128)) is padding
    float v = 0.f;
    if (j < r && term < 3) v = row < m ? W[row * r + j] : H[static_cast<int64_t>(j) * n + (row - m)];
    const float v1 = __bfloat162float(__float2bfloat16_rn(v));
    const float v2 = __bfloat162float(__float2bfloat16_rn(v - v1));
    const float t = term == 0 ? v1 : term == 1 ? v2 : v - v1 - v2;
    const __nv_bfloat16 out = __float2bfloat16_rn(term < 3 ? t : 0.f);
    if (row < m) Wsp[e] = out;
    else Hsp[e - m * 128] = out;
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

}  // namespace

bool residual_tc_supported(int64_t m, int64_t n, int64_t ldx, const float* X, int r) {
  if (r < 1 || r > 32 || ldx % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return false;
  if (m < 1 || n < 1 || m > (int64_t(1) << 31) - kRC || n > (int64_t(1) << 31) - kRC) return false;
  return encode_fn() != nullptr;
}

size_t residual_tc_operand_bytes(int64_t m, int64_t n) {
  return static_cast<size_t>(m + n) * 256 + 256;
}

cudaError_t launch_residual_tc(const Launcher& L, const float* X, int64_t m, int64_t n,
                               int64_t ldx, const float* W, const float* H, int r, double* part,
                               int max_grid, int* grid_out, void* ws, size_t ws_bytes, int* status,
                               const int* gate) {
  if (ws_bytes < residual_tc_operand_bytes(m, n) || max_grid < 1) return cudaErrorInvalidValue;
  uintptr_t q = (reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255);
  __nv_bfloat16* Wsp = reinterpret_cast<__nv_bfloat16*>(q);
  __nv_bfloat16* Hsp = Wsp + m * 128;   // (m * 256 bytes keeps 16-byte alignment)
  CUtensorMap mx, mw, mh;
  if (!make_map_f32(&mx, X, static_cast<uint64_t>(n), static_cast<uint64_t>(m),
                    static_cast<uint64_t>(ldx), kRC, kRR) ||
      !make_map(&mw, Wsp, 128, static_cast<uint64_t>(m), 128, 64, kRR) ||
      !make_map(&mh, Hsp, 128, static_cast<uint64_t>(n), 128, 64, kRC))
    return cudaErrorInvalidValue;
  // grid-stride over the (m + n) x 128 entries with a few blocks an SM: a check the error
  // monitor skips then costs one short wave instead of thousands of blocks that exit at once
  const int64_t tot = (m + n) * 128, cap = 4 * static_cast<int64_t>(sm_count());
  split_rows_kernel<<<static_cast<unsigned>(cdiv(tot, 256) < cap ? cdiv(tot, 256) : cap), 256, 0,
                      L.stream>>>(W, m, H, n, r, Wsp, Hsp, gate);
  RtArgs a;
  a.m = m;
  a.n = n;
  a.nk = r <= 16 ? 1 : 2;
  a.nct = cdiv(n, kRC);
  a.tiles = cdiv(m, kRR) * a.nct;
  a.part = part;
  a.status = status;
  a.gate = gate;
  int grid = sm_count() < max_grid ? sm_count() : max_grid;
  if (a.tiles < grid) grid = static_cast<int>(a.tiles);
  const size_t smem = kRStagesUsed * (kXTile + 2 * kHHalf) + kWBufs * 2 * kWHalf + 1024;
  cudaError_t err = cudaFuncSetAttribute(residual_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  residual_tc_kernel<<<grid, kRThreads, smem, L.stream>>>(mx, mw, mh, a);
  L.count(2);
  *grid_out = grid;
  return cudaGetLastError();
}

}  // namespace nmfrp
