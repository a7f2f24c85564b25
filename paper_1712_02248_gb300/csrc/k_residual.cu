// Full-size residual of Eq. 2.2: ||X - W H||_F^2 and ||X||_F^2 in one read of X.
//
// Streaming kernel (X rows 16-byte aligned): one persistent block per SM walks a contiguous range
// of 128 x 64 tiles of X in row-block-major order. X tiles and the matching 64 columns of H arrive through a 2-stage
// cp.async pipeline in shared memory (two blocks per SM); the 128 rows of W (transposed) are staged once per row
// block. Each thread rebuilds 8 x 4 outputs of W H in registers (K = r FMAs each) and adds
// (x - wh)^2 and x^2 to per-thread sums. Per-tile sums are FP32 (32 terms), accumulated across
// tiles in float-float (FSum: the FP64 pipe of this GPU is too narrow for a per-tile FP64 add);
// block sums and the final sum are FP64 in a fixed order (deterministic).
//
// General kernel (any ldx): a block walks 128 x 128 tiles, staging W and H per tile, with its X
// loads issued first so that their latency overlaps the W H arithmetic.
#include <mutex>

#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kT = 128, kThreads = 256;
constexpr int kWS = kT + 4;   // padded row of the transposed W tile

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads, 1) residual_kernel(
    const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx, const float* __restrict__ W,
    const float* __restrict__ H, int r, double* __restrict__ part, const int* gate) {
  if (gate && !*reinterpret_cast<const volatile int*>(gate)) return;
  extern __shared__ __align__(16) float sh[];
  float* WsT = sh;                 // [r][kWS]   W tile transposed
  float* Hs = WsT + r * kWS;       // [r][kT]
  __shared__ double red[2][kThreads / 32];
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int64_t tiles_c = cdiv(n, kT), tiles = cdiv(m, kT) * tiles_c;
  FSum se2, sx2;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t r0 = (tile / tiles_c) * kT, c0 = (tile % tiles_c) * kT;
    // X loads for this thread's 8 x 8 outputs: rows r0 + 8 ty + a, columns c0 + 4 tx + {0..3}
    // and c0 + 64 + 4 tx + {0..3}
    float xv[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t gr = r0 + 8 * ty + a;
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int64_t gc = c0 + 64 * g + 4 * tx;
        if (gr < m) {
          const float* xp = X + gr * ldx + gc;
          if (VEC && gc + 3 < n) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(xp));
            xv[a][4 * g] = v.x;
            xv[a][4 * g + 1] = v.y;
            xv[a][4 * g + 2] = v.z;
            xv[a][4 * g + 3] = v.w;
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[a][4 * g + q] = (gc + q < n) ? __ldcs(xp + q) : 0.f;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) xv[a][4 * g + q] = 0.f;
        }
      }
    }
    __syncthreads();
    // W tile: 128 rows x r, contiguous in global; stored transposed
    for (int i = t >> 3; i < kT; i += kThreads >> 3) {
      const int64_t gr = r0 + i;
      for (int k = t & 7; k < r; k += 8) WsT[k * kWS + i] = (gr < m) ? W[gr * r + k] : 0.f;
    }
    // H tile: r rows x 128 columns
    for (int k = t >> 5; k < r; k += kThreads >> 5) {
      for (int c = t & 31; c < kT; c += 32) {
        const int64_t gc = c0 + c;
        Hs[k * kT + c] = (gc < n) ? H[k * n + gc] : 0.f;
      }
    }
    __syncthreads();
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    for (int k = 0; k < r; ++k) {
      const float4 w0 = *reinterpret_cast<const float4*>(&WsT[k * kWS + 8 * ty]);
      const float4 w1 = *reinterpret_cast<const float4*>(&WsT[k * kWS + 8 * ty + 4]);
      const float4 h0 = *reinterpret_cast<const float4*>(&Hs[k * kT + 4 * tx]);
      const float4 h1 = *reinterpret_cast<const float4*>(&Hs[k * kT + 64 + 4 * tx]);
      const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
      const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(wv[a], hv[b], acc[a][b]);
    }
    // padded rows/columns have x = 0 and w h = 0 (zero-filled W, H tiles)
    float te = 0.f, tx2 = 0.f;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float d = xv[a][b] - acc[a][b];
        te = fmaf(d, d, te);
        tx2 = fmaf(xv[a][b], xv[a][b], tx2);
      }
    se2.add(te);
    sx2.add(tx2);
  }
  const double e2 = warp_sum(se2.value()), x2 = warp_sum(sx2.value());
  if ((t & 31) == 0) {
    red[0][t >> 5] = e2;
    red[1][t >> 5] = x2;
  }
  __syncthreads();
  if (t < 32) {
    double a = (t < kThreads / 32) ? red[0][t] : 0.0;
    double b = (t < kThreads / 32) ? red[1][t] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (t == 0) {
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = b;
    }
  }
}

// ---------------------------------------------------------------- streaming kernel

constexpr int kSR = 128, kSC = 64, kSThreads = 256, kSStages = 2;
constexpr int kXS = kSC + 4;   // padded X tile row (floats): rows 16 B apart mod 128 B

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct StreamGeom {
  int64_t m, n, ldx;
  int r, RS;                 // RS: stride of a staged H row (64 floats)
  int64_t tiles_c, tiles;    // column tiles per row block, all tiles
};

// Issue the cp.async copies of tile `tile` into stage buffers xs (kSR x kXS) and hs (r x kSC).
// Out-of-range rows / columns are not copied; the compute masks them.
__device__ __forceinline__ void stream_issue(const float* __restrict__ X, const float* __restrict__ H,
                                             const StreamGeom& g, int64_t tile, float* xs,
                                             float* hs) {
  const int64_t r0 = (tile / g.tiles_c) * kSR, c0 = (tile % g.tiles_c) * kSC;
  for (int e = threadIdx.x; e < kSR * (kSC / 4); e += kSThreads) {
    const int i = e / (kSC / 4), c4 = e % (kSC / 4);
    const int64_t gr = r0 + i, gc = c0 + 4 * c4;
    if (gr < g.m && gc + 3 < g.n) cp_async16(xs + i * kXS + 4 * c4, X + gr * g.ldx + gc);
  }
  for (int e = threadIdx.x; e < g.r * (kSC / 4); e += kSThreads) {
    const int k = e / (kSC / 4), c4 = e % (kSC / 4);
    const int64_t gc = c0 + 4 * c4;
    if (gc + 3 < g.n) cp_async16(hs + k * g.RS + 4 * c4, H + static_cast<int64_t>(k) * g.n + gc);
  }
}

__global__ void __launch_bounds__(kSThreads, 2) residual_stream_kernel(
    const float* __restrict__ X, const float* __restrict__ W, const float* __restrict__ H,
    StreamGeom g, double* __restrict__ part, const int* gate) {
  if (gate && !*reinterpret_cast<const volatile int*>(gate)) return;
  extern __shared__ __align__(16) float sh[];
  const int r = g.r;
  const int stage_f = kSR * kXS + r * kSC;     // floats per stage
  float* WsT = sh + kSStages * stage_f;         // [r][kSR + 4]
  const int WS = kSR + 4;
  __shared__ double red[2][kSThreads / 32];
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;   // rows 8 ty + a, columns 4 tx + b
  FSum se2, sx2;
  // tiles of this block: a contiguous range (W is staged again only when the range crosses
  // into the next row block)
  const int64_t first = blockIdx.x * g.tiles / gridDim.x;
  const int64_t mine = (blockIdx.x + 1) * g.tiles / gridDim.x - first;
  const int64_t step = 1;
  // prologue: stages 0 .. kSStages - 2
  for (int s = 0; s < kSStages - 1; ++s) {
    if (s < mine) stream_issue(X, H, g, first + s * step, sh + s * stage_f, sh + s * stage_f + kSR * kXS);
    cp_async_commit();
  }
  int64_t cur_rb = -1;
  for (int64_t k = 0; k < mine; ++k) {
    // keep kSStages - 1 tiles in flight: issue tile k + kSStages - 1 into the stage freed last
    {
      const int64_t nk = k + kSStages - 1;
      const int s = static_cast<int>(nk % kSStages);
      if (nk < mine) stream_issue(X, H, g, first + nk * step, sh + s * stage_f, sh + s * stage_f + kSR * kXS);
      cp_async_commit();
    }
    const int64_t tile = first + k * step;
    const int64_t rb = tile / g.tiles_c, r0 = rb * kSR, c0 = (tile % g.tiles_c) * kSC;
    if (rb != cur_rb) {
      // W rows of this row block, transposed (plain loads: once per row block)
      __syncthreads();
      for (int e = t; e < kSR * r; e += kSThreads) {
        const int i = e / r, kk = e - i * r;
        const int64_t gr = r0 + i;
        WsT[kk * WS + i] = gr < g.m ? W[gr * r + kk] : 0.f;
      }
      cur_rb = rb;
    }
    cp_async_wait<kSStages - 1>();
    __syncthreads();
    const float* xs = sh + (k % kSStages) * stage_f;
    const float* hs = xs + kSR * kXS;
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
    for (int kk = 0; kk < r; ++kk) {
      const float4 w0 = *reinterpret_cast<const float4*>(&WsT[kk * WS + 8 * ty]);
      const float4 w1 = *reinterpret_cast<const float4*>(&WsT[kk * WS + 8 * ty + 4]);
      const float4 h0 = *reinterpret_cast<const float4*>(&hs[kk * g.RS + 4 * tx]);
      const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
      const float hv[4] = {h0.x, h0.y, h0.z, h0.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wv[a], hv[b], acc[a][b]);
    }
    float te = 0.f, tx2 = 0.f;
    const bool cols_in = c0 + 4 * tx + 3 < g.n;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const bool in = cols_in && (r0 + 8 * ty + a < g.m);
      const float4 x4 = *reinterpret_cast<const float4*>(&xs[(8 * ty + a) * kXS + 4 * tx]);
      const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float xb = in ? xv[b] : 0.f;
        const float d = in ? xb - acc[a][b] : 0.f;
        te = fmaf(d, d, te);
        tx2 = fmaf(xb, xb, tx2);
      }
    }
    se2.add(te);
    sx2.add(tx2);
    __syncthreads();   // the stage is reused by the copies issued at the next step
  }
  cp_async_wait<0>();
  const double e2 = warp_sum(se2.value()), x2 = warp_sum(sx2.value());
  if ((t & 31) == 0) {
    red[0][t >> 5] = e2;
    red[1][t >> 5] = x2;
  }
  __syncthreads();
  if (t < 32) {
    double a = (t < kSThreads / 32) ? red[0][t] : 0.0;
    double b = (t < kSThreads / 32) ? red[1][t] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (t == 0) {
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = b;
    }
  }
}

__global__ void residual_final_kernel(const double* __restrict__ part, int nparts,
                                      double* __restrict__ out2, const int* gate) {
  if (gate && !*reinterpret_cast<const volatile int*>(gate)) return;
  const int t = threadIdx.x;  // one warp
  double a = 0.0, b = 0.0;
  for (int i = t; i < nparts; i += 32) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (t == 0) {
    out2[0] = a;
    out2[1] = b;
  }
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

// upper bound on the grid (blocks per SM is at most 4 for this kernel)
int residual_grid() { return num_sms() * 4; }

}  // namespace

size_t residual_ws_bytes(int64_t, int64_t) {
  return sizeof(double) * 2 * static_cast<size_t>(residual_grid()) + 256;
}

size_t residual_ws_bytes_tc(int64_t m, int64_t n) {
  return residual_ws_bytes(m, n) + residual_tc_operand_bytes(m, n);
}

cudaError_t launch_residual(const Launcher& L, const float* X, int64_t m, int64_t n, int64_t ldx,
                            const float* W, const float* H, int r, double* out2, void* ws,
                            size_t ws_bytes, const int* gate, int* status) {
  if (ws_bytes < residual_ws_bytes(m, n)) return cudaErrorInvalidValue;
  double* part = static_cast<double*>(ws);
  // tensor-core rebuild of W H when the workspace holds its split operands
  if (ws_bytes >= residual_ws_bytes_tc(m, n) && residual_tc_supported(m, n, ldx, X, r)) {
    const size_t pb = residual_ws_bytes(m, n);
    int grid = 0;
    cudaError_t err = launch_residual_tc(L, X, m, n, ldx, W, H, r, part, residual_grid(), &grid,
                                         static_cast<char*>(ws) + pb, ws_bytes - pb, status, gate);
    if (err != cudaSuccess) return err;
    residual_final_kernel<<<1, 32, 0, L.stream>>>(part, grid, out2, gate);
    L.count();
    return cudaGetLastError();
  }
  // streaming kernel: rows 16-byte aligned, columns a multiple of 4 (the ragged tail of a row
  // would need element copies), W H rank small enough for the shared-memory stages (r <= 48)
  if (ldx % 4 == 0 && n % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
      reinterpret_cast<uintptr_t>(H) % 16 == 0 && r <= 48) {
    StreamGeom g;
    g.m = m;
    g.n = n;
    g.ldx = ldx;
    g.r = r;
    g.RS = kSC;
    g.tiles_c = cdiv(n, kSC);
    g.tiles = cdiv(m, kSR) * g.tiles_c;
    const size_t sm = sizeof(float) * (static_cast<size_t>(kSStages) * (kSR * kXS + r * kSC) +
                                       static_cast<size_t>(r) * (kSR + 4));
    cudaError_t err = cudaFuncSetAttribute(residual_stream_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(sm));
    if (err != cudaSuccess) return err;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, residual_stream_kernel, kSThreads,
                                                      sm) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    int grid = num_sms() * (per_sm < 2 ? per_sm : 2);
    if (g.tiles < grid) grid = static_cast<int>(g.tiles);
    residual_stream_kernel<<<grid, kSThreads, sm, L.stream>>>(X, W, H, g, part, gate);
    residual_final_kernel<<<1, 32, 0, L.stream>>>(part, grid, out2, gate);
    L.count(2);
    return cudaGetLastError();
  }
  const int64_t tiles = cdiv(m, kT) * cdiv(n, kT);
  const size_t sm = sizeof(float) * (r * kWS + r * kT);
  const bool vec = (ldx % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  auto k = vec ? residual_kernel<true> : residual_kernel<false>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
  if (err != cudaSuccess) return err;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, sm) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  int grid = num_sms() * (per_sm < 4 ? per_sm : 4);
  if (tiles < grid) grid = static_cast<int>(tiles);
  k<<<grid, kThreads, sm, L.stream>>>(X, m, n, ldx, W, H, r, part, gate);
  residual_final_kernel<<<1, 32, 0, L.stream>>>(part, grid, out2, gate);
  L.count(2);
  return cudaGetLastError();
}

namespace {

// sum of x^2 over X: FP32 within 4 elements, float-float across them, fixed-order FP64 block and
// final sums
__global__ void __launch_bounds__(256) sumsq_kernel(const float* __restrict__ X, int64_t m,
                                                    int64_t n, int64_t ldx,
                                                    double* __restrict__ part) {
  __shared__ double red[8];
  const bool vec = (ldx % 4 == 0) && (n % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  FSum sacc;
  if (vec) {
    const int64_t n4 = n / 4, total = m * n4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = e / n4, j = e - i * n4;
      const float4 v = __ldcs(reinterpret_cast<const float4*>(X + i * ldx) + j);
      sacc.add(fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w))));
    }
  } else {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = e / n, j = e - i * n;
      const float v = X[i * ldx + j];
      sacc.add(v * v);
    }
  }
  const double acc = warp_sum(sacc.value());
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = threadIdx.x < 8 ? red[threadIdx.x] : 0.0;
    a = warp_sum(a);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
  }
}

__global__ void sumsq_final_kernel(const double* __restrict__ part, int nparts,
                                   double* __restrict__ out) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) a += part[i];
  a = warp_sum(a);
  if (threadIdx.x == 0) *out = a;
}

}  // namespace

cudaError_t launch_sumsq(const Launcher& L, const float* X, int64_t m, int64_t n, int64_t ldx,
                         double* out, void* ws, size_t ws_bytes) {
  const int grid = num_sms() * 4;
  if (ws_bytes < sizeof(double) * grid) return cudaErrorInvalidValue;
  double* part = static_cast<double*>(ws);
  sumsq_kernel<<<grid, 256, 0, L.stream>>>(X, m, n, ldx, part);
  sumsq_final_kernel<<<1, 32, 0, L.stream>>>(part, grid, out);
  L.count(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- residual with static scratch
// A caller that cannot allocate device memory when it wants the residual (a serving loop whose
// device memory is all handed to its own pools, or code that must not stall the device's other
// streams, as cudaFree does by synchronising the device) gets the per-block partial sums in a
// fixed array of this module's global memory instead of a context workspace. Each block writes
// its two slots before the final sum reads them, so the array needs no clearing; two calls in
// flight on one device at the same time share it and race.
namespace {

// two doubles for each of up to 2048 blocks (4 a multiprocessor on devices of up to 512) plus the
// 256-byte alignment slack residual_ws_bytes counts: 33,024 bytes
constexpr int kStaticPartialDoubles = 2 * 4 * 512 + 32;
__device__ __align__(256) double g_residual_partials[kStaticPartialDoubles];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

}  // namespace

size_t residual_static_capacity_bytes() { return sizeof(double) * kStaticPartialDoubles; }

cudaError_t residual_static_scratch(int device, void** addr) {
  if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  if (cur != device) return cudaErrorInvalidDevice;   // set-up needs the device current
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_residual_partials);
    if (e != cudaSuccess) return e;
    g_static_addr[device] = p;
  }
  *addr = g_static_addr[device];
  return cudaSuccess;
}

}  // namespace nmfrp
