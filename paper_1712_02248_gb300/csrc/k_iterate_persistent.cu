// All iterations of FastHALS-RP / MU-RP in one cooperative (persistent) launch.
//
// The update rules are those of k_iterate.cu (Section 4, Eq. fastHALS_a with the Section 4.1
// terms; Section 3.1, Algorithm 3 with the semi-NMF rule). Each block owns a fixed slice of the
// rows of W and of the columns of H for the whole run. One iteration is two phases:
//
//   A  (rows of W)   from H_tld, G_W: S_W row, sweep over j, W row written; the block adds its
//                    rows' contributions to W_tld_raw = Q_L^T W and to the column sums of
//                    squares into an FP64 accumulator (red.add.f64).
//   -- grid barrier --
//   B  (columns of H) every block reads W_tld_raw and the squares, forms s_j, W_tld = raw/s,
//                    G_H; compensation h_j *= s_j, S_H column, sweep; adds H Q_R contributions
//                    into the FP64 accumulator of H_tld.
//   -- grid barrier --
//
// Partial sums are FP32 within a block and FP64 across blocks; the order of the cross-block
// additions varies from run to run, but FP64 sums of FP32 values round back to the same FP32
// result except in rare ties. W's normalisation by s_j is applied when phase A of the next
// iteration (or the final pass) reads the row. Every wait is bounded: on time-out the kernel
// latches NMF_ERR_TIMEOUT and all blocks leave.
#include "common.cuh"

namespace nmfrp {
namespace {

constexpr int kPT = 256;          // threads per block
constexpr int kCopies = 8;        // copies of each cross-block accumulator (spreads the atomics)
constexpr long long kWaitCycles = 4000000000LL;   // about two seconds of polling before giving up

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
        __nanosleep(32);
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
  float alpha, beta, eps;
  const float* QL;
  const float* QR;
  const float* Xhat;
  const float* Xchk;
  float* W;
  float* H;
  double* accW;   // [2][kCopies][ell*r + r]
  double* accH;   // [2][kCopies][r*ell]
  Barrier* bar;
  int* status;
  int* abort_flag;
};

template <int RP, int RULE>
__global__ void __launch_bounds__(kPT) iterate_persistent_kernel(PArgs a) {
  extern __shared__ __align__(16) float sh[];
  const int r = a.r, ell = a.ell, t = threadIdx.x;
  const int EW = ell * r + r;  // W-phase partial entries: W_tld_raw (ell x r) + colsq (r)
  const int EH = r * ell;      // H-phase partial entries: H_tld (r x ell)
  float* HtT = sh;                   // [ell][RP]   H_tld^T
  float* Gw = HtT + ell * RP;        // [RP][RP]
  float* WtS = Gw + RP * RP;         // [ell][RP]   W_tld (normalised)
  float* Gh = WtS + ell * RP;        // [RP][RP]
  float* sc = Gh + RP * RP;          // [RP]        s_j of the last W phase
  float* stA = sc + RP;              // [kPT][r]    staged rows of W / columns of H
  float* stB = stA + kPT * RP;       // [kPT][ell]  staged rows of Q_L / rows of Q_R
  const unsigned G = gridDim.x;
  const int64_t rb = (a.m + G - 1) / G, cbk = (a.n + G - 1) / G;
  const int64_t r0 = blockIdx.x * rb, r1 = min(a.m, r0 + rb);
  const int64_t c0 = blockIdx.x * cbk, c1 = min(a.n, c0 + cbk);
  const bool normalize = (RULE == 0);

  for (int j = t; j < RP; j += kPT) sc[j] = 1.f;

  // H_tld partial of this block's columns of H into accH[slot]
  auto h_partial = [&](int slot, bool scale_h) {
    float acc[8];
    for (int64_t cc = c0; cc < c1; cc += kPT) {
      const int64_t c = cc + t;
      __syncthreads();
      if (c < c1) {
        for (int j = 0; j < r; ++j) stA[t * RP + j] = a.H[j * a.n + c] * (scale_h ? sc[j] : 1.f);
        for (int k = 0; k < ell; ++k) stB[t * ell + k] = a.QR[c * ell + k];
      } else {
        for (int j = 0; j < r; ++j) stA[t * RP + j] = 0.f;
        for (int k = 0; k < ell; ++k) stB[t * ell + k] = 0.f;
      }
      __syncthreads();
      const int cnt = static_cast<int>(c1 - cc < kPT ? c1 - cc : kPT);
      for (int e0 = 0; e0 < EH; e0 += kPT * 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kPT + t;
          if (e < EH) {
            const int j = e / ell, k = e - j * ell;
            float s = 0.f;
            for (int q = 0; q < cnt; ++q) s = fmaf(stA[q * RP + j], stB[q * ell + k], s);
            acc[u] = s;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kPT + t;
          if (e < EH)
            atomicAdd(&a.accH[(slot * kCopies + blockIdx.x % kCopies) * EH + e],
                      static_cast<double>(acc[u]));
        }
      }
    }
  };

  // prologue: H_tld of the initial H into accH[1]
  if (a.iters > 0) h_partial(1, false);
  if (!grid_sync(a.bar, G, a.status, a.abort_flag)) return;

  for (int it = 0; it < a.iters; ++it) {
    const int ph = it & 1;        // parity of this iteration's accumulators
    const int pr = ph ^ 1;        // parity of the previous ones
    // ---------------- phase A: rows of W
    // clear the W accumulators of the next iteration (last read one phase ago), a slice per block
    for (int64_t e = blockIdx.x * kPT + t; e < kCopies * EW; e += static_cast<int64_t>(G) * kPT)
      a.accW[pr * kCopies * EW + e] = 0.0;
    for (int e = t; e < ell * RP; e += kPT) {
      const int k = e / RP, j = e - k * RP;
      double v = 0.0;
      if (j < r)
        for (int c = 0; c < kCopies; ++c) v += a.accH[(pr * kCopies + c) * EH + j * ell + k];
      HtT[e] = static_cast<float>(v);
    }
    __syncthreads();
    for (int e = t; e < RP * RP; e += kPT) {
      const int p = e / RP, q = e - p * RP;
      float g = 0.f;
      if (p < r && q < r)
        for (int k = 0; k < ell; ++k) g = fmaf(HtT[k * RP + p], HtT[k * RP + q], g);
      Gw[e] = g;
    }
    __syncthreads();
    float accw[4];
    for (int64_t ii = r0; ii < r1; ii += kPT) {
      const int64_t i = ii + t;
      if (i < r1) {
        float w[RP], s[RP];
#pragma unroll
        for (int j = 0; j < RP; ++j) {
          w[j] = (j < r) ? a.W[i * r + j] / sc[j] : 0.f;
          s[j] = 0.f;
        }
        const float* xr = a.Xchk + i * ell;
        for (int k = 0; k < ell; ++k) {
          const float xk = xr[k];
#pragma unroll
          for (int j = 0; j < RP; ++j) s[j] = fmaf(xk, HtT[k * RP + j], s[j]);
        }
        if (RULE == 0) {
#pragma unroll
          for (int j = 0; j < RP; ++j) {
            const float g = Gw[j * RP + j];
            if (j < r && g > 0.f) {
              float tt = s[j];
#pragma unroll
              for (int q = 0; q < RP; ++q) tt = fmaf(-w[q], Gw[q * RP + j], tt);
              w[j] = fmaxf(0.f, w[j] + tt / g);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < RP; ++j) {
            float num = posp(s[j]), den = negp(s[j]) + a.eps;
#pragma unroll
            for (int q = 0; q < RP; ++q) {
              const float gq = Gw[q * RP + j];
              num = fmaf(w[q], negp(gq), num);
              den = fmaf(w[q], posp(gq), den);
            }
            s[j] = w[j] * sqrtf(num / den);
          }
#pragma unroll
          for (int j = 0; j < RP; ++j) w[j] = s[j];
        }
#pragma unroll
        for (int j = 0; j < RP; ++j) {
          if (j < r) a.W[i * r + j] = w[j];
          stA[t * RP + j] = w[j];
        }
        for (int k = 0; k < ell; ++k) stB[t * ell + k] = a.QL[i * ell + k];
      } else {
        for (int j = 0; j < RP; ++j) stA[t * RP + j] = 0.f;
        for (int k = 0; k < ell; ++k) stB[t * ell + k] = 0.f;
      }
      __syncthreads();
      const int cnt = static_cast<int>(r1 - ii < kPT ? r1 - ii : kPT);
      for (int e0 = 0; e0 < EW; e0 += kPT * 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * kPT + t;
          float v = 0.f;
          if (e < ell * r) {
            const int k = e / r, j = e - k * r;
            for (int q = 0; q < cnt; ++q) v = fmaf(stB[q * ell + k], stA[q * RP + j], v);
          } else if (e < EW) {
            const int j = e - ell * r;
            for (int q = 0; q < cnt; ++q) v = fmaf(stA[q * RP + j], stA[q * RP + j], v);
          }
          accw[u] = v;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * kPT + t;
          if (e < EW)
            atomicAdd(&a.accW[(ph * kCopies + blockIdx.x % kCopies) * EW + e],
                      static_cast<double>(accw[u]));
        }
      }
      __syncthreads();
    }
    if (!grid_sync(a.bar, G, a.status, a.abort_flag)) return;

    // ---------------- phase B: columns of H
    for (int64_t e = blockIdx.x * kPT + t; e < kCopies * EH; e += static_cast<int64_t>(G) * kPT)
      a.accH[pr * kCopies * EH + e] = 0.0;
    for (int j = t; j < RP; j += kPT) {
      double c2 = 0.0;
      if (j < r)
        for (int c = 0; c < kCopies; ++c) c2 += a.accW[(ph * kCopies + c) * EW + ell * r + j];
      const float c2f = static_cast<float>(c2);
      sc[j] = (normalize && j < r && c2f > 0.f) ? sqrtf(c2f) : 1.f;
    }
    __syncthreads();
    for (int e = t; e < ell * RP; e += kPT) {
      const int k = e / RP, j = e - k * RP;
      double v = 0.0;
      if (j < r)
        for (int c = 0; c < kCopies; ++c) v += a.accW[(ph * kCopies + c) * EW + k * r + j];
      WtS[e] = (j < r) ? static_cast<float>(v) / sc[j] : 0.f;
    }
    __syncthreads();
    for (int e = t; e < RP * RP; e += kPT) {
      const int p = e / RP, q = e - p * RP;
      float g = 0.f;
      if (p < r && q < r)
        for (int k = 0; k < ell; ++k) g = fmaf(WtS[k * RP + p], WtS[k * RP + q], g);
      Gh[e] = g;
    }
    __syncthreads();
    const bool plain = (a.alpha == 0.f && a.beta == 0.f);
    for (int64_t cc = c0; cc < c1; cc += kPT) {
      const int64_t c = cc + t;
      if (c < c1) {
        float h[RP], s[RP];
#pragma unroll
        for (int j = 0; j < RP; ++j) {
          h[j] = (j < r) ? a.H[j * a.n + c] * sc[j] : 0.f;
          s[j] = 0.f;
        }
        for (int k = 0; k < ell; ++k) {
          const float xk = a.Xhat[k * a.n + c];
#pragma unroll
          for (int j = 0; j < RP; ++j) s[j] = fmaf(xk, WtS[k * RP + j], s[j]);
        }
        if (RULE == 0) {
#pragma unroll
          for (int j = 0; j < RP; ++j) {
            if (j >= r) continue;
            const float g = Gh[j * RP + j];
            float tt = s[j];
#pragma unroll
            for (int q = 0; q < RP; ++q) tt = fmaf(-Gh[j * RP + q], h[q], tt);
            if (plain) {
              if (g > 0.f) h[j] = fmaxf(0.f, h[j] + tt / g);
            } else if (g + a.beta > 0.f) {
              h[j] = fmaxf(0.f, (fmaf(h[j], g, tt) - a.alpha) / (g + a.beta));
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < RP; ++j) {
            float num = posp(s[j]), den = negp(s[j]) + a.eps;
#pragma unroll
            for (int q = 0; q < RP; ++q) {
              const float gq = Gh[j * RP + q];
              num = fmaf(negp(gq), h[q], num);
              den = fmaf(posp(gq), h[q], den);
            }
            s[j] = h[j] * sqrtf(num / den);
          }
#pragma unroll
          for (int j = 0; j < RP; ++j) h[j] = s[j];
        }
#pragma unroll
        for (int j = 0; j < RP; ++j)
          if (j < r) a.H[j * a.n + c] = h[j];
      }
    }
    // H_tld of the new H (next iteration's phase A); this block's columns were just written
    // by this block's own threads
    __syncthreads();
    h_partial(ph, false);
    if (!grid_sync(a.bar, G, a.status, a.abort_flag)) return;
  }
  // final normalisation of W's rows by the last s_j
  if (normalize && a.iters > 0) {
    for (int64_t i = r0 + t; i < r1; i += kPT)
      for (int j = 0; j < r; ++j) a.W[i * r + j] /= sc[j];
  }
}

int rp_for(int r) {
  if (r <= 8) return 8;
  if (r <= 16) return 16;
  return 32;
}

template <int RP, int RULE>
cudaError_t launch(const Launcher& L, PArgs& a, int device_sms) {
  auto k = iterate_persistent_kernel<RP, RULE>;
  const size_t smem = sizeof(float) * (2 * a.ell * RP + 2 * RP * RP + RP + kPT * RP + kPT * a.ell);
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPT, smem)) != cudaSuccess)
    return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int grid = device_sms;   // one block per SM
  void* args[] = {&a};
  err = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k), dim3(grid), dim3(kPT), args, smem,
                                    L.stream);
  L.count();
  return err;
}

}  // namespace

size_t iterate_persistent_ws_bytes(int r, int ell) {
  return sizeof(double) * kCopies * (2 * (ell * r + r) + 2 * r * ell) + sizeof(Barrier) +
         2 * sizeof(int) + 1024;
}

bool iterate_persistent_supported(int r, int ell) { return r <= 32 && ell <= 128; }

cudaError_t launch_iterate_persistent(const Launcher& L, const IterArgs& ia, int iters, void* ws,
                                      size_t ws_bytes, int* status) {
  if (ws_bytes < iterate_persistent_ws_bytes(ia.r, ia.ell)) return cudaErrorInvalidValue;
  if (iters <= 0) return cudaSuccess;
  char* p = static_cast<char*>(ws);
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
  a.accW = reinterpret_cast<double*>(p);
  a.accH = a.accW + 2 * kCopies * (ia.ell * ia.r + ia.r);
  a.bar = reinterpret_cast<Barrier*>(a.accH + 2 * kCopies * ia.r * ia.ell);
  a.abort_flag = reinterpret_cast<int*>(a.bar + 1);
  a.status = status;
  const size_t clear = reinterpret_cast<char*>(a.abort_flag + 1) - p;
  cudaError_t err = cudaMemsetAsync(ws, 0, clear, L.stream);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int RP = rp_for(ia.r);
  const bool mu = ia.rule != 0;
  switch (RP) {
    case 8: return mu ? launch<8, 1>(L, a, sms) : launch<8, 0>(L, a, sms);
    case 16: return mu ? launch<16, 1>(L, a, sms) : launch<16, 0>(L, a, sms);
    default: return mu ? launch<32, 1>(L, a, sms) : launch<32, 0>(L, a, sms);
  }
}

}  // namespace nmfrp
