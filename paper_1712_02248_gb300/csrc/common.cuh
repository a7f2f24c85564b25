// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

namespace nmfrp {

// Device status codes (same values as nmf_status in include/nmf_rp.h).
enum : int {
  kStOk = 0,
  kStQrBreakdown = 4,
  kStNotFinite = 5,
  kStTimeout = 6,
};

// Running sum held as an unevaluated pair hi + lo of FP32 values, each addition by Knuth's
// TwoSum (about 48 significant bits). Long sums stay off the FP64 pipe, which on this GPU is so
// narrow that one FP64 add per 64 streamed elements halved the bandwidth of a streaming kernel.
struct FSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float s = __fadd_rn(hi, v);
    const float b = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, b)), __fsub_rn(v, b)));
    hi = s;
  }
  // += a * b with the product's rounding error kept (FMA)
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    lo = __fadd_rn(lo, __fmaf_rn(a, b, -p));
    add(p);
  }
  __device__ __forceinline__ double value() const {
    return static_cast<double>(hi) + static_cast<double>(lo);
  }
};

// Record the first failure only.
__device__ __forceinline__ void latch(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Launch bookkeeping: every kernel launch goes through a Launcher so that the library can report
// how many kernels it queued.
struct Launcher {
  cudaStream_t stream = nullptr;
  int64_t* counter = nullptr;
  void count(int k = 1) const {
    if (counter) *counter += k;
  }
};

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int pad_to(int v, int q) { return (v + q - 1) / q * q; }

// ---------------------------------------------------------------- launch functions
// Every function queues work on L.stream and returns the launch error (cudaSuccess if none).

// Philox4x32-10 + Box-Muller standard normals, rows x cols row-major.
cudaError_t launch_gaussian(const Launcher& L, int64_t rows, int64_t cols, uint64_t seed,
                            uint32_t stream_id, float* out);

// FP32 -> BF16 (RNE) copy of X (m x n, leading dimension ldx) into Xq (m x n, leading
// dimension ldq >= n; columns n..ldq-1 are set to zero).
cudaError_t launch_quantize_bf16(const Launcher& L, const float* X, int64_t m, int64_t n,
                                 int64_t ldx, __nv_bfloat16* Xq, int64_t ldq);

// The same copy plus ||X||^2 (into *x2_out) and <X - X_q, X> (into *corr_out), both FP64 on the
// device (either pointer may be null); ws holds quantize_stats_ws_bytes() of block partials.
size_t quantize_stats_ws_bytes();
cudaError_t launch_quantize_bf16_stats(const Launcher& L, const float* X, int64_t m, int64_t n,
                                       int64_t ldx, __nv_bfloat16* Xq, int64_t ldq, double* x2_out,
                                       double* corr_out, void* ws, size_t ws_bytes);

// Element type of X in the dual pass: FP32 (ldx any), BF16 (dense), or the FP8 copy made by
// launch_quantize_fp8_stats (ldx ignored: the copy's own row pitch and tile scales are used).
enum : int { kXFp32 = 0, kXBf16 = 1, kXFp8 = 2 };

// Bytes of the FP8 copy of an m x n matrix: E4M3 codes with row pitch ldq = n rounded up to 16
// (pad columns zero), then at byte scale_off (a multiple of 256) one E8M0 byte a 32 x 32 tile,
// ceil(m / 32) rows of ceil(n / 32).
size_t fp8_copy_bytes(int64_t m, int64_t n, int64_t* ldq = nullptr, int64_t* scale_off = nullptr);
// FP32 X -> the FP8 copy (codes and scales), plus ||X||^2 and <X - X_q, X> (either output may
// be null). ws: quantize_stats_ws_bytes() + 64 bytes.
cudaError_t launch_quantize_fp8_stats(const Launcher& L, const float* X, int64_t m, int64_t n,
                                      int64_t ldx, uint8_t* Xq, double* x2_out, double* corr_out,
                                      void* ws, size_t ws_bytes);

// Dual pass Y = X V (m x ell), Z = X^T U (n x ell). x_type selects the element type of X.
// ws: workspace for partial sums (size from dual_pass_ws_bytes).
// BF16 X with both products goes to the tensor-core kernel when TMA can address X (ldx a
// multiple of 8, X 16-byte aligned) unless force_simt is set; FP32 X likewise (ldx a multiple
// of 4, ell <= 80), FP8 X always when its copy is at least one 128 x 128 tile.
size_t dual_pass_ws_bytes(int64_t m, int64_t n, int ell);
// split: on the tensor-core path, V and U enter as hi + lo BF16 pairs (only X is rounded to
// BF16), which the compression uses; ignored elsewhere.
// z_kmajor: Z is written ell x n (the layout of X_hat) instead of n x ell; only the tensor-core
// path does this (dual_pass_uses_tc tells which path a pass takes).
cudaError_t launch_dual_pass(const Launcher& L, const void* X, int x_type, int64_t m, int64_t n,
                             int64_t ldx, int ell, const float* V, const float* U, float* Y,
                             float* Z, void* ws, size_t ws_bytes, int* status,
                             bool force_simt = false, bool split = false, bool z_kmajor = false);
bool dual_pass_uses_tc(const void* X, int x_type, int64_t m, int64_t n, int64_t ldx, int ell,
                       bool both, bool force_simt);
// tcgen05 + TMA dual pass on the FP8 copy (codes converted to BF16 in shared memory).
bool dual_pass_tc_fp8_supported(int64_t m, int64_t n, int ell, const void* Xq);
cudaError_t launch_dual_pass_tc_fp8(const Launcher& L, const uint8_t* Xq, int64_t m, int64_t n,
                                    int ell, const float* V, const float* U, float* Y, float* Z,
                                    void* ws, size_t ws_bytes, int* status, bool z_kmajor = false);
// tcgen05 + TMA dual pass on FP32 X (hi + lo BF16 split in shared memory, split V and U), for
// ell <= 80, ldx a multiple of 4 and X 16-byte aligned.
bool dual_pass_tc_f32_supported(int64_t m, int64_t n, int64_t ldx, int ell, const void* X);
cudaError_t launch_dual_pass_tc_f32(const Launcher& L, const float* X, int64_t m, int64_t n,
                                    int64_t ldx, int ell, const float* V, const float* U, float* Y,
                                    float* Z, void* ws, size_t ws_bytes, int* status,
                                    bool z_kmajor = false);
// tcgen05 + TMA dual pass (BF16 X).
bool dual_pass_tc_supported(int64_t m, int64_t n, int64_t ldx, int ell, const void* X);
size_t dual_pass_tc_ws_bytes(int64_t m, int64_t n, int ell);
cudaError_t launch_dual_pass_tc(const Launcher& L, const __nv_bfloat16* X, int64_t m, int64_t n,
                                int64_t ldx, int ell, const float* V, const float* U, float* Y,
                                float* Z, void* ws, size_t ws_bytes, int* status, bool split,
                                bool z_kmajor = false);

// Thin QR via CholeskyQR2 with FP64 Gram and Cholesky. Q may alias Y.
size_t qr_ws_bytes(int64_t rows, int ell);
cudaError_t launch_qr(const Launcher& L, const float* Y, int64_t rows, int ell, float* Q,
                      void* ws, size_t ws_bytes, int* status);
// Up to two independent QRs (same ell) through one set of launches; qr_ws_bytes(max rows, ell)
// of workspace suffices. bad_cols (4 words a matrix, may be null) receives the columns whose
// Cholesky pivot fell below the rank tolerance (those runs also latch kStQrBreakdown).
cudaError_t launch_qr_batch(const Launcher& L, int nmat, const float* const* Y,
                            const int64_t* rows, int ell, float* const* Q, void* ws,
                            size_t ws_bytes, int* status, uint32_t* bad_cols = nullptr);
// Y (rows x ell) column j <- N(0, 1) draws (Philox4x32-10, key = seed, counter stream stream_id)
// for every bit j set in mask[0..3].
cudaError_t launch_replace_columns(const Launcher& L, float* Y, int64_t rows, int ell,
                                   const uint32_t* mask, uint64_t seed, uint32_t stream_id);

// Iterations of FastHALS-RP (rule 0) or MU-RP (rule 1).
struct IterArgs {
  int64_t m, n;
  int r, ell;
  int rule;
  float alpha, beta, eps;
  const float* QL;    // m x ell
  const float* QR;    // n x ell
  const float* Xhat;  // ell x n
  const float* Xchk;  // m x ell
  float* W;           // m x r
  float* H;           // r x n
  long long wait_cycles = 0;   // persistent kernel: polling budget of a grid barrier (0: default)
};
size_t iterate_ws_bytes(int64_t m, int64_t n, int r, int ell);
cudaError_t launch_iterate(const Launcher& L, const IterArgs& a, int iters, void* ws,
                           size_t ws_bytes);

// All iterations in one cooperative launch (r <= 48); status receives NMF_ERR_TIMEOUT if a
// grid barrier wait runs out.
bool iterate_persistent_supported(int64_t m, int64_t n, int r, int ell);
size_t iterate_persistent_ws_bytes(int r, int ell);
// mon (2 floats) receives the error monitor's cross and quadratic terms of the last iteration;
// if *done is non-zero on entry the launch does nothing.
cudaError_t launch_iterate_persistent(const Launcher& L, const IterArgs& a, int iters, void* ws,
                                      size_t ws_bytes, int* status, float* mon, const int* done);
// The solve's loop in the persistent kernel: iterations continue from solve[6] (a count, kept
// as a double) and stop at the first check point (every `every` iterations, and the last of
// `total`) where the error monitor, compared with `target` as the solve's gate does (margin
// before the first exact check, margin_cal once solve[5] holds a calibration), calls for an
// exact residual; the launch then leaves the count in solve[6], the estimate in solve[4] and
// flags[1] = 1. flags[0] set on entry (converged) or no iterations left: flags[1] = 0, no work.
struct SolveGate {
  int total = 0, every = 0;
  int* flags = nullptr;      // [0] converged, [1] exact check due
  double* solve = nullptr;   // [0] ||X||^2, [3] BF16 rounding term, [4], [5], [6] as above
  double target = 0.0, margin = 0.0, margin_cal = 0.0;
};
cudaError_t launch_iterate_persistent_gated(const Launcher& L, const IterArgs& a,
                                            const SolveGate& g, void* ws, size_t ws_bytes,
                                            int* status, float* mon);

// Several independent problems in cooperative launches ("waves" packed into the SMs, one class
// of padded rank and rule per launch); problem i runs iters[i] iterations on blocks[i] blocks
// (at least iterate_multi_min_blocks, at most the number of SMs). mon: 2 floats per problem.
int iterate_multi_min_blocks(int64_t m, int64_t n, int r, int ell);
size_t iterate_multi_ws_bytes(const IterArgs* ia, int nprob);
cudaError_t launch_iterate_multi(const Launcher& L, const IterArgs* ia, const int* iters,
                                 const int* blocks, int nprob, void* ws, size_t ws_bytes,
                                 int* status, float* mon, const int* done_zero);

// Sparse X (CSR: row pointers int64 m + 1, column indices int32 distinct within a row, FP32
// values) and its transpose in CSC form (built once per matrix by launch_csc_build into `csc`,
// csc_bytes(n, nnz) of device memory; ws: csc_ws_bytes).
struct CsrView {
  const int64_t* ptr;
  const int* idx;
  const float* val;
};
struct CscView {
  int64_t* ptr;
  int* idx;
  float* val;
};
size_t csc_bytes(int64_t n, int64_t nnz);
size_t csc_ws_bytes(int64_t m, int64_t n, int64_t nnz);
cudaError_t launch_csc_build(const Launcher& L, const int64_t* ptr, const int* idx,
                             const float* val, int64_t m, int64_t n, int64_t nnz, void* csc,
                             void* ws, size_t ws_bytes, CscView* out);
// Y = X V (m x ell) through the CSR form, Z = X^T U (n x ell) through the CSC form; either pair
// may be null.
cudaError_t launch_csr_dual(const Launcher& L, const CsrView& X, const CscView& XT, int64_t m,
                            int64_t n, int ell, const float* V, const float* U, float* Y, float* Z);
// out2[0] = ||X - W H||^2, out2[1] = ||X||^2 (device doubles) for sparse X.
size_t sparse_residual_ws_bytes(int64_t m, int64_t n, int r);
cudaError_t launch_sparse_residual(const Launcher& L, const CsrView& X, int64_t m, int64_t n,
                                   const float* W, const float* H, int r, double* out2, void* ws,
                                   size_t ws_bytes);

// Singular values of X_hat (ell x n, ell <= 128), descending, into sigma (ell floats, device).
size_t spectrum_ws_bytes(int64_t n, int ell);
cudaError_t launch_spectrum(const Launcher& L, int64_t n, int ell, const float* Xhat, void* ws,
                            size_t ws_bytes, float* sigma);

// Iterations on the full data X (FastHALS, rule 0; Lee-Seung MU, rule 1), r <= 64: two passes
// over X an iteration (X H^T, then X^T W with the new W). x_type and ldx as for the dual pass.
size_t iterate_full_ws_bytes(int64_t m, int64_t n, int r);
cudaError_t launch_iterate_full(const Launcher& L, const void* X, int x_type, int64_t m, int64_t n,
                                int64_t ldx, int r, int rule, float alpha, float beta, float eps,
                                float* W, float* H, int iters, void* ws, size_t ws_bytes,
                                int* status, bool force_simt);

// Gini coefficient sums of `count` floats (Section 5.1): out2[0] = sum (2 i - N - 1) b_(i),
// out2[1] = sum b_(i) over the ascending order (device, FP64). ws: gini_ws_bytes(count).
size_t gini_ws_bytes(int64_t count);
cudaError_t launch_gini(const Launcher& L, const float* B, int64_t count, void* ws,
                        size_t ws_bytes, double* out2);

// Residual partial sums: writes 2 doubles (||X-WH||^2, ||X||^2) to out2 (device). If gate is
// non-null and *gate == 0 the kernels return without work.
// With residual_ws_bytes_tc(m, n) of workspace, FP32 X with rows 16-byte aligned and r <= 32,
// the W H rebuild runs on the tensor cores (BF16 hi + lo splits of W and H); status receives
// NMF_ERR_TIMEOUT if one of that kernel's waits runs out.
size_t residual_ws_bytes(int64_t m, int64_t n);
size_t residual_ws_bytes_tc(int64_t m, int64_t n);
cudaError_t launch_residual(const Launcher& L, const float* X, int64_t m, int64_t n, int64_t ldx,
                            const float* W, const float* H, int r, double* out2, void* ws,
                            size_t ws_bytes, const int* gate = nullptr, int* status = nullptr);
bool residual_tc_supported(int64_t m, int64_t n, int64_t ldx, const float* X, int r);
size_t residual_tc_operand_bytes(int64_t m, int64_t n);
cudaError_t launch_residual_tc(const Launcher& L, const float* X, int64_t m, int64_t n,
                               int64_t ldx, const float* W, const float* H, int r, double* part,
                               int max_grid, int* grid_out, void* ws, size_t ws_bytes, int* status,
                               const int* gate);
// Static scratch for launch_residual: the device address (resolved once per device, which must be
// current) of a fixed array of residual_static_capacity_bytes() bytes in global memory.
size_t residual_static_capacity_bytes();
cudaError_t residual_static_scratch(int device, void** addr);
// ||X||^2 into *out (device, FP64).
cudaError_t launch_sumsq(const Launcher& L, const float* X, int64_t m, int64_t n, int64_t ldx,
                         double* out, void* ws, size_t ws_bytes);

// NNDSVD from compressed data.
size_t nndsvd_ws_bytes(int64_t m, int64_t n, int r, int ell);
cudaError_t launch_nndsvd(const Launcher& L, int64_t m, int64_t n, int r, int ell,
                          const float* QL, const float* Xhat, float* W, float* H, void* ws,
                          size_t ws_bytes, int* status);

// Learned warm start: NNDSVD-based W_b (m x r), H_b (r x n), hscale (r) and row features F_w
// (m x 3r), F_h (n x 3r); nndsvd_ws_bytes of workspace.
cudaError_t launch_warmstart_features(const Launcher& L, int64_t m, int64_t n, int r, int ell,
                                      const float* QL, const float* Xhat, float* Wb, float* Hb,
                                      float* hscale, float* Fw, float* Fh, void* ws,
                                      size_t ws_bytes);
int64_t mlp_param_count(int F, int Hd, int r);
size_t mlp_ws_bytes(int64_t rows, int Hd, int r);
cudaError_t launch_mlp_forward(const Launcher& L, int F, int Hd, int r, const float* params,
                               const float* X, int64_t rows, float* Y, void* ws, size_t ws_bytes);
cudaError_t launch_mlp_loss_grad(const Launcher& L, int F, int Hd, int r, const float* params,
                                 const float* X, const float* T, int64_t rows, float* grad,
                                 double* loss, void* ws, size_t ws_bytes);
cudaError_t launch_adam(const Launcher& L, float* p, float* m, float* v, const float* g,
                        int64_t count, float lr, int step);
cudaError_t launch_warmstart_apply(const Launcher& L, int64_t m, int64_t n, int r,
                                   const float* Wb, const float* Dw, const float* Hb,
                                   const float* Dh, const float* hscale, float* W, float* H);
cudaError_t launch_warmstart_targets(const Launcher& L, int64_t m, int64_t n, int r,
                                     const float* Wb, const float* Hb, const float* hscale,
                                     const float* Wstar, const float* Hstar, float* Tw,
                                     float* Th);

}  // namespace nmfrp
