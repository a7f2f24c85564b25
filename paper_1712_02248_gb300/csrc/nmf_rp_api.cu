// C ABI of the library (include/nmf_rp.h): argument checks, workspace, and the order of the
// kernels of each step. No arithmetic of the method happens here.
#include <cstdio>
#include <cstring>
#include <cstdarg>
#include <algorithm>
#include <cmath>

#include <utility>
#include <vector>

#include "nmf_rp.h"
#include "common.cuh"

// Optional per-phase timing: CUDA events recorded on the context stream around each phase.
struct PhaseMark {
  int phase;
  cudaEvent_t a, b;
};

struct nmf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* d_status = nullptr;   // latched device status word
  uint32_t* d_qrbad = nullptr;   // [8] columns the sketch QRs found dependent (2 matrices x 128 bits)
  float* d_wh0 = nullptr;        // initial W, H kept for a rerun of nmf_solve
  size_t wh0_cap = 0;
  double* d_res = nullptr;   // residual sums (2 doubles)
  double* h_res = nullptr;   // pinned host copy
  // solve-loop state on the device (one allocation)
  float* d_mon = nullptr;    // [2] monitor terms of the last iteration run
  int* d_flags = nullptr;    // [0] done, [1] gate, [2] always zero, [3] exact checks run
  double* d_solve = nullptr; // [0] ||X||^2, [1] last exact rel_err, [2] iterations at that check,
                             // [3] <X - X_q, X>, [4] monitor estimate at the last exact check,
                             // [5] exact / estimate there (0 before the first exact check)
  int* h_done = nullptr;     // pinned [2] copies of the done flag
  int last_iters = 0, last_checks = 0;
  int64_t wait_cycles = 0;   // grid-barrier polling budget of the persistent kernel (0: default)
  int64_t launches = 0;
  char msg[512] = {0};
  bool profiling = false;
  std::vector<PhaseMark> marks;
  std::vector<cudaEvent_t> pool;
  double phase_ms[NMF_PHASE_COUNT] = {0};
  int64_t phase_n[NMF_PHASE_COUNT] = {0};
  // batched solves: side streams (fork / join through events) and their sizes
  static constexpr int kSide = 8;
  cudaStream_t side[kSide] = {};
  cudaEvent_t side_ev[kSide] = {};
  cudaEvent_t fork_ev = nullptr;
  double* d_bres = nullptr;   // 2 doubles per problem
  double* h_bres = nullptr;
  int bres_cap = 0;
  int last_batch_rows_per_block = 0;
  // autotuned rows per block of the batched iterations, keyed by a hash of the batch's shapes
  std::vector<std::pair<uint64_t, int>> tuned;
  // the batched solve's first phase as a CUDA graph, replayed while its inputs stay the same
  cudaGraphExec_t batch_graph = nullptr;
  uint64_t batch_key = 0;
  int64_t batch_graph_launches = 0;
  // learned warm start (NMF_INIT_MLP): the two networks' parameters on the device
  float* warm = nullptr;      // [W net | H net]
  int warm_hidden = 0, warm_r = 0;
  double* d_loss = nullptr;
};

namespace {

using nmfrp::cdiv;

cudaEvent_t pool_event(nmf_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Scoped phase timer (no-op unless profiling is on).
struct Phase {
  nmf_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  Phase(nmf_ctx* ctx, int ph) : c(ctx), phase(ph) {
    if (c->profiling && (a = pool_event(c))) cudaEventRecord(a, c->stream);
  }
  void end() {
    if (!a) return;
    cudaEvent_t b = pool_event(c);
    if (!b) {
      c->pool.push_back(a);
    } else {
      cudaEventRecord(b, c->stream);
      c->marks.push_back({phase, a, b});
    }
    a = nullptr;
  }
  ~Phase() { end(); }
};

// Fold recorded marks into the per-phase totals (synchronises).
void resolve_marks(nmf_ctx* c) {
  if (c->marks.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (const PhaseMark& mk : c->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, mk.a, mk.b) == cudaSuccess) {
      c->phase_ms[mk.phase] += ms;
      c->phase_n[mk.phase] += 1;
    } else {
      cudaGetLastError();
    }
    c->pool.push_back(mk.a);
    c->pool.push_back(mk.b);
  }
  c->marks.clear();
}

nmf_status fail(nmf_ctx* c, nmf_status st, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
    va_end(ap);
  }
  return st;
}

nmf_status cuda_fail(nmf_ctx* c, cudaError_t e, const char* where) {
  return fail(c, NMF_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define NMF_CUDA(call, where)                       \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

nmfrp::Launcher launcher(nmf_ctx* c) {
  nmfrp::Launcher L;
  L.stream = c->stream;
  L.counter = &c->launches;
  return L;
}

// Grow the context workspace to at least `bytes` (synchronises before freeing the old one).
nmf_status ensure_ws(nmf_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return NMF_OK;
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  const size_t want = bytes + (bytes >> 3) + (1 << 20);
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, NMF_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
  }
  ctx->ws_bytes = want;
  return NMF_OK;
}

// Bump allocator over the workspace (256-byte aligned slices).
struct Arena {
  char* base;
  size_t cap, off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~static_cast<size_t>(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * count;
    return p;
  }
  void* rest(size_t* bytes) {
    off = (off + 255) & ~static_cast<size_t>(255);
    *bytes = cap > off ? cap - off : 0;
    return base + off;
  }
};

nmf_status check_params(nmf_ctx* ctx, const nmf_params* p) {
  if (!p) return fail(ctx, NMF_ERR_INVALID_ARG, "params is NULL");
  if (p->m < 1 || p->n < 1) return fail(ctx, NMF_ERR_INVALID_ARG, "m, n must be >= 1");
  if (p->r < 1 || p->r > p->ell)
    return fail(ctx, NMF_ERR_INVALID_ARG, "need 1 <= r <= ell (r=%d ell=%d)", p->r, p->ell);
  if (p->ell > 128) return fail(ctx, NMF_ERR_INVALID_ARG, "ell must be <= 128");
  if (p->ell > std::min(p->m, p->n))
    return fail(ctx, NMF_ERR_INVALID_ARG, "ell must be <= min(m, n)");
  if (p->power_iters < 0 || p->power_iters > 32)
    return fail(ctx, NMF_ERR_INVALID_ARG, "power_iters must be in [0, 32]");
  if (p->rule != NMF_RULE_FASTHALS_RP && p->rule != NMF_RULE_MU_RP)
    return fail(ctx, NMF_ERR_INVALID_ARG, "unknown rule %d", p->rule);
  if (p->prec != NMF_PREC_FP32 && p->prec != NMF_PREC_BF16 && p->prec != NMF_PREC_FP8_E4M3)
    return fail(ctx, NMF_ERR_INVALID_ARG, "precision %d not available", p->prec);
  if (p->alpha < 0 || p->beta < 0) return fail(ctx, NMF_ERR_INVALID_ARG, "alpha, beta must be >= 0");
  return NMF_OK;
}

nmf_status check_x(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx) {
  if (!X) return fail(ctx, NMF_ERR_INVALID_ARG, "X is NULL");
  if (p->prec == NMF_PREC_BF16 && ldx != p->n)
    return fail(ctx, NMF_ERR_INVALID_ARG, "BF16 X must be dense (ldx == n)");
  if (p->prec == NMF_PREC_FP8_E4M3 && ldx != p->n)
    return fail(ctx, NMF_ERR_INVALID_ARG, "FP8 X is the nmf_quantize layout (pass ldx == n)");
  if (ldx < p->n) return fail(ctx, NMF_ERR_INVALID_ARG, "ldx < n");
  return NMF_OK;
}

float eps_of(const nmf_params* p) { return p->eps > 0 ? static_cast<float>(p->eps) : 1e-12f; }

// One dual pass with its scratch; prec (nmf_precision) names the element type of X.
int x_type_of(int prec) {
  return prec == NMF_PREC_BF16 ? nmfrp::kXBf16 : prec == NMF_PREC_FP8_E4M3 ? nmfrp::kXFp8
                                                                           : nmfrp::kXFp32;
}

nmf_status dual(nmf_ctx* ctx, const void* X, int prec, int64_t m, int64_t n, int64_t ldx, int ell,
                const float* V, const float* U, float* Y, float* Z, Arena a, bool simt = false,
                bool split = false, bool z_kmajor = false) {
  Phase ph(ctx, NMF_PHASE_DUAL_PASS);
  size_t rest = 0;
  void* ws = a.rest(&rest);
  NMF_CUDA(nmfrp::launch_dual_pass(launcher(ctx), X, x_type_of(prec), m, n, ldx, ell, V, U, Y, Z,
                                   ws, rest, ctx->d_status, simt, split, z_kmajor),
           "dual pass");
  return NMF_OK;
}

// QR of the m-side and the n-side output of one pass together (both chains of the sketch).
nmf_status qr2(nmf_ctx* ctx, float* Ym, int64_t m, float* Yn, int64_t n, int ell, Arena a) {
  Phase ph(ctx, NMF_PHASE_QR);
  size_t rest = 0;
  void* ws = a.rest(&rest);
  const float* ys[2] = {Ym, Yn};
  float* qs[2] = {Ym, Yn};
  const int64_t rows[2] = {m, n};
  NMF_CUDA(nmfrp::launch_qr_batch(launcher(ctx), 2, ys, rows, ell, qs, ws, rest, ctx->d_status),
           "qr");
  return NMF_OK;
}

// qr2 that repairs a numerically rank-deficient pass output: Y is kept; when a Cholesky pivot
// falls below the rank tolerance, the columns it names are replaced by Gaussian draws (a column
// that depends on the ones before it adds nothing to range(Y), so the span keeps range(Y) and
// gains a random direction) and CholeskyQR2 runs again. Every update of the method depends on Q
// only through Q Q^T X, which is X on range(Y) either way. Synchronises after each attempt.
nmf_status qr2_robust(nmf_ctx* ctx, float* Ym, int64_t m, float* Yn, int64_t n, int ell,
                      uint64_t seed, Arena a) {
  Phase ph(ctx, NMF_PHASE_QR);
  float* keep_m = a.take<float>(m * ell);
  float* keep_n = a.take<float>(n * ell);
  NMF_CUDA(cudaMemcpyAsync(keep_m, Ym, sizeof(float) * m * ell, cudaMemcpyDeviceToDevice,
                           ctx->stream), "qr copy");
  NMF_CUDA(cudaMemcpyAsync(keep_n, Yn, sizeof(float) * n * ell, cudaMemcpyDeviceToDevice,
                           ctx->stream), "qr copy");
  size_t rest = 0;
  void* ws = a.rest(&rest);
  const float* ys[2] = {Ym, Yn};
  float* qs[2] = {Ym, Yn};
  const int64_t rows[2] = {m, n};
  for (int attempt = 0; attempt < 4; ++attempt) {
    uint32_t bad[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int st = 0;
    NMF_CUDA(cudaMemsetAsync(ctx->d_qrbad, 0, sizeof(bad), ctx->stream), "qr mask");
    NMF_CUDA(nmfrp::launch_qr_batch(launcher(ctx), 2, ys, rows, ell, qs, ws, rest, ctx->d_status,
                                    ctx->d_qrbad),
             "qr");
    NMF_CUDA(cudaMemcpyAsync(bad, ctx->d_qrbad, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream),
             "qr mask");
    NMF_CUDA(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
             "qr status");
    NMF_CUDA(cudaStreamSynchronize(ctx->stream), "qr sync");
    if (st != NMF_ERR_QR_BREAKDOWN) return NMF_OK;   // other statuses stay latched
    NMF_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream), "status reset");
    // restore Y, replace the named columns, keep the repaired copy for the next attempt
    float* Ys[2] = {Ym, Yn};
    float* keeps[2] = {keep_m, keep_n};
    for (int k = 0; k < 2; ++k) {
      NMF_CUDA(cudaMemcpyAsync(Ys[k], keeps[k], sizeof(float) * rows[k] * ell,
                               cudaMemcpyDeviceToDevice, ctx->stream), "qr restore");
      if (bad[4 * k] | bad[4 * k + 1] | bad[4 * k + 2] | bad[4 * k + 3]) {
        NMF_CUDA(nmfrp::launch_replace_columns(launcher(ctx), Ys[k], rows[k], ell, bad + 4 * k,
                                               seed, 0x52430000u + 2u * attempt + k),
                 "qr repair");
        NMF_CUDA(cudaMemcpyAsync(keeps[k], Ys[k], sizeof(float) * rows[k] * ell,
                                 cudaMemcpyDeviceToDevice, ctx->stream), "qr copy");
      }
    }
  }
  return fail(ctx, NMF_ERR_QR_BREAKDOWN, "sketch QR still rank deficient after column repair");
}

size_t pass_scratch(int64_t m, int64_t n, int ell) {
  return std::max(nmfrp::dual_pass_ws_bytes(m, n, ell),
                  std::max(nmfrp::qr_ws_bytes(m, ell), nmfrp::qr_ws_bytes(n, ell))) + 4096;
}

size_t sketch_ws(const nmf_params* p, bool need_omega) {
  const int64_t m = p->m, n = p->n, l = p->ell;
  size_t b = sizeof(float) * (m * l + n * l) + 1024;         // other chain's m- and n-side bases
  if (need_omega) b += sizeof(float) * (m * l + n * l) + 1024;
  b += sizeof(float) * (m * l + n * l) + 1024;               // pass outputs kept by qr2_robust
  return b + pass_scratch(m, n, p->ell);
}

// Both chains of Eq. 3.5 advance together: pass 0 applies X to Omega_L and X^T to Omega_R; pass
// p >= 1 applies X to one chain's n-side basis and X^T to the other chain's m-side basis.
// `pass(V, U, Y, Z)` runs one fused pass Y = X V, Z = X^T U over whatever form X has.
template <typename Pass>
nmf_status sketch_core(nmf_ctx* ctx, const nmf_params* p, Pass pass, const float* omega_L,
                       const float* omega_R, float* QL, float* QR, Arena& a, bool robust) {
  const int64_t m = p->m, n = p->n;
  const int l = p->ell;
  float* mR = a.take<float>(m * l);   // right chain, m-side
  float* nL = a.take<float>(n * l);   // left chain, n-side
  if (!omega_L || !omega_R) {
    float* oL = a.take<float>(n * l);
    float* oR = a.take<float>(m * l);
    if (!omega_L) {
      NMF_CUDA(nmfrp::launch_gaussian(launcher(ctx), n, l, p->seed, 0u, oL), "gaussian");
      omega_L = oL;
    }
    if (!omega_R) {
      NMF_CUDA(nmfrp::launch_gaussian(launcher(ctx), m, l, p->seed, 1u, oR), "gaussian");
      omega_R = oR;
    }
  }
  nmf_status st;
  auto orth = [&](float* Ym, float* Yn, int k) {
    return robust ? qr2_robust(ctx, Ym, m, Yn, n, l, p->seed + 0x9E37u * (k + 1), a)
                  : qr2(ctx, Ym, m, Yn, n, l, a);
  };
  // pass 0
  if ((st = pass(omega_L, omega_R, QL, QR)) != NMF_OK) return st;
  if ((st = orth(QL, QR, 0)) != NMF_OK) return st;
  for (int k = 1; k <= 2 * p->power_iters; ++k) {
    if (k & 1) {
      // right chain: X * (n-side) -> m-side; left chain: X^T * (m-side) -> n-side
      if ((st = pass(QR, QL, mR, nL)) != NMF_OK) return st;
      if ((st = orth(mR, nL, k)) != NMF_OK) return st;
    } else {
      if ((st = pass(nL, mR, QL, QR)) != NMF_OK) return st;
      if ((st = orth(QL, QR, k)) != NMF_OK) return st;
    }
  }
  return NMF_OK;
}

nmf_status sketch_impl(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                       const float* omega_L, const float* omega_R, float* QL, float* QR, Arena a,
                       bool robust = false) {
  const bool simt = (p->flags & NMF_FLAG_SIMT_DUAL_PASS) != 0;
  auto pass = [&](const float* V, const float* U, float* Y, float* Z) {
    return dual(ctx, X, p->prec, p->m, p->n, ldx, p->ell, V, U, Y, Z, a, simt);
  };
  return sketch_core(ctx, p, pass, omega_L, omega_R, QL, QR, a, robust);
}

__global__ void transpose_kernel(const float* __restrict__ in, int64_t rows, int cols,
                                 float* __restrict__ out) {
  // out (cols x rows) = in^T (in: rows x cols)
  __shared__ float tile[32][33];
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i;
    const int c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    const int64_t r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[static_cast<int64_t>(c) * rows + r] = tile[threadIdx.x][i];
  }
}

nmf_status compress_impl(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                         const float* QL, const float* QR, float* Xhat, float* Xchk, Arena a) {
  const int64_t m = p->m, n = p->n;
  const int l = p->ell;
  const bool simt = (p->flags & NMF_FLAG_SIMT_DUAL_PASS) != 0;
  // the compressed data feed every iteration and the error monitor: Q_L, Q_R enter the BF16
  // tensor-core pass as hi + lo pairs so that only X itself is rounded. The tensor-core pass
  // writes X_hat = Q_L^T X directly in its l x n layout; the SIMT pass writes its transpose
  if (nmfrp::dual_pass_uses_tc(X, x_type_of(p->prec), m, n, ldx, l, true, simt))
    return dual(ctx, X, p->prec, m, n, ldx, l, QR, QL, Xchk, Xhat, a, simt, true, true);
  float* XhatT = a.take<float>(n * l);
  nmf_status st = dual(ctx, X, p->prec, m, n, ldx, l, QR, QL, Xchk, XhatT, a, simt, true);
  if (st != NMF_OK) return st;
  dim3 grid(static_cast<unsigned>(cdiv(n, 32)), static_cast<unsigned>(cdiv(l, 32)));
  transpose_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(XhatT, n, l, Xhat);
  ctx->launches++;
  NMF_CUDA(cudaGetLastError(), "transpose");
  return NMF_OK;
}

nmfrp::IterArgs iter_args(const nmf_ctx* ctx, const nmf_params* p, const float* QL,
                          const float* QR, const float* Xhat, const float* Xchk, float* W,
                          float* H) {
  nmfrp::IterArgs ia;
  ia.m = p->m;
  ia.n = p->n;
  ia.r = p->r;
  ia.ell = p->ell;
  ia.rule = p->rule;
  ia.alpha = static_cast<float>(p->alpha);
  ia.beta = static_cast<float>(p->beta);
  ia.eps = eps_of(p);
  ia.QL = QL;
  ia.QR = QR;
  ia.Xhat = Xhat;
  ia.Xchk = Xchk;
  ia.W = W;
  ia.H = H;
  ia.wait_cycles = ctx->wait_cycles;
  return ia;
}

nmf_status iterate_impl(nmf_ctx* ctx, const nmf_params* p, const float* QL, const float* QR,
                        const float* Xhat, const float* Xchk, float* W, float* H, int iters,
                        Arena a, const int* done = nullptr) {
  if (p->r > 64) return fail(ctx, NMF_ERR_UNSUPPORTED, "iterations support r <= 64");
  const nmfrp::IterArgs ia = iter_args(ctx, p, QL, QR, Xhat, Xchk, W, H);
  Phase ph(ctx, NMF_PHASE_ITERATE);
  size_t rest = 0;
  void* ws = a.rest(&rest);
  if (!(p->flags & NMF_FLAG_STAGED_ITERATE) && nmfrp::iterate_persistent_supported(p->m, p->n, p->r, p->ell)) {
    NMF_CUDA(nmfrp::launch_iterate_persistent(launcher(ctx), ia, iters, ws, rest, ctx->d_status,
                                              ctx->d_mon, done ? done : ctx->d_flags + 2),
             "iterate (persistent)");
  } else {
    NMF_CUDA(nmfrp::launch_iterate(launcher(ctx), ia, iters, ws, rest), "iterate");
  }
  return NMF_OK;
}

nmf_status take_status(nmf_ctx* ctx);

nmf_status residual_impl(nmf_ctx* ctx, const nmf_params* p, const float* X, int64_t ldx,
                         const float* W, const float* H, double* rel, double* e2o, double* x2o,
                         Arena a) {
  size_t rest = 0;
  void* ws = a.rest(&rest);
  // the FP32 rebuild unless the caller asks for the tensor-core one (the kernel is chosen by the
  // workspace it is given)
  if (!(p->flags & NMF_FLAG_TC_RESIDUAL)) rest = std::min(rest, nmfrp::residual_ws_bytes(p->m, p->n));
  Phase ph(ctx, NMF_PHASE_RESIDUAL);
  NMF_CUDA(nmfrp::launch_residual(launcher(ctx), X, p->m, p->n, ldx, W, H, p->r, ctx->d_res, ws,
                                  rest, nullptr, ctx->d_status),
           "residual");
  ph.end();
  NMF_CUDA(cudaMemcpyAsync(ctx->h_res, ctx->d_res, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "residual copy");
  NMF_CUDA(cudaStreamSynchronize(ctx->stream), "residual sync");
  nmf_status st = take_status(ctx);   // a wait of the tensor-core kernel that ran out
  if (st != NMF_OK) return st;
  const double e2 = ctx->h_res[0], x2 = ctx->h_res[1];
  if (e2o) *e2o = e2;
  if (x2o) *x2o = x2;
  if (!(e2 == e2) || !(x2 == x2) || e2 > 1e308 || x2 > 1e308)
    return fail(ctx, NMF_ERR_NOT_FINITE, "residual is not finite");
  if (rel) *rel = x2 > 0 ? std::sqrt(e2 / x2) : std::sqrt(e2);
  return NMF_OK;
}

nmf_status take_status(nmf_ctx* ctx) {
  int st = 0;
  NMF_CUDA(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
           "status copy");
  NMF_CUDA(cudaStreamSynchronize(ctx->stream), "status sync");
  if (st != 0) {
    NMF_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream), "status reset");
    NMF_CUDA(cudaStreamSynchronize(ctx->stream), "status sync");
    switch (st) {
      case NMF_ERR_QR_BREAKDOWN:
        return fail(ctx, NMF_ERR_QR_BREAKDOWN, "Cholesky pivot not positive in the sketch QR");
      case NMF_ERR_TIMEOUT: return fail(ctx, NMF_ERR_TIMEOUT, "device wait ran out");
      default: return fail(ctx, static_cast<nmf_status>(st), "device status %d", st);
    }
  }
  return NMF_OK;
}

// Decide whether the exact residual of this check must run: always for the last check, else
// when the error monitor (||X||^2 - 2 cross + quad, X replaced by its projection, plus the
// rounding term of a BF16 copy) is within `margin` of the target. After the first exact check
// the estimate is scaled by the ratio exact / estimate measured there (the monitor's bias drifts
// slowly: on the dense 20000 x 5000 workloads the ratio moved by less than 1e-5 over 100
// iterations), and the margin shrinks to `margin_cal`. The gate only saves work: the solve
// stops on the exact residual alone.
__global__ void solve_gate_kernel(const float* mon, double* solve, double target, double margin,
                                  double margin_cal, int force, int* flags) {
  if (flags[0]) {
    flags[1] = 0;
    return;
  }
  // solve[3] = <X - X_q, X> when the compressed data come from a BF16 copy X_q (else 0):
  // <X, W H> ~ <X_hat, W_tld H> + <X - X_q, X>
  const double x2 = solve[0];
  const double e2 = x2 - 2.0 * (static_cast<double>(mon[0]) + solve[3]) + static_cast<double>(mon[1]);
  const double est = x2 > 0.0 ? sqrt(fmax(e2, 0.0) / x2) : 0.0;
  int check = 1;
  if (!force && target > 0.0) {
    const double cal = solve[5];
    check = cal > 0.0 ? (est * cal <= target * (1.0 + margin_cal))
                      : (est <= target * (1.0 + margin));
  }
  flags[1] = check;
  if (check) solve[4] = est;
}

// After a gated exact residual: record it, calibrate the monitor against it, and raise `done`
// when the target is reached.
__global__ void solve_decide_kernel(const double* res2, double target, int iters_done,
                                    double* solve, int* flags) {
  if (flags[0] || !flags[1]) return;
  const double e2 = res2[0], x2 = solve[0];
  const double rel = x2 > 0.0 ? sqrt(e2 / x2) : sqrt(e2);
  solve[1] = rel;
  solve[2] = iters_done;
  if (solve[4] > 0.0) solve[5] = rel / solve[4];
  flags[3] += 1;
  if (target > 0.0 && rel <= target) flags[0] = 1;
}

// The same after a check that the persistent kernel's own gate asked for (it stops there): the
// iteration count is the one it left in solve[6], `done` is also raised once the budget `total`
// is spent, and the gate flag is cleared.
__global__ void solve_decide_gated_kernel(const double* res2, double target, int total,
                                          double* solve, int* flags) {
  if (flags[0] || !flags[1]) return;
  const double e2 = res2[0], x2 = solve[0];
  const double rel = x2 > 0.0 ? sqrt(e2 / x2) : sqrt(e2);
  solve[1] = rel;
  solve[2] = solve[6];
  if (solve[4] > 0.0) solve[5] = rel / solve[4];
  flags[3] += 1;
  flags[1] = 0;
  if ((target > 0.0 && rel <= target) || solve[6] >= static_cast<double>(total)) flags[0] = 1;
}

// Workspace of the learned warm start for hidden width <= hidden_max: W_b, H_b, hscale, F_w, F_h,
// the two network outputs and the forward pass activations.
size_t warm_ws_bytes(const nmf_params* p, int hidden_max) {
  const int64_t m = p->m, n = p->n, r = p->r;
  return sizeof(float) * static_cast<size_t>((m + n) * r * 5 + r) + 8 * 256 +
         std::max(nmfrp::nndsvd_ws_bytes(m, n, p->r, p->ell),
                  nmfrp::mlp_ws_bytes(std::max(m, n), hidden_max, p->r));
}

// NNDSVD features, both networks, and the initial factors into W, H.
nmf_status warm_init(nmf_ctx* ctx, const nmf_params* p, const float* QL, const float* Xhat,
                     float* W, float* H, Arena a) {
  if (!ctx->warm || ctx->warm_r != p->r)
    return fail(ctx, NMF_ERR_INVALID_ARG, "no warm-start network for r = %d (nmf_set_warmstart)", p->r);
  const int64_t m = p->m, n = p->n;
  const int r = p->r, F = 3 * r, Hd = ctx->warm_hidden;
  float* Wb = a.take<float>(m * r);
  float* Hb = a.take<float>(r * n);
  float* hs = a.take<float>(r);
  float* Fw = a.take<float>(m * F);
  float* Fh = a.take<float>(n * F);
  float* Dw = a.take<float>(m * r);
  float* Dh = a.take<float>(n * r);
  size_t rest = 0;
  void* ws = a.rest(&rest);
  NMF_CUDA(nmfrp::launch_warmstart_features(launcher(ctx), m, n, r, p->ell, QL, Xhat, Wb, Hb, hs,
                                            Fw, Fh, ws, rest),
           "warm-start features");
  const int64_t np_ = nmfrp::mlp_param_count(F, Hd, r);
  NMF_CUDA(nmfrp::launch_mlp_forward(launcher(ctx), F, Hd, r, ctx->warm, Fw, m, Dw, ws, rest),
           "warm-start network (W)");
  NMF_CUDA(nmfrp::launch_mlp_forward(launcher(ctx), F, Hd, r, ctx->warm + np_, Fh, n, Dh, ws, rest),
           "warm-start network (H)");
  NMF_CUDA(nmfrp::launch_warmstart_apply(launcher(ctx), m, n, r, Wb, Dw, Hb, Dh, hs, W, H),
           "warm-start factors");
  return NMF_OK;
}

bool mlp_shape_ok(int F, int hidden, int r) {
  return F >= 1 && F <= 4096 && hidden >= 1 && hidden <= 1024 && r >= 1 && r <= 1024;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

nmf_status nmf_create(nmf_ctx** out, int device, void* cuda_stream) {
  if (!out) return NMF_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return NMF_ERR_CUDA;
  }
  nmf_ctx* ctx = new nmf_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(device);
  if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_qrbad, 8 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&ctx->d_res, 2 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_res, 2 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_mon, 4 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&ctx->d_flags, 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_solve, 8 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_done, 2 * sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_flags, 0, 4 * sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_mon, 0, 4 * sizeof(float)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    nmf_destroy(ctx);
    return NMF_ERR_CUDA;
  }
  *out = ctx;
  return NMF_OK;
}

void nmf_destroy(nmf_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (const PhaseMark& mk : ctx->marks) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_qrbad) cudaFree(ctx->d_qrbad);
  if (ctx->d_wh0) cudaFree(ctx->d_wh0);
  if (ctx->d_res) cudaFree(ctx->d_res);
  if (ctx->h_res) cudaFreeHost(ctx->h_res);
  if (ctx->d_mon) cudaFree(ctx->d_mon);
  if (ctx->d_flags) cudaFree(ctx->d_flags);
  if (ctx->d_solve) cudaFree(ctx->d_solve);
  if (ctx->h_done) cudaFreeHost(ctx->h_done);
  for (int i = 0; i < nmf_ctx::kSide; ++i) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->side_ev[i]) cudaEventDestroy(ctx->side_ev[i]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
  if (ctx->warm) cudaFree(ctx->warm);
  if (ctx->d_loss) cudaFree(ctx->d_loss);
  if (ctx->d_bres) cudaFree(ctx->d_bres);
  if (ctx->h_bres) cudaFreeHost(ctx->h_bres);
  delete ctx;
}

nmf_status nmf_set_stream(nmf_ctx* ctx, void* cuda_stream) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return NMF_OK;
}

const char* nmf_last_error(const nmf_ctx* ctx) { return ctx ? ctx->msg : "context is NULL"; }

int64_t nmf_launch_count(const nmf_ctx* ctx) { return ctx ? ctx->launches : 0; }

nmf_status nmf_last_solve_info(const nmf_ctx* ctx, int32_t* iters, int32_t* exact_checks) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (iters) *iters = ctx->last_iters;
  if (exact_checks) *exact_checks = ctx->last_checks;
  return NMF_OK;
}

nmf_status nmf_last_batch_info(const nmf_ctx* ctx, int32_t* rows_per_block) {
  if (!ctx || !rows_per_block) return NMF_ERR_INVALID_ARG;
  *rows_per_block = ctx->last_batch_rows_per_block;
  return NMF_OK;
}

// ---------------------------------------------------------------- sparse X (CSR)

nmf_status check_csr(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr, const int32_t* col,
                     const float* val, int64_t nnz) {
  if (!row_ptr || nnz < 0 || (nnz > 0 && (!col || !val)))
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad CSR arrays (row_ptr, col, val, nnz)");
  if (p->n > 0x7fffffffLL) return fail(ctx, NMF_ERR_INVALID_ARG, "n must fit in int32 columns");
  return NMF_OK;
}

// Workspace of a sparse call beyond `extra`: the CSC transpose, then the larger of its build
// scratch and the call's own scratch.
size_t csr_ws(const nmf_params* p, int64_t nnz, size_t extra) {
  return nmfrp::csc_bytes(p->n, nnz) + 1024 +
         std::max(nmfrp::csc_ws_bytes(p->m, p->n, nnz) + 1024, extra);
}

nmf_status csr_prepare(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr,
                       const int32_t* col, const float* val, int64_t nnz, Arena& a,
                       nmfrp::CsrView* X, nmfrp::CscView* XT) {
  X->ptr = row_ptr;
  X->idx = col;
  X->val = val;
  void* csc = a.take<char>(nmfrp::csc_bytes(p->n, nnz));
  size_t rest = 0;
  void* ws = a.rest(&rest);   // the build's counts: free again once the transpose is placed
  NMF_CUDA(nmfrp::launch_csc_build(launcher(ctx), row_ptr, col, val, p->m, p->n, nnz, csc, ws,
                                   rest, XT),
           "CSC transpose");
  return NMF_OK;
}

nmf_status csr_pass(nmf_ctx* ctx, const nmf_params* p, const nmfrp::CsrView& X,
                    const nmfrp::CscView& XT, const float* V, const float* U, float* Y, float* Z) {
  Phase ph(ctx, NMF_PHASE_DUAL_PASS);
  NMF_CUDA(nmfrp::launch_csr_dual(launcher(ctx), X, XT, p->m, p->n, p->ell, V, U, Y, Z),
           "sparse pass");
  return NMF_OK;
}

nmf_status csr_compress(nmf_ctx* ctx, const nmf_params* p, const nmfrp::CsrView& X,
                        const nmfrp::CscView& XT, const float* QL, const float* QR, float* Xhat,
                        float* Xchk, Arena a) {
  const int64_t n = p->n;
  const int l = p->ell;
  float* XhatT = a.take<float>(n * l);
  nmf_status st = csr_pass(ctx, p, X, XT, QR, QL, Xchk, XhatT);
  if (st != NMF_OK) return st;
  dim3 grid(static_cast<unsigned>(cdiv(n, 32)), static_cast<unsigned>(cdiv(l, 32)));
  transpose_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(XhatT, n, l, Xhat);
  ctx->launches++;
  NMF_CUDA(cudaGetLastError(), "transpose");
  return NMF_OK;
}

nmf_status csr_residual(nmf_ctx* ctx, const nmf_params* p, const nmfrp::CsrView& X,
                        const float* W, const float* H, double* rel, double* e2o, double* x2o,
                        Arena a) {
  size_t rest = 0;
  void* ws = a.rest(&rest);
  Phase ph(ctx, NMF_PHASE_RESIDUAL);
  NMF_CUDA(nmfrp::launch_sparse_residual(launcher(ctx), X, p->m, p->n, W, H, p->r, ctx->d_res, ws,
                                         rest),
           "sparse residual");
  ph.end();
  NMF_CUDA(cudaMemcpyAsync(ctx->h_res, ctx->d_res, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "residual copy");
  NMF_CUDA(cudaStreamSynchronize(ctx->stream), "residual sync");
  const double e2 = ctx->h_res[0], x2 = ctx->h_res[1];
  if (e2o) *e2o = e2;
  if (x2o) *x2o = x2;
  if (!std::isfinite(e2) || !std::isfinite(x2))
    return fail(ctx, NMF_ERR_NOT_FINITE, "residual is not finite");
  // the expanded form can round a tiny error below zero
  if (rel) *rel = x2 > 0 ? std::sqrt(std::max(e2, 0.0) / x2) : std::sqrt(std::max(e2, 0.0));
  return NMF_OK;
}

nmf_status nmf_sketch_csr(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr,
                          const int32_t* col, const float* val, int64_t nnz,
                          const float* omega_L, const float* omega_R, float* QL, float* QR) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if ((st = check_csr(ctx, p, row_ptr, col, val, nnz)) != NMF_OK) return st;
  if (!QL || !QR) return fail(ctx, NMF_ERR_INVALID_ARG, "QL/QR is NULL");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, csr_ws(p, nnz, sketch_ws(p, !omega_L || !omega_R)))) != NMF_OK)
    return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  nmfrp::CsrView X;
  nmfrp::CscView XT;
  if ((st = csr_prepare(ctx, p, row_ptr, col, val, nnz, a, &X, &XT)) != NMF_OK) return st;
  auto pass = [&](const float* V, const float* U, float* Y, float* Z) {
    return csr_pass(ctx, p, X, XT, V, U, Y, Z);
  };
  return sketch_core(ctx, p, pass, omega_L, omega_R, QL, QR, a,
                     (p->flags & NMF_FLAG_ROBUST_QR) != 0);
}

nmf_status nmf_compress_csr(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr,
                            const int32_t* col, const float* val, int64_t nnz, const float* QL,
                            const float* QR, float* Xhat, float* Xchk) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if ((st = check_csr(ctx, p, row_ptr, col, val, nnz)) != NMF_OK) return st;
  if (!QL || !QR || !Xhat || !Xchk) return fail(ctx, NMF_ERR_INVALID_ARG, "NULL output");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, csr_ws(p, nnz, sizeof(float) * p->n * p->ell + 1024))) != NMF_OK)
    return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  nmfrp::CsrView X;
  nmfrp::CscView XT;
  if ((st = csr_prepare(ctx, p, row_ptr, col, val, nnz, a, &X, &XT)) != NMF_OK) return st;
  return csr_compress(ctx, p, X, XT, QL, QR, Xhat, Xchk, a);
}

nmf_status nmf_residual_csr(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr,
                            const int32_t* col, const float* val, int64_t nnz, const float* W,
                            const float* H, double* rel_err_host, double* err2_host,
                            double* x2_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!p || p->m < 1 || p->n < 1 || p->r < 1 || p->r > 128)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad sizes (m, n >= 1, 1 <= r <= 128)");
  nmf_status st = check_csr(ctx, p, row_ptr, col, val, nnz);
  if (st != NMF_OK) return st;
  if (!W || !H || !rel_err_host) return fail(ctx, NMF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, nmfrp::sparse_residual_ws_bytes(p->m, p->n, p->r) + 1024)) != NMF_OK)
    return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  nmfrp::CsrView X{row_ptr, col, val};
  return csr_residual(ctx, p, X, W, H, rel_err_host, err2_host, x2_host, a);
}

nmf_status nmf_solve_csr(nmf_ctx* ctx, const nmf_params* p, int32_t init, const int64_t* row_ptr,
                         const int32_t* col, const float* val, int64_t nnz, float* W, float* H,
                         double* rel_err_host, int32_t* iters_done_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if ((st = check_csr(ctx, p, row_ptr, col, val, nnz)) != NMF_OK) return st;
  if (!W || !H) return fail(ctx, NMF_ERR_INVALID_ARG, "W/H is NULL");
  if (init != NMF_INIT_GIVEN && init != NMF_INIT_NNDSVD && init != NMF_INIT_MLP)
    return fail(ctx, NMF_ERR_INVALID_ARG, "unknown init %d", init);
  if (init == NMF_INIT_MLP && (!ctx->warm || ctx->warm_r != p->r))
    return fail(ctx, NMF_ERR_INVALID_ARG, "no warm-start network for r = %d (nmf_set_warmstart)", p->r);
  if (p->iters < 0) return fail(ctx, NMF_ERR_INVALID_ARG, "iters < 0");
  DeviceGuard g(ctx->device);
  const int64_t m = p->m, n = p->n, l = p->ell;
  size_t scratch = sketch_ws(p, true);
  scratch = std::max(scratch, sizeof(float) * n * l + 1024);
  scratch = std::max(scratch, nmfrp::iterate_ws_bytes(m, n, p->r, p->ell));
  scratch = std::max(scratch, nmfrp::iterate_persistent_ws_bytes(p->r, p->ell));
  scratch = std::max(scratch, nmfrp::sparse_residual_ws_bytes(m, n, p->r));
  scratch = std::max(scratch, nmfrp::nndsvd_ws_bytes(m, n, p->r, p->ell));
  scratch = std::max(scratch, warm_ws_bytes(p, std::max(ctx->warm_hidden, 256)));
  const size_t fixed = sizeof(float) * (2 * (m * l + n * l)) + 4096;   // QL QR Xhat Xchk
  if ((st = ensure_ws(ctx, csr_ws(p, nnz, fixed + scratch))) != NMF_OK) return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  nmfrp::CsrView X;
  nmfrp::CscView XT;
  if ((st = csr_prepare(ctx, p, row_ptr, col, val, nnz, a, &X, &XT)) != NMF_OK) return st;
  float* QL = a.take<float>(m * l);
  float* QR = a.take<float>(n * l);
  float* Xhat = a.take<float>(l * n);
  float* Xchk = a.take<float>(m * l);
  auto pass = [&](const float* V, const float* U, float* Y, float* Z) {
    return csr_pass(ctx, p, X, XT, V, U, Y, Z);
  };
  // sparse term-count matrices can be numerically rank deficient: repairing QRs throughout
  Arena sa = a;
  if ((st = sketch_core(ctx, p, pass, nullptr, nullptr, QL, QR, sa, true)) != NMF_OK) return st;
  if ((st = csr_compress(ctx, p, X, XT, QL, QR, Xhat, Xchk, a)) != NMF_OK) return st;
  if (init == NMF_INIT_NNDSVD) {
    Phase ph(ctx, NMF_PHASE_INIT);
    size_t rest = 0;
    void* ws = a.rest(&rest);
    cudaError_t e = nmfrp::launch_nndsvd(launcher(ctx), m, n, p->r, p->ell, QL, Xhat, W, H, ws,
                                         rest, ctx->d_status);
    if (e == cudaErrorNotSupported) return fail(ctx, NMF_ERR_UNSUPPORTED, "nndsvd not available");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nndsvd");
  } else if (init == NMF_INIT_MLP) {
    Phase ph(ctx, NMF_PHASE_INIT);
    if ((st = warm_init(ctx, p, QL, Xhat, W, H, a)) != NMF_OK) return st;
  }
  // iterate in chunks of residual_every; the exact sparse residual (nnz-proportional) after each
  const int every = p->residual_every > 0 ? p->residual_every : std::max(p->iters, 1);
  int done = 0, checks = 0;
  double rel = 0.0;
  do {
    const int k = std::min(every, p->iters - done);
    if (k > 0 && (st = iterate_impl(ctx, p, QL, QR, Xhat, Xchk, W, H, k, a)) != NMF_OK) return st;
    done += std::max(k, 0);
    if ((st = csr_residual(ctx, p, X, W, H, &rel, nullptr, nullptr, a)) != NMF_OK) return st;
    ++checks;
    if ((st = take_status(ctx)) != NMF_OK) return st;
    if (p->target_rel_err > 0.0 && rel <= p->target_rel_err) break;
  } while (done < p->iters);
  ctx->last_iters = done;
  ctx->last_checks = checks;
  if (rel_err_host) *rel_err_host = rel;
  if (iters_done_host) *iters_done_host = done;
  return NMF_OK;
}

nmf_status nmf_iterate_full(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                            float* W, float* H, int32_t iters) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!p) return fail(ctx, NMF_ERR_INVALID_ARG, "NULL params");
  if (p->m < 1 || p->n < 1 || p->r < 1 || p->r > std::min<int64_t>(p->m, p->n))
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad sizes (m, n >= 1, 1 <= r <= min(m, n))");
  if (p->r > 64) return fail(ctx, NMF_ERR_UNSUPPORTED, "full-data iterations support r <= 64");
  if (p->rule != NMF_RULE_FASTHALS_RP && p->rule != NMF_RULE_MU_RP)
    return fail(ctx, NMF_ERR_INVALID_ARG, "unknown rule %d", p->rule);
  if (p->prec < NMF_PREC_FP32 || p->prec > NMF_PREC_FP8_E4M3)
    return fail(ctx, NMF_ERR_INVALID_ARG, "unknown precision %d", p->prec);
  if (!X || !W || !H || iters < 0) return fail(ctx, NMF_ERR_INVALID_ARG, "bad arguments");
  if (p->prec == NMF_PREC_FP32 ? ldx < p->n : ldx != p->n)
    return fail(ctx, NMF_ERR_INVALID_ARG, "ldx must be >= n (FP32 X) or n (BF16 / FP8 copy)");
  DeviceGuard g(ctx->device);
  nmf_status st = ensure_ws(ctx, nmfrp::iterate_full_ws_bytes(p->m, p->n, p->r));
  if (st != NMF_OK) return st;
  Phase ph(ctx, NMF_PHASE_ITERATE);
  const cudaError_t e = nmfrp::launch_iterate_full(
      launcher(ctx), X, x_type_of(p->prec), p->m, p->n, ldx, p->r, p->rule,
      static_cast<float>(p->alpha), static_cast<float>(p->beta), eps_of(p), W, H, iters, ctx->ws,
      ctx->ws_bytes, ctx->d_status, (p->flags & NMF_FLAG_SIMT_DUAL_PASS) != 0);
  if (e == cudaErrorNotSupported) return fail(ctx, NMF_ERR_UNSUPPORTED, "full-data iterations");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "full-data iterations");
  return NMF_OK;
}

nmf_status nmf_spectrum(nmf_ctx* ctx, int64_t n, int32_t ell, const float* Xhat,
                        double* sigma_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!Xhat || !sigma_host || n < 1 || ell < 1 || ell > 128 || ell > n)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad spectrum arguments (1 <= ell <= min(n, 128))");
  DeviceGuard g(ctx->device);
  const size_t need = nmfrp::spectrum_ws_bytes(n, ell) + sizeof(float) * 128 + 256;
  nmf_status st = ensure_ws(ctx, need);
  if (st != NMF_OK) return st;
  char* base = static_cast<char*>(ctx->ws);
  float* sig = reinterpret_cast<float*>(base);
  void* rest = base + 1024;
  NMF_CUDA(nmfrp::launch_spectrum(launcher(ctx), n, ell, Xhat, rest, ctx->ws_bytes - 1024, sig),
           "spectrum");
  float h[128];
  NMF_CUDA(cudaMemcpyAsync(h, sig, sizeof(float) * ell, cudaMemcpyDeviceToHost, ctx->stream),
           "spectrum copy");
  NMF_CUDA(cudaStreamSynchronize(ctx->stream), "spectrum sync");
  for (int j = 0; j < ell; ++j) sigma_host[j] = h[j];
  return NMF_OK;
}

nmf_status nmf_decay_rate(const double* sigma, int32_t count, double rel_floor, double* p_out) {
  if (!sigma || !p_out || count < 2 || !(rel_floor >= 0.0)) return NMF_ERR_INVALID_ARG;
  // least-squares slope of log sigma_j against j over the values above rel_floor * sigma_1
  const double top = sigma[0];
  if (!(top > 0.0)) return NMF_ERR_INVALID_ARG;
  double sj = 0, sl = 0, sjj = 0, sjl = 0;
  int k = 0;
  for (int j = 0; j < count; ++j) {
    if (!(sigma[j] > rel_floor * top) || !(sigma[j] > 0.0)) continue;
    const double x = j, y = std::log(sigma[j]);
    sj += x;
    sl += y;
    sjj += x * x;
    sjl += x * y;
    ++k;
  }
  if (k < 2) return NMF_ERR_INVALID_ARG;
  const double den = k * sjj - sj * sj;
  if (!(den > 0.0)) return NMF_ERR_INVALID_ARG;
  *p_out = -(k * sjl - sj * sl) / den;
  return NMF_OK;
}

nmf_status nmf_gini(nmf_ctx* ctx, const float* B, int64_t count, double* gini_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!B || count < 1 || !gini_host) return fail(ctx, NMF_ERR_INVALID_ARG, "bad gini arguments");
  DeviceGuard g(ctx->device);
  nmf_status st = ensure_ws(ctx, nmfrp::gini_ws_bytes(count));
  if (st != NMF_OK) return st;
  NMF_CUDA(nmfrp::launch_gini(launcher(ctx), B, count, ctx->ws, ctx->ws_bytes, ctx->d_res),
           "gini");
  NMF_CUDA(cudaMemcpyAsync(ctx->h_res, ctx->d_res, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "gini copy");
  NMF_CUDA(cudaStreamSynchronize(ctx->stream), "gini sync");
  const double num = ctx->h_res[0], tot = ctx->h_res[1];
  if (!std::isfinite(num) || !std::isfinite(tot))
    return fail(ctx, NMF_ERR_NOT_FINITE, "gini sums are not finite");
  *gini_host = tot != 0.0 ? num / (static_cast<double>(count) * tot) : 0.0;
  return NMF_OK;
}

nmf_status nmf_set_wait_limit(nmf_ctx* ctx, int64_t cycles) {
  if (!ctx || cycles < 0) return NMF_ERR_INVALID_ARG;
  ctx->wait_cycles = cycles;
  return NMF_OK;
}

nmf_status nmf_monitor_terms(nmf_ctx* ctx, double* terms) {
  if (!ctx || !terms) return NMF_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  float mon[2] = {0.f, 0.f};
  double solve[4] = {0, 0, 0, 0};
  NMF_CUDA(cudaMemcpyAsync(mon, ctx->d_mon, sizeof(mon), cudaMemcpyDeviceToHost, ctx->stream),
           "monitor copy");
  NMF_CUDA(cudaMemcpyAsync(solve, ctx->d_solve, sizeof(solve), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "monitor copy");
  NMF_CUDA(cudaStreamSynchronize(ctx->stream), "monitor sync");
  terms[0] = mon[0];
  terms[1] = mon[1];
  terms[2] = solve[0];
  terms[3] = solve[3];
  return NMF_OK;
}

nmf_status nmf_set_profiling(nmf_ctx* ctx, int32_t on) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  ctx->profiling = on != 0;
  return NMF_OK;
}

nmf_status nmf_phase_times(nmf_ctx* ctx, double* ms, int64_t* counts, int32_t reset) {
  if (!ctx || !ms || !counts) return NMF_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  resolve_marks(ctx);
  for (int i = 0; i < NMF_PHASE_COUNT; ++i) {
    ms[i] = ctx->phase_ms[i];
    counts[i] = ctx->phase_n[i];
    if (reset) {
      ctx->phase_ms[i] = 0.0;
      ctx->phase_n[i] = 0;
    }
  }
  return NMF_OK;
}

nmf_status nmf_sync(nmf_ctx* ctx) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  return take_status(ctx);
}

nmf_status nmf_workspace_size(const nmf_params* p, size_t* bytes) {
  if (!p || !bytes) return NMF_ERR_INVALID_ARG;
  if (check_params(nullptr, p) != NMF_OK) return NMF_ERR_INVALID_ARG;
  const int64_t m = p->m, n = p->n, l = p->ell, r = p->r;
  size_t b = 0;
  if (p->prec == NMF_PREC_BF16) b += 2 * static_cast<size_t>(m * ((n + 7) / 8 * 8)) + 1024;
  if (p->prec == NMF_PREC_FP8_E4M3) b += nmfrp::fp8_copy_bytes(m, n) + 1024;
  b += sizeof(float) * (2 * (m * l + n * l) + l * n + m * l) + 4096;  // QL QR Xhat Xchk + omega
  size_t scratch = sketch_ws(p, true);
  scratch = std::max(scratch, sizeof(float) * n * l + 1024 + pass_scratch(m, n, p->ell));
  scratch = std::max(scratch, nmfrp::iterate_ws_bytes(m, n, p->r, p->ell));
  scratch = std::max(scratch, nmfrp::iterate_persistent_ws_bytes(p->r, p->ell));
  scratch = std::max(scratch, nmfrp::residual_ws_bytes_tc(m, n));
  scratch = std::max(scratch, nmfrp::nndsvd_ws_bytes(m, n, p->r, p->ell));
  scratch = std::max(scratch, warm_ws_bytes(p, 256));
  (void)r;
  *bytes = b + scratch;
  return NMF_OK;
}

nmf_status nmf_gaussian(nmf_ctx* ctx, int64_t rows, int64_t cols, uint64_t seed,
                        uint32_t stream_id, float* out) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (rows < 0 || cols < 0 || (!out && rows * cols > 0))
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad gaussian arguments");
  DeviceGuard g(ctx->device);
  NMF_CUDA(nmfrp::launch_gaussian(launcher(ctx), rows, cols, seed, stream_id, out), "gaussian");
  return NMF_OK;
}

size_t nmf_quantized_bytes(int32_t prec, int64_t m, int64_t n) {
  if (m < 1 || n < 1) return 0;
  if (prec == NMF_PREC_BF16) return 2 * static_cast<size_t>(m * n);
  if (prec == NMF_PREC_FP8_E4M3) return nmfrp::fp8_copy_bytes(m, n);
  if (prec == NMF_PREC_FP32) return 4 * static_cast<size_t>(m * n);
  return 0;
}

nmf_status nmf_quantize(nmf_ctx* ctx, int32_t prec, const float* X, int64_t m, int64_t n,
                        int64_t ldx, void* Xq) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (prec != NMF_PREC_BF16 && prec != NMF_PREC_FP8_E4M3)
    return fail(ctx, NMF_ERR_INVALID_ARG, "quantize makes a BF16 or an FP8 copy");
  if (!X || !Xq || m < 1 || n < 1 || ldx < n)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad quantize arguments");
  DeviceGuard g(ctx->device);
  if (prec == NMF_PREC_FP8_E4M3) {
    nmf_status st = ensure_ws(ctx, nmfrp::quantize_stats_ws_bytes() + 4096);
    if (st != NMF_OK) return st;
    NMF_CUDA(nmfrp::launch_quantize_fp8_stats(launcher(ctx), X, m, n, ldx,
                                              static_cast<uint8_t*>(Xq), nullptr, nullptr,
                                              ctx->ws, ctx->ws_bytes),
             "quantize");
    return NMF_OK;
  }
  NMF_CUDA(nmfrp::launch_quantize_bf16(launcher(ctx), X, m, n, ldx,
                                       static_cast<__nv_bfloat16*>(Xq), n),
           "quantize");
  return NMF_OK;
}

nmf_status nmf_dual_pass(nmf_ctx* ctx, int32_t prec, const void* X, int64_t m, int64_t n,
                         int64_t ldx, int32_t ell, const float* V, const float* U, float* Y,
                         float* Z) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!X || m < 1 || n < 1 || ell < 1 || ell > 128 || ldx < n)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad dual pass sizes");
  if (prec != NMF_PREC_FP32 && prec != NMF_PREC_BF16 && prec != NMF_PREC_FP8_E4M3)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad precision %d", prec);
  if (prec != NMF_PREC_FP32 && ldx != n)
    return fail(ctx, NMF_ERR_INVALID_ARG, "BF16 / FP8 X must be the dense copy (ldx == n)");
  if ((V == nullptr) != (Y == nullptr) || (U == nullptr) != (Z == nullptr) || (!V && !U))
    return fail(ctx, NMF_ERR_INVALID_ARG, "V/Y and U/Z must be given in pairs");
  DeviceGuard g(ctx->device);
  nmf_status st = ensure_ws(ctx, nmfrp::dual_pass_ws_bytes(m, n, ell) + 4096);
  if (st != NMF_OK) return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  return dual(ctx, X, prec, m, n, ldx, ell, V, U, Y, Z, a);
}

nmf_status nmf_qr(nmf_ctx* ctx, const float* Y, int64_t rows, int32_t ell, float* Q) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!Y || !Q || ell < 1 || ell > 128 || rows < ell)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad qr arguments");
  DeviceGuard g(ctx->device);
  nmf_status st = ensure_ws(ctx, nmfrp::qr_ws_bytes(rows, ell) + 4096);
  if (st != NMF_OK) return st;
  NMF_CUDA(nmfrp::launch_qr(launcher(ctx), Y, rows, ell, Q, ctx->ws, ctx->ws_bytes,
                            ctx->d_status),
           "qr");
  return NMF_OK;
}

nmf_status nmf_sketch(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                      const float* omega_L, const float* omega_R, float* QL, float* QR) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if ((st = check_x(ctx, p, X, ldx)) != NMF_OK) return st;
  if (!QL || !QR) return fail(ctx, NMF_ERR_INVALID_ARG, "QL/QR is NULL");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, sketch_ws(p, !omega_L || !omega_R))) != NMF_OK) return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  return sketch_impl(ctx, p, X, ldx, omega_L, omega_R, QL, QR, a,
                     (p->flags & NMF_FLAG_ROBUST_QR) != 0);
}

nmf_status nmf_compress(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                        const float* QL, const float* QR, float* Xhat, float* Xchk) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if ((st = check_x(ctx, p, X, ldx)) != NMF_OK) return st;
  if (!QL || !QR || !Xhat || !Xchk) return fail(ctx, NMF_ERR_INVALID_ARG, "NULL output");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, sizeof(float) * p->n * p->ell + 1024 +
                               pass_scratch(p->m, p->n, p->ell))) != NMF_OK)
    return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  return compress_impl(ctx, p, X, ldx, QL, QR, Xhat, Xchk, a);
}

nmf_status nmf_iterate(nmf_ctx* ctx, const nmf_params* p, const float* QL, const float* QR,
                       const float* Xhat, const float* Xchk, float* W, float* H, int32_t iters) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if (!QL || !QR || !Xhat || !Xchk || !W || !H)
    return fail(ctx, NMF_ERR_INVALID_ARG, "NULL argument");
  if (iters < 0) return fail(ctx, NMF_ERR_INVALID_ARG, "iters < 0");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, std::max(nmfrp::iterate_ws_bytes(p->m, p->n, p->r, p->ell),
                                     nmfrp::iterate_persistent_ws_bytes(p->r, p->ell)))) != NMF_OK)
    return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  return iterate_impl(ctx, p, QL, QR, Xhat, Xchk, W, H, iters, a);
}

nmf_status nmf_residual(nmf_ctx* ctx, const nmf_params* p, const float* X, int64_t ldx,
                        const float* W, const float* H, double* rel_err_host, double* err2_host,
                        double* x2_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!p || p->m < 1 || p->n < 1 || p->r < 1 || p->r > 128)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad residual sizes");
  if (!X || !W || !H || ldx < p->n) return fail(ctx, NMF_ERR_INVALID_ARG, "bad residual arguments");
  DeviceGuard g(ctx->device);
  nmf_status st = ensure_ws(ctx, (p->flags & NMF_FLAG_TC_RESIDUAL)
                                     ? nmfrp::residual_ws_bytes_tc(p->m, p->n)
                                     : nmfrp::residual_ws_bytes(p->m, p->n));
  if (st != NMF_OK) return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  return residual_impl(ctx, p, X, ldx, W, H, rel_err_host, err2_host, x2_host, a);
}

nmf_status nmf_residual_static(int32_t device, void* stream, const float* X, int64_t m,
                               int64_t n, int64_t ldx, int32_t r, const float* W, const float* H,
                               double* out_dev) {
  if (!X || !W || !H || !out_dev || m < 1 || n < 1 || ldx < n || r < 1 || r > 128)
    return NMF_ERR_INVALID_ARG;
  DeviceGuard g(device);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != device) return NMF_ERR_INVALID_ARG;
  void* scratch = nullptr;
  if (nmfrp::residual_static_scratch(device, &scratch) != cudaSuccess) return NMF_ERR_CUDA;
  const size_t cap = nmfrp::residual_static_capacity_bytes();
  if (nmfrp::residual_ws_bytes(m, n) > cap) return NMF_ERR_UNSUPPORTED;
  nmfrp::Launcher L;
  L.stream = static_cast<cudaStream_t>(stream);
  if (nmfrp::launch_residual(L, X, m, n, ldx, W, H, r, out_dev, scratch, cap) != cudaSuccess)
    return NMF_ERR_CUDA;
  return NMF_OK;
}

nmf_status nmf_nndsvd(nmf_ctx* ctx, const nmf_params* p, const float* QL, const float* Xhat,
                      float* W, float* H) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if (!QL || !Xhat || !W || !H) return fail(ctx, NMF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, nmfrp::nndsvd_ws_bytes(p->m, p->n, p->r, p->ell))) != NMF_OK) return st;
  cudaError_t e = nmfrp::launch_nndsvd(launcher(ctx), p->m, p->n, p->r, p->ell, QL, Xhat, W, H,
                                       ctx->ws, ctx->ws_bytes, ctx->d_status);
  if (e == cudaErrorNotSupported) return fail(ctx, NMF_ERR_UNSUPPORTED, "nndsvd not available");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "nndsvd");
  return NMF_OK;
}

// One run of the whole pipeline; robust: sketch QRs repair rank-deficient pass outputs.
nmf_status solve_impl(nmf_ctx* ctx, const nmf_params* p, int32_t init, const float* X,
                      int64_t ldx, float* W, float* H, double* rel_err_host,
                      int32_t* iters_done_host, bool robust) {
  nmf_status st = NMF_OK;
  size_t need = 0;
  nmf_workspace_size(p, &need);
  if (init == NMF_INIT_MLP && ctx->warm_hidden > 256)
    need += warm_ws_bytes(p, ctx->warm_hidden);
  if ((st = ensure_ws(ctx, need)) != NMF_OK) return st;
  const int64_t m = p->m, n = p->n, l = p->ell;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  const void* Xp = X;
  int64_t ldp = ldx;
  NMF_CUDA(cudaMemsetAsync(ctx->d_solve, 0, 8 * sizeof(double), ctx->stream), "solve state");
  if (p->prec == NMF_PREC_BF16) {
    const int64_t ldq = (n + 7) / 8 * 8;   // row pitch a TMA descriptor can address
    __nv_bfloat16* Xq = a.take<__nv_bfloat16>(m * ldq);
    Phase ph(ctx, NMF_PHASE_QUANTIZE);
    size_t qrest = 0;
    void* qws = a.rest(&qrest);
    // ||X||^2 into solve[0] and the rounding term <X - X_q, X> of the monitor into solve[3]
    NMF_CUDA(nmfrp::launch_quantize_bf16_stats(launcher(ctx), X, m, n, ldx, Xq, ldq,
                                               ctx->d_solve, ctx->d_solve + 3, qws, qrest),
             "quantize");
    Xp = Xq;
    ldp = ldq;
  } else if (p->prec == NMF_PREC_FP8_E4M3) {
    uint8_t* Xq = a.take<uint8_t>(static_cast<int64_t>(nmfrp::fp8_copy_bytes(m, n)));
    Phase ph(ctx, NMF_PHASE_QUANTIZE);
    size_t qrest = 0;
    void* qws = a.rest(&qrest);
    // ||X||^2 into solve[0]; the compression reads the FP32 X (below), so the monitor needs no
    // rounding term and solve[3] stays 0
    NMF_CUDA(nmfrp::launch_quantize_fp8_stats(launcher(ctx), X, m, n, ldx, Xq, ctx->d_solve,
                                              nullptr, qws, qrest),
             "quantize");
    Xp = Xq;
    ldp = n;
  }
  float* QL = a.take<float>(m * l);
  float* QR = a.take<float>(n * l);
  float* Xhat = a.take<float>(l * n);
  float* Xchk = a.take<float>(m * l);
  if ((st = sketch_impl(ctx, p, Xp, ldp, nullptr, nullptr, QL, QR, a, robust)) != NMF_OK)
    return st;
  if (p->prec == NMF_PREC_FP8_E4M3) {
    // precision recovery: the E4M3 rounding of X (relative error up to 2^-4) would set the
    // floor of the compressed problem, so the compression reads the FP32 X with the final Q
    nmf_params p32 = *p;
    p32.prec = NMF_PREC_FP32;
    if ((st = compress_impl(ctx, &p32, X, ldx, QL, QR, Xhat, Xchk, a)) != NMF_OK) return st;
  } else if ((st = compress_impl(ctx, p, Xp, ldp, QL, QR, Xhat, Xchk, a)) != NMF_OK) {
    return st;
  }
  if (init == NMF_INIT_NNDSVD) {
    Phase ph(ctx, NMF_PHASE_INIT);
    cudaError_t e = nmfrp::launch_nndsvd(launcher(ctx), m, n, p->r, p->ell, QL, Xhat, W, H, a.rest(&need),
                                         need, ctx->d_status);
    if (e == cudaErrorNotSupported) return fail(ctx, NMF_ERR_UNSUPPORTED, "nndsvd not available");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nndsvd");
  } else if (init == NMF_INIT_MLP) {
    Phase ph(ctx, NMF_PHASE_INIT);
    if ((st = warm_init(ctx, p, QL, Xhat, W, H, a)) != NMF_OK) return st;
  }
  // Device-side loop: iterate a chunk, gate the exact residual on the error monitor, run it,
  // decide; the host queues one chunk ahead and stops once the device has raised `done`.
  const int every = p->residual_every > 0 ? p->residual_every : std::max(p->iters, 1);
  const double margin = 0.05, margin_cal = 0.002;
  size_t rest = 0;
  void* ws = a.rest(&rest);
  NMF_CUDA(cudaMemsetAsync(ctx->d_flags, 0, 4 * sizeof(int), ctx->stream), "solve flags");
  NMF_CUDA(cudaMemsetAsync(ctx->d_mon, 0, 4 * sizeof(float), ctx->stream), "solve monitor");
  if (p->prec == NMF_PREC_FP32)
    NMF_CUDA(nmfrp::launch_sumsq(launcher(ctx), X, m, n, ldx, ctx->d_solve, ws, rest), "sumsq");
  const bool staged = (p->flags & NMF_FLAG_STAGED_ITERATE) || !nmfrp::iterate_persistent_supported(p->m, p->n, p->r, p->ell);
  cudaEvent_t ev[2] = {pool_event(ctx), pool_event(ctx)};
  if (!ev[0] || !ev[1]) return fail(ctx, NMF_ERR_CUDA, "event creation");
  int done = 0, chunk = 0;
  nmf_status result = NMF_OK;
  if (!staged && p->iters > 0) {
    // The persistent kernel gates the checks itself and returns only when an exact residual is
    // due; each launch resumes from the count it left on the device. The host queues one launch
    // ahead (a launch after convergence does nothing) and stops once the device raises `done`.
    if (p->r > 64) return fail(ctx, NMF_ERR_UNSUPPORTED, "iterations support r <= 64");
    const nmfrp::IterArgs ia = iter_args(ctx, p, QL, QR, Xhat, Xchk, W, H);
    nmfrp::SolveGate g;
    g.total = p->iters;
    g.every = every;
    g.flags = ctx->d_flags;
    g.solve = ctx->d_solve;
    g.target = p->target_rel_err;
    g.margin = margin;
    g.margin_cal = margin_cal;
    const int max_chunks = (p->iters + every - 1) / every + 2;
    for (chunk = 0; chunk < max_chunks; ++chunk) {
      {
        Phase ph(ctx, NMF_PHASE_ITERATE);
        NMF_CUDA(nmfrp::launch_iterate_persistent_gated(launcher(ctx), ia, g, ws, rest,
                                                        ctx->d_status, ctx->d_mon),
                 "iterate (persistent, gated)");
      }
      {
        Phase ph(ctx, NMF_PHASE_RESIDUAL);
        NMF_CUDA(nmfrp::launch_residual(launcher(ctx), X, m, n, ldx, W, H, p->r, ctx->d_res, ws,
                                        rest, ctx->d_flags + 1, ctx->d_status),
                 "residual");
      }
      solve_decide_gated_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_res, p->target_rel_err,
                                                          p->iters, ctx->d_solve, ctx->d_flags);
      ctx->launches += 1;
      NMF_CUDA(cudaGetLastError(), "solve loop");
      NMF_CUDA(cudaMemcpyAsync(ctx->h_done + (chunk & 1), ctx->d_flags, sizeof(int),
                               cudaMemcpyDeviceToHost, ctx->stream),
               "done copy");
      NMF_CUDA(cudaEventRecord(ev[chunk & 1], ctx->stream), "event");
      if (chunk >= 1) {
        NMF_CUDA(cudaEventSynchronize(ev[(chunk - 1) & 1]), "event wait");
        if (ctx->h_done[(chunk - 1) & 1]) break;
      }
    }
    done = p->iters;   // the loop below does not run
  }
  while (done < p->iters || (p->iters == 0 && chunk == 0)) {
    const int k = std::min(every, p->iters - done);
    if (k > 0 && (st = iterate_impl(ctx, p, QL, QR, Xhat, Xchk, W, H, k, a, ctx->d_flags)) != NMF_OK) {
      result = st;
      break;
    }
    done += std::max(k, 0);
    const bool last = done >= p->iters;
    // the staged iteration kernels do not feed the monitor: check exactly every time
    solve_gate_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_mon, ctx->d_solve, p->target_rel_err,
                                                margin, margin_cal, (last || staged) ? 1 : 0,
                                                ctx->d_flags);
    {
      Phase ph(ctx, NMF_PHASE_RESIDUAL);
      NMF_CUDA(nmfrp::launch_residual(launcher(ctx), X, m, n, ldx, W, H, p->r, ctx->d_res, ws,
                                      rest, ctx->d_flags + 1, ctx->d_status),
               "residual");
    }
    solve_decide_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_res, p->target_rel_err, done,
                                                  ctx->d_solve, ctx->d_flags);
    ctx->launches += 2;
    NMF_CUDA(cudaGetLastError(), "solve loop");
    NMF_CUDA(cudaMemcpyAsync(ctx->h_done + (chunk & 1), ctx->d_flags, sizeof(int),
                             cudaMemcpyDeviceToHost, ctx->stream),
             "done copy");
    NMF_CUDA(cudaEventRecord(ev[chunk & 1], ctx->stream), "event");
    // the persistent kernel skips its work once `done` is set, so one chunk may be queued ahead;
    // the per-stage kernels do not look at the flag, so their chunks are waited for one by one
    const int look = staged ? chunk : chunk - 1;
    if (look >= 0) {
      NMF_CUDA(cudaEventSynchronize(ev[look & 1]), "event wait");
      if (ctx->h_done[look & 1]) break;
    }
    ++chunk;
    if (p->iters == 0) break;
  }
  ctx->pool.push_back(ev[0]);
  ctx->pool.push_back(ev[1]);
  if (result != NMF_OK) return result;
  double out[3] = {0, 0, 0};
  int flags[4] = {0, 0, 0, 0};
  NMF_CUDA(cudaMemcpyAsync(out, ctx->d_solve, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "solve result");
  NMF_CUDA(cudaMemcpyAsync(flags, ctx->d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "solve flags");
  NMF_CUDA(cudaStreamSynchronize(ctx->stream), "solve sync");
  ctx->last_iters = static_cast<int>(out[2]);
  ctx->last_checks = flags[3];
  if (!std::isfinite(out[0])) {
    // a NaN or an infinity in X: every later quantity is meaningless, whatever else the device
    // latched on the way (a QR breakdown from a NaN pivot, say), so clear it and report X
    take_status(ctx);
    return fail(ctx, NMF_ERR_NOT_FINITE, "X holds a NaN or an infinity (||X||^2 is not finite)");
  }
  if ((st = take_status(ctx)) != NMF_OK) return st;   // a QR breakdown is reported as such
  if (!(out[1] == out[1]) || out[1] > 1e300) return fail(ctx, NMF_ERR_NOT_FINITE, "residual is not finite");
  if (rel_err_host) *rel_err_host = out[1];
  if (iters_done_host) *iters_done_host = static_cast<int32_t>(out[2]);
  return NMF_OK;
}

nmf_status nmf_solve(nmf_ctx* ctx, const nmf_params* p, int32_t init, const float* X, int64_t ldx,
                     float* W, float* H, double* rel_err_host, int32_t* iters_done_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if (!X || !W || !H || ldx < p->n) return fail(ctx, NMF_ERR_INVALID_ARG, "bad solve arguments");
  if (init != NMF_INIT_GIVEN && init != NMF_INIT_NNDSVD && init != NMF_INIT_MLP)
    return fail(ctx, NMF_ERR_INVALID_ARG, "unknown init %d", init);
  if (init == NMF_INIT_MLP && (!ctx->warm || ctx->warm_r != p->r))
    return fail(ctx, NMF_ERR_INVALID_ARG, "no warm-start network for r = %d (nmf_set_warmstart)", p->r);
  if (p->iters < 0) return fail(ctx, NMF_ERR_INVALID_ARG, "iters < 0");
  DeviceGuard g(ctx->device);
  // given initial factors are kept so that a rank-deficient sketch can run again with repaired
  // QRs (the first run updates W, H in place)
  const size_t wh = static_cast<size_t>(p->m * p->r + p->r * p->n);
  if (init == NMF_INIT_GIVEN) {
    if (ctx->wh0_cap < wh) {
      if (ctx->d_wh0) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->d_wh0);
        ctx->d_wh0 = nullptr;
        ctx->wh0_cap = 0;
      }
      NMF_CUDA(cudaMalloc(&ctx->d_wh0, sizeof(float) * wh), "initial factors");
      ctx->wh0_cap = wh;
    }
    NMF_CUDA(cudaMemcpyAsync(ctx->d_wh0, W, sizeof(float) * p->m * p->r,
                             cudaMemcpyDeviceToDevice, ctx->stream), "initial factors");
    NMF_CUDA(cudaMemcpyAsync(ctx->d_wh0 + p->m * p->r, H, sizeof(float) * p->r * p->n,
                             cudaMemcpyDeviceToDevice, ctx->stream), "initial factors");
  }
  st = solve_impl(ctx, p, init, X, ldx, W, H, rel_err_host, iters_done_host, false);
  if (st != NMF_ERR_QR_BREAKDOWN) return st;
  if (init == NMF_INIT_GIVEN) {
    NMF_CUDA(cudaMemcpyAsync(W, ctx->d_wh0, sizeof(float) * p->m * p->r,
                             cudaMemcpyDeviceToDevice, ctx->stream), "initial factors");
    NMF_CUDA(cudaMemcpyAsync(H, ctx->d_wh0 + p->m * p->r, sizeof(float) * p->r * p->n,
                             cudaMemcpyDeviceToDevice, ctx->stream), "initial factors");
  }
  return solve_impl(ctx, p, init, X, ldx, W, H, rel_err_host, iters_done_host, true);
}

int64_t nmf_mlp_param_count(int32_t F, int32_t hidden, int32_t r) {
  if (!mlp_shape_ok(F, hidden, r)) return -1;
  return nmfrp::mlp_param_count(F, hidden, r);
}

nmf_status nmf_warmstart_features(nmf_ctx* ctx, const nmf_params* p, const float* QL,
                                  const float* Xhat, float* Wb, float* Hb, float* hscale,
                                  float* Fw, float* Fh) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  nmf_status st = check_params(ctx, p);
  if (st != NMF_OK) return st;
  if (!QL || !Xhat || !Wb || !Hb || !hscale || !Fw || !Fh)
    return fail(ctx, NMF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(ctx->device);
  if ((st = ensure_ws(ctx, nmfrp::nndsvd_ws_bytes(p->m, p->n, p->r, p->ell))) != NMF_OK) return st;
  cudaError_t e = nmfrp::launch_warmstart_features(launcher(ctx), p->m, p->n, p->r, p->ell, QL,
                                                   Xhat, Wb, Hb, hscale, Fw, Fh, ctx->ws,
                                                   ctx->ws_bytes);
  if (e == cudaErrorNotSupported) return fail(ctx, NMF_ERR_UNSUPPORTED, "r or ell too large");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "warm-start features");
  return NMF_OK;
}

nmf_status nmf_mlp_forward(nmf_ctx* ctx, int32_t F, int32_t hidden, int32_t r,
                           const float* params, const float* X, int64_t rows, float* Y) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!mlp_shape_ok(F, hidden, r) || rows < 1 || rows > (int64_t(1) << 30) || !params || !X || !Y)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad network forward arguments");
  DeviceGuard g(ctx->device);
  nmf_status st = ensure_ws(ctx, nmfrp::mlp_ws_bytes(rows, hidden, r));
  if (st != NMF_OK) return st;
  NMF_CUDA(nmfrp::launch_mlp_forward(launcher(ctx), F, hidden, r, params, X, rows, Y, ctx->ws,
                                     ctx->ws_bytes),
           "network forward");
  return NMF_OK;
}

nmf_status nmf_mlp_loss_grad(nmf_ctx* ctx, int32_t F, int32_t hidden, int32_t r,
                             const float* params, const float* X, const float* T, int64_t rows,
                             float* grad, double* loss_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!mlp_shape_ok(F, hidden, r) || rows < 1 || rows > (int64_t(1) << 30) || !params || !X ||
      !T || !grad)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad network gradient arguments");
  DeviceGuard g(ctx->device);
  nmf_status st = ensure_ws(ctx, nmfrp::mlp_ws_bytes(rows, hidden, r));
  if (st != NMF_OK) return st;
  if (!ctx->d_loss) NMF_CUDA(cudaMalloc(&ctx->d_loss, sizeof(double)), "loss slot");
  NMF_CUDA(nmfrp::launch_mlp_loss_grad(launcher(ctx), F, hidden, r, params, X, T, rows, grad,
                                       ctx->d_loss, ctx->ws, ctx->ws_bytes),
           "network gradient");
  if (loss_host) {
    NMF_CUDA(cudaMemcpyAsync(ctx->h_res, ctx->d_loss, sizeof(double), cudaMemcpyDeviceToHost,
                             ctx->stream),
             "loss copy");
    NMF_CUDA(cudaStreamSynchronize(ctx->stream), "loss sync");
    *loss_host = ctx->h_res[0];
  }
  return NMF_OK;
}

nmf_status nmf_mlp_adam(nmf_ctx* ctx, int64_t count, float* params, float* m, float* v,
                        const float* grad, int32_t step, float lr) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (count < 1 || !params || !m || !v || !grad || step < 1 || !(lr > 0.f))
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad Adam arguments");
  DeviceGuard g(ctx->device);
  NMF_CUDA(nmfrp::launch_adam(launcher(ctx), params, m, v, grad, count, lr, step), "Adam");
  return NMF_OK;
}

nmf_status nmf_mlp_train_step(nmf_ctx* ctx, int32_t F, int32_t hidden, int32_t r, float* params,
                              float* m, float* v, float* grad, int32_t step, float lr,
                              const float* X, const float* T, int64_t rows, double* loss_host) {
  nmf_status st = nmf_mlp_loss_grad(ctx, F, hidden, r, params, X, T, rows, grad, loss_host);
  if (st != NMF_OK) return st;
  return nmf_mlp_adam(ctx, nmfrp::mlp_param_count(F, hidden, r), params, m, v, grad, step, lr);
}

nmf_status nmf_warmstart_apply(nmf_ctx* ctx, int64_t m, int64_t n, int32_t r, const float* Wb,
                               const float* Dw, const float* Hb, const float* Dh,
                               const float* hscale, float* W, float* H) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || r < 1 || !Wb || !Dw || !Hb || !Dh || !hscale || !W || !H)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad warm-start arguments");
  DeviceGuard g(ctx->device);
  NMF_CUDA(nmfrp::launch_warmstart_apply(launcher(ctx), m, n, r, Wb, Dw, Hb, Dh, hscale, W, H),
           "warm-start factors");
  return NMF_OK;
}

nmf_status nmf_warmstart_targets(nmf_ctx* ctx, int64_t m, int64_t n, int32_t r, const float* Wb,
                                 const float* Hb, const float* hscale, const float* Wstar,
                                 const float* Hstar, float* Tw, float* Th) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || r < 1 || !Wb || !Hb || !hscale || !Wstar || !Hstar || !Tw || !Th)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad warm-start target arguments");
  DeviceGuard g(ctx->device);
  NMF_CUDA(nmfrp::launch_warmstart_targets(launcher(ctx), m, n, r, Wb, Hb, hscale, Wstar, Hstar,
                                           Tw, Th),
           "warm-start targets");
  return NMF_OK;
}

nmf_status nmf_set_warmstart(nmf_ctx* ctx, int32_t hidden, int32_t r, const float* params_w,
                             const float* params_h) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (!mlp_shape_ok(3 * r, hidden, r) || !params_w || !params_h)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad warm-start network");
  DeviceGuard g(ctx->device);
  const int64_t np_ = nmfrp::mlp_param_count(3 * r, hidden, r);
  if (ctx->warm) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->warm);
    ctx->warm = nullptr;
  }
  NMF_CUDA(cudaMalloc(&ctx->warm, sizeof(float) * 2 * np_), "warm-start network");
  NMF_CUDA(cudaMemcpyAsync(ctx->warm, params_w, sizeof(float) * np_, cudaMemcpyDefault, ctx->stream),
           "warm-start network");
  NMF_CUDA(cudaMemcpyAsync(ctx->warm + np_, params_h, sizeof(float) * np_, cudaMemcpyDefault,
                           ctx->stream),
           "warm-start network");
  ctx->warm_hidden = hidden;
  ctx->warm_r = r;
  return NMF_OK;
}

nmf_status nmf_solve_batched(nmf_ctx* ctx, int32_t count, const nmf_params* p, int32_t init,
                             const float* const* X, const int64_t* ldx, float* const* W,
                             float* const* H, int32_t rows_per_block, double* rel_err_host) {
  if (!ctx) return NMF_ERR_INVALID_ARG;
  if (count < 1 || !p || !X || !ldx || !W || !H || !rel_err_host)
    return fail(ctx, NMF_ERR_INVALID_ARG, "bad batched arguments");
  if (init != NMF_INIT_GIVEN && init != NMF_INIT_NNDSVD && init != NMF_INIT_MLP)
    return fail(ctx, NMF_ERR_INVALID_ARG, "unknown init %d", init);
  if (rows_per_block < 0) return fail(ctx, NMF_ERR_INVALID_ARG, "rows_per_block < 0");
  for (int i = 0; i < count; ++i) {
    nmf_status st = check_params(ctx, &p[i]);
    if (st != NMF_OK) return st;
    if (p[i].prec == NMF_PREC_FP8_E4M3)
      return fail(ctx, NMF_ERR_UNSUPPORTED, "problem %d: FP8 copies are single-solve only", i);
    if (!X[i] || !W[i] || !H[i] || ldx[i] < p[i].n)
      return fail(ctx, NMF_ERR_INVALID_ARG, "problem %d: bad pointers or ldx", i);
    if (p[i].iters < 0) return fail(ctx, NMF_ERR_INVALID_ARG, "problem %d: iters < 0", i);
    if (init == NMF_INIT_MLP && (!ctx->warm || ctx->warm_r != p[i].r))
      return fail(ctx, NMF_ERR_INVALID_ARG, "problem %d: no warm-start network for r = %d", i, p[i].r);
    if (nmfrp::iterate_multi_min_blocks(p[i].m, p[i].n, p[i].r, p[i].ell) < 1)
      return fail(ctx, NMF_ERR_UNSUPPORTED, "problem %d: r or ell too large for batching", i);
  }
  DeviceGuard g(ctx->device);
  const int nside = count < nmf_ctx::kSide ? count : nmf_ctx::kSide;
  for (int k = 0; k < nside; ++k) {
    if (!ctx->side[k]) {
      NMF_CUDA(cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking), "side stream");
      NMF_CUDA(cudaEventCreateWithFlags(&ctx->side_ev[k], cudaEventDisableTiming), "side event");
    }
  }
  if (!ctx->fork_ev) NMF_CUDA(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "fork event");
  if (ctx->bres_cap < count) {
    if (ctx->d_bres) cudaFree(ctx->d_bres);
    if (ctx->h_bres) cudaFreeHost(ctx->h_bres);
    ctx->d_bres = nullptr;
    ctx->h_bres = nullptr;
    ctx->bres_cap = 0;
    NMF_CUDA(cudaMalloc(&ctx->d_bres, sizeof(double) * 2 * count + sizeof(float) * 2 * count + 64),
             "batch results");
    NMF_CUDA(cudaMallocHost(&ctx->h_bres, sizeof(double) * 2 * count), "batch results");
    ctx->bres_cap = count;
  }
  float* d_mon = reinterpret_cast<float*>(ctx->d_bres + 2 * count);
  // workspace: per problem Q_L, Q_R, X_hat, X_chk; the iteration sums; one scratch per stream
  std::vector<nmfrp::IterArgs> ia(count);
  size_t keep = 0, scratch = 0;
  for (int i = 0; i < count; ++i) {
    const nmf_params* q = &p[i];
    keep += sizeof(float) * (2 * (q->m + q->n) * q->ell) + 4 * 256;
    const int64_t ldq = (q->n + 7) / 8 * 8;
    size_t s = q->prec == NMF_PREC_BF16 ? 2 * static_cast<size_t>(q->m * ldq) + 256 : 0;
    size_t rest = sketch_ws(q, true);
    rest = std::max(rest, sizeof(float) * q->n * q->ell + 1024 + pass_scratch(q->m, q->n, q->ell));
    rest = std::max(rest, nmfrp::nndsvd_ws_bytes(q->m, q->n, q->r, q->ell));
    rest = std::max(rest, nmfrp::residual_ws_bytes(q->m, q->n));
    rest = std::max(rest, nmfrp::quantize_stats_ws_bytes());
    if (init == NMF_INIT_MLP) rest = std::max(rest, warm_ws_bytes(q, std::max(ctx->warm_hidden, 1)));
    scratch = std::max(scratch, s + rest + 1024);
    ia[i].m = q->m;
    ia[i].n = q->n;
    ia[i].r = q->r;
    ia[i].ell = q->ell;
    ia[i].rule = q->rule;
    ia[i].alpha = static_cast<float>(q->alpha);
    ia[i].beta = static_cast<float>(q->beta);
    ia[i].eps = eps_of(q);
  }
  const size_t iter_ws = nmfrp::iterate_multi_ws_bytes(ia.data(), count);
  nmf_status st = ensure_ws(ctx, keep + iter_ws + nside * scratch + 8192);
  if (st != NMF_OK) return st;
  Arena a{static_cast<char*>(ctx->ws), ctx->ws_bytes};
  for (int i = 0; i < count; ++i) {
    ia[i].QL = a.take<float>(p[i].m * p[i].ell);
    ia[i].QR = a.take<float>(p[i].n * p[i].ell);
    ia[i].Xhat = a.take<float>(p[i].ell * p[i].n);
    ia[i].Xchk = a.take<float>(p[i].m * p[i].ell);
    ia[i].W = W[i];
    ia[i].H = H[i];
  }
  char* iter_base = a.take<char>(iter_ws);
  std::vector<char*> sbase(nside);
  for (int k = 0; k < nside; ++k) sbase[k] = a.take<char>(scratch);
  const cudaStream_t main_stream = ctx->stream;
  // fork from / join to `origin`
  auto fork = [&](cudaStream_t origin) -> nmf_status {
    NMF_CUDA(cudaEventRecord(ctx->fork_ev, origin), "fork");
    for (int k = 0; k < nside; ++k)
      if (ctx->side[k] != origin) NMF_CUDA(cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0), "fork");
    return NMF_OK;
  };
  auto join = [&](cudaStream_t origin) -> nmf_status {
    for (int k = 0; k < nside; ++k) {
      if (ctx->side[k] == origin) continue;
      NMF_CUDA(cudaEventRecord(ctx->side_ev[k], ctx->side[k]), "join");
      NMF_CUDA(cudaStreamWaitEvent(origin, ctx->side_ev[k], 0), "join");
    }
    return NMF_OK;
  };
  // phase 1: sketch, compression (and NNDSVD) of each problem on its side stream
  auto phase1 = [&](cudaStream_t origin) -> nmf_status {
    nmf_status r1 = fork(origin);
    if (r1 != NMF_OK) return r1;
    for (int i = 0; i < count && r1 == NMF_OK; ++i) {
      const int k = i % nside;
      ctx->stream = ctx->side[k];
      const nmf_params* q = &p[i];
      Arena sa{sbase[k], scratch};
      const void* Xp = X[i];
      int64_t ldp = ldx[i];
      if (q->prec == NMF_PREC_BF16) {
        const int64_t ldq = (q->n + 7) / 8 * 8;
        __nv_bfloat16* Xq = sa.take<__nv_bfloat16>(q->m * ldq);
        Phase ph(ctx, NMF_PHASE_QUANTIZE);
        cudaError_t e = nmfrp::launch_quantize_bf16(launcher(ctx), X[i], q->m, q->n, ldx[i], Xq, ldq);
        if (e != cudaSuccess) {
          r1 = cuda_fail(ctx, e, "quantize");
          break;
        }
        Xp = Xq;
        ldp = ldq;
      }
      if ((r1 = sketch_impl(ctx, q, Xp, ldp, nullptr, nullptr, const_cast<float*>(ia[i].QL),
                            const_cast<float*>(ia[i].QR), sa)) != NMF_OK)
        break;
      if ((r1 = compress_impl(ctx, q, Xp, ldp, ia[i].QL, ia[i].QR, const_cast<float*>(ia[i].Xhat),
                              const_cast<float*>(ia[i].Xchk), sa)) != NMF_OK)
        break;
      if (init == NMF_INIT_NNDSVD) {
        Phase ph(ctx, NMF_PHASE_INIT);
        size_t rest = 0;
        void* ws = sa.rest(&rest);
        cudaError_t e = nmfrp::launch_nndsvd(launcher(ctx), q->m, q->n, q->r, q->ell, ia[i].QL,
                                             ia[i].Xhat, W[i], H[i], ws, rest, ctx->d_status);
        if (e != cudaSuccess) r1 = cuda_fail(ctx, e, "nndsvd");
      } else if (init == NMF_INIT_MLP) {
        Phase ph(ctx, NMF_PHASE_INIT);
        r1 = warm_init(ctx, q, ia[i].QL, ia[i].Xhat, W[i], H[i], sa);
      }
    }
    ctx->stream = main_stream;
    if (r1 != NMF_OK) return r1;
    return join(origin);
  };
  // Without per-phase timing, phase 1 (thousands of small launches for a large batch) is captured
  // into a CUDA graph once and replayed while the problems, X, the workspace (and for NNDSVD, W
  // and H) stay the same; the capture runs on side stream 0, which waits for the context stream.
  bool replayed = false;
  if (!ctx->profiling) {
    uint64_t key = 1469598103934665603ull;
    auto mix = [&key](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
    mix(static_cast<uint64_t>(count));
    mix(static_cast<uint64_t>(init));
    mix(reinterpret_cast<uintptr_t>(ctx->ws));
    mix(static_cast<uint64_t>(ctx->ws_bytes));
    for (int i = 0; i < count; ++i) {
      const unsigned char* pb = reinterpret_cast<const unsigned char*>(&p[i]);
      for (size_t b = 0; b < sizeof(nmf_params); ++b) mix(pb[b]);
      mix(reinterpret_cast<uintptr_t>(X[i]));
      mix(static_cast<uint64_t>(ldx[i]));
      if (init != NMF_INIT_GIVEN) {
        mix(reinterpret_cast<uintptr_t>(W[i]));
        mix(reinterpret_cast<uintptr_t>(H[i]));
      }
    }
    if (init == NMF_INIT_MLP) {
      mix(reinterpret_cast<uintptr_t>(ctx->warm));
      mix(static_cast<uint64_t>(ctx->warm_hidden));
    }
    const cudaStream_t origin = ctx->side[0];
    if (!(ctx->batch_graph && ctx->batch_key == key)) {
      if (ctx->batch_graph) {
        cudaGraphExecDestroy(ctx->batch_graph);
        ctx->batch_graph = nullptr;
      }
      const int64_t l0 = ctx->launches;
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        nmf_status cst = phase1(origin);
        const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
        if (cst == NMF_OK && ec == cudaSuccess && graph &&
            cudaGraphInstantiate(&ctx->batch_graph, graph, 0) == cudaSuccess) {
          ctx->batch_key = key;
          ctx->batch_graph_launches = ctx->launches - l0;
        } else {
          ctx->batch_graph = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();
      ctx->launches = l0;
      ctx->msg[0] = 0;
    }
    if (ctx->batch_graph) {
      NMF_CUDA(cudaEventRecord(ctx->fork_ev, main_stream), "graph fork");
      NMF_CUDA(cudaStreamWaitEvent(origin, ctx->fork_ev, 0), "graph fork");
      NMF_CUDA(cudaGraphLaunch(ctx->batch_graph, origin), "graph launch");
      NMF_CUDA(cudaEventRecord(ctx->side_ev[0], origin), "graph join");
      NMF_CUDA(cudaStreamWaitEvent(main_stream, ctx->side_ev[0], 0), "graph join");
      ctx->launches += ctx->batch_graph_launches;
      replayed = true;
    }
  }
  if (!replayed && (st = phase1(main_stream)) != NMF_OK) return st;
  // phase 2: every problem's iterations, several problems per cooperative launch
  {
    const int sms = [] {
      int dev = 0, n = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      return n > 0 ? n : 148;
    }();
    std::vector<int> iters(count), blocks(count);
    auto plan_blocks = [&](int rpb) {
      for (int i = 0; i < count; ++i) {
        const int64_t want = (p[i].m + rpb - 1) / rpb;
        int b = static_cast<int>(want < sms ? want : sms);
        b = std::max(b, nmfrp::iterate_multi_min_blocks(p[i].m, p[i].n, p[i].r, p[i].ell));
        blocks[i] = std::max(1, b);
      }
    };
    NMF_CUDA(cudaMemsetAsync(ctx->d_flags + 2, 0, sizeof(int), main_stream), "zero flag");
    int rpb = rows_per_block;
    if (rpb == 0) {
      // autotuner: rows of W per block, timed on a few iterations of scratch copies of W, H
      uint64_t key = 1469598103934665603ull;
      for (int i = 0; i < count; ++i)
        for (int64_t v : {p[i].m, p[i].n, static_cast<int64_t>(p[i].r), static_cast<int64_t>(p[i].ell),
                          static_cast<int64_t>(p[i].rule)})
          key = (key ^ static_cast<uint64_t>(v)) * 1099511628211ull;
      for (const auto& kv : ctx->tuned)
        if (kv.first == key) rpb = kv.second;
      if (rpb == 0) {
        static const int kCand[] = {128, 256, 512, 1024};
        size_t wh = 0;
        for (int i = 0; i < count; ++i)
          wh += (sizeof(float) * p[i].m * p[i].r + 255) / 256 * 256 +
                (sizeof(float) * p[i].r * p[i].n + 255) / 256 * 256;
        float* trial = nullptr;
        NMF_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&trial), wh, main_stream), "tuning copies");
        std::vector<nmfrp::IterArgs> ta = ia;
        char* q = reinterpret_cast<char*>(trial);
        for (int i = 0; i < count; ++i) {
          ta[i].W = reinterpret_cast<float*>(q);
          q += (sizeof(float) * p[i].m * p[i].r + 255) / 256 * 256;
          ta[i].H = reinterpret_cast<float*>(q);
          q += (sizeof(float) * p[i].r * p[i].n + 255) / 256 * 256;
        }
        for (int i = 0; i < count; ++i) iters[i] = std::min(p[i].iters, 4);
        cudaEvent_t e0 = pool_event(ctx), e1 = pool_event(ctx);
        float best = 1e30f;
        for (int c : kCand) {
          plan_blocks(c);
          for (int i = 0; i < count; ++i) {
            NMF_CUDA(cudaMemcpyAsync(ta[i].W, W[i], sizeof(float) * p[i].m * p[i].r,
                                     cudaMemcpyDeviceToDevice, main_stream), "tuning copy");
            NMF_CUDA(cudaMemcpyAsync(ta[i].H, H[i], sizeof(float) * p[i].r * p[i].n,
                                     cudaMemcpyDeviceToDevice, main_stream), "tuning copy");
          }
          NMF_CUDA(cudaEventRecord(e0, main_stream), "tuning event");
          NMF_CUDA(nmfrp::launch_iterate_multi(launcher(ctx), ta.data(), iters.data(),
                                               blocks.data(), count, iter_base, iter_ws,
                                               ctx->d_status, d_mon, ctx->d_flags + 2),
                   "tuning iterations");
          NMF_CUDA(cudaEventRecord(e1, main_stream), "tuning event");
          NMF_CUDA(cudaEventSynchronize(e1), "tuning sync");
          float ms = 0.f;
          NMF_CUDA(cudaEventElapsedTime(&ms, e0, e1), "tuning time");
          if (ms < best) {
            best = ms;
            rpb = c;
          }
        }
        ctx->pool.push_back(e0);
        ctx->pool.push_back(e1);
        NMF_CUDA(cudaFreeAsync(trial, main_stream), "tuning copies");
        ctx->tuned.emplace_back(key, rpb);
      }
    }
    ctx->last_batch_rows_per_block = rpb;
    plan_blocks(rpb);
    for (int i = 0; i < count; ++i) iters[i] = p[i].iters;
    Phase ph(ctx, NMF_PHASE_ITERATE);
    NMF_CUDA(nmfrp::launch_iterate_multi(launcher(ctx), ia.data(), iters.data(), blocks.data(),
                                         count, iter_base, iter_ws, ctx->d_status, d_mon,
                                         ctx->d_flags + 2),
             "batched iterations");
  }
  // phase 3: exact residual of each problem
  if ((st = fork(main_stream)) != NMF_OK) return st;
  for (int i = 0; i < count && st == NMF_OK; ++i) {
    const int k = i % nside;
    ctx->stream = ctx->side[k];
    Arena sa{sbase[k], scratch};
    size_t rest = 0;
    void* ws = sa.rest(&rest);
    Phase ph(ctx, NMF_PHASE_RESIDUAL);
    cudaError_t e = nmfrp::launch_residual(launcher(ctx), X[i], p[i].m, p[i].n, ldx[i], W[i], H[i],
                                           p[i].r, ctx->d_bres + 2 * i, ws, rest, nullptr,
                                           ctx->d_status);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "residual");
  }
  ctx->stream = main_stream;
  if (st != NMF_OK) return st;
  if ((st = join(main_stream)) != NMF_OK) return st;
  NMF_CUDA(cudaMemcpyAsync(ctx->h_bres, ctx->d_bres, sizeof(double) * 2 * count,
                           cudaMemcpyDeviceToHost, main_stream),
           "batch results");
  NMF_CUDA(cudaStreamSynchronize(main_stream), "batch sync");
  for (int i = 0; i < count; ++i) {
    const double e2 = ctx->h_bres[2 * i], x2 = ctx->h_bres[2 * i + 1];
    rel_err_host[i] = x2 > 0 ? std::sqrt(e2 / x2) : std::sqrt(e2);
  }
  return take_status(ctx);
}

}  // extern "C"
