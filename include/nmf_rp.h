/*
 * nmf_rp.h -- C ABI of the GB300 (sm_103a) library for random-projection compressed NMF
 * (Torre & Graber, "An Efficient Algorithm for Non-Negative Matrix Factorization with Random
 * Projections", arXiv:1712.02248).
 *
 * Problem (Section 2, Eq. 2.2): min 1/2 ||X - W H||_F^2 over W >= 0 (m x r), H >= 0 (r x n), for a
 * non-negative X (m x n). The paper's A is W and its B is H^T.
 *
 * Conventions for every entry point
 *  - Matrix arguments are DEVICE pointers (cudaMalloc / torch CUDA tensors) unless the name says
 *    `_host`. They are owned by the caller; the library never frees or retains them past a call.
 *  - All matrices are row-major. X has leading dimension `ldx` (elements, ldx >= n). The others are
 *    dense: Omega_L n x l, Omega_R m x l, Q_L m x l, Q_R n x l, X_hat l x n, X_chk m x l,
 *    W m x r, H r x n. l ("ell") is the sketch width r + oversampling.
 *  - Work is queued on the context's CUDA stream and is asynchronous unless the entry point
 *    returns a host value (it then synchronises that stream). Kernel-side failures (QR breakdown,
 *    non-finite values, a bounded wait that ran out) are latched in a device status word and
 *    reported by the next synchronising call (nmf_sync, nmf_residual, nmf_solve).
 *  - Errors are returned as nmf_status; nothing is thrown across the ABI. nmf_last_error() gives
 *    a one-line message for the last failing call on that context.
 *  - The context owns an internal device workspace (grown on demand with cudaMalloc, freed by
 *    nmf_destroy). Calls on one context must not overlap from several host threads.
 */
#ifndef NMF_RP_H
#define NMF_RP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NMF_OK = 0,
  NMF_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or enum value */
  NMF_ERR_CUDA = 2,          /* a CUDA runtime call failed (message in nmf_last_error) */
  NMF_ERR_OOM = 3,           /* workspace allocation failed */
  NMF_ERR_QR_BREAKDOWN = 4,  /* Cholesky pivot not positive: sketch numerically rank deficient */
  NMF_ERR_NOT_FINITE = 5,    /* NaN/Inf met in the residual */
  NMF_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
  NMF_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} nmf_status;

/* Arithmetic type of the X-sized contractions (sketch passes and compression). */
typedef enum {
  NMF_PREC_FP32 = 0,         /* X read as FP32 */
  NMF_PREC_BF16 = 1,         /* X read as BF16, tensor cores, FP32 accumulation */
  NMF_PREC_FP8_E4M3 = 2      /* X read as the FP8 copy of nmf_quantize (E4M3 codes, one E8M0
                                scale a 32 x 32 tile); nmf_solve compresses from the FP32 X */
} nmf_precision;

/* Update rule of the iterations. */
typedef enum {
  NMF_RULE_FASTHALS_RP = 0,  /* Section 4, Eq. fastHALS_a (+ Section 4.1 alpha/beta on H) */
  NMF_RULE_MU_RP = 1         /* Section 3.1, Algorithm 3 with the semi-NMF multiplicative rule */
} nmf_rule;

/* Initialisation used by nmf_solve. */
typedef enum {
  NMF_INIT_GIVEN = 0,        /* W, H hold the caller's initial factors */
  NMF_INIT_NNDSVD = 1,       /* NNDSVD of the compressed data (Boutsidis & Gallopoulos 2008) */
  NMF_INIT_MLP = 2           /* NNDSVD corrected by the learned warm start (nmf_set_warmstart) */
} nmf_init;

/* nmf_params.flags bits. */
enum {
  /* run the iterations as one kernel launch per stage instead of one persistent cooperative
     launch for all iterations (same arithmetic; for comparison and for r > 48, which always
     uses the per-stage kernels) */
  NMF_FLAG_STAGED_ITERATE = 1,
  /* run BF16 / FP8 passes over X on the SIMT pipes instead of the tcgen05 tensor-core kernel */
  NMF_FLAG_SIMT_DUAL_PASS = 2,
  /* nmf_sketch: orthonormalise rank-deficient pass outputs by replacing the columns whose
     Cholesky pivot falls below 1e-12 of their diagonal with Gaussian draws (seeded by p->seed)
     and repeating CholeskyQR2, instead of latching NMF_ERR_QR_BREAKDOWN; synchronises after
     every QR. nmf_solve does this by itself when a first run meets a breakdown. */
  NMF_FLAG_ROBUST_QR = 4,
  /* nmf_residual: rebuild W H on the tensor cores from BF16 hi + lo splits of W and H (FP32 X
     with rows 16-byte aligned, r <= 32; else the FP32 kernels run). Each product is then within
     about 2^-17 of its FP32 value and the squared error within about 1e-6 relative at a 1 %
     residual. nmf_solve's exact residual checks always take this path where it applies. */
  NMF_FLAG_TC_RESIDUAL = 8
};

typedef struct {
  int64_t m, n;              /* X is m x n */
  int32_t r;                 /* number of components (the paper's k), 1 <= r <= ell */
  int32_t ell;               /* sketch width r + r_ov (Section 3), ell <= min(m, n), ell <= 128 */
  int32_t power_iters;       /* w of Eq. 3.5, 0 <= w <= 32 */
  int32_t iters;             /* nmf_solve: maximum number of iterations */
  int32_t rule;              /* nmf_rule */
  int32_t prec;              /* nmf_precision of the sketch / compression contractions */
  uint64_t seed;             /* Philox4x32-10 key for Omega when the caller passes none */
  int32_t residual_every;    /* nmf_solve: exact residual every k iterations (0: at the end) */
  int32_t flags;             /* NMF_FLAG_* bits (0 = defaults) */
  double target_rel_err;     /* nmf_solve: stop at the first check with rel_err <= target (0: off) */
  double alpha, beta;        /* Section 4.1 sparsity / smoothness weights on H (FastHALS-RP) */
  double eps;                /* MU-RP denominator guard (<= 0: 1e-12) */
} nmf_params;

typedef struct nmf_ctx nmf_ctx;

/* Create a context on CUDA device `device` that queues all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
nmf_status nmf_create(nmf_ctx** ctx, int device, void* cuda_stream);
/* Free the context and its workspace. NULL is ignored. Synchronises the stream first. */
void nmf_destroy(nmf_ctx* ctx);
/* Replace the stream future calls are queued on. */
nmf_status nmf_set_stream(nmf_ctx* ctx, void* cuda_stream);
/* One-line description of the last error on this context ("" if none). */
const char* nmf_last_error(const nmf_ctx* ctx);
/* Synchronise the context's stream and return (then clear) the latched device status. */
nmf_status nmf_sync(nmf_ctx* ctx);
/* Number of kernels this context has launched so far (for launch accounting). */
int64_t nmf_launch_count(const nmf_ctx* ctx);
/*
 * Per-phase timing. When profiling is on, every phase below is bracketed by CUDA events recorded
 * on the context stream; nmf_phase_times (synchronises) returns the summed milliseconds and the
 * number of timed spans of each phase (arrays of NMF_PHASE_COUNT), optionally resetting them.
 */
enum {
  NMF_PHASE_QUANTIZE = 0,   /* FP32 -> BF16 copy of X */
  NMF_PHASE_DUAL_PASS = 1,  /* one fused pass over X (sketch pass or compression) */
  NMF_PHASE_QR = 2,         /* one CholeskyQR2 */
  NMF_PHASE_ITERATE = 3,    /* a run of iterations */
  NMF_PHASE_RESIDUAL = 4,   /* one full residual */
  NMF_PHASE_INIT = 5,       /* NNDSVD initialisation */
  NMF_PHASE_COUNT = 6
};
nmf_status nmf_set_profiling(nmf_ctx* ctx, int32_t on);
/*
 * Polling budget, in SM clock cycles, of each grid-barrier wait of the persistent iteration
 * kernel in later launches on this context (0 restores the default of about two seconds; < 0 is
 * NMF_ERR_INVALID_ARG). A wait that runs out latches NMF_ERR_TIMEOUT, raises the launch's abort
 * flag and every block leaves the kernel (no copies are in flight in that kernel); the next
 * synchronising call returns the status and clears it, and W, H then hold partial updates.
 * For testing the time-out path: a budget of a few cycles makes the first barrier run out.
 * The tensor-core pass keeps its own fixed budget (its waits guard asynchronous copies).
 */
nmf_status nmf_set_wait_limit(nmf_ctx* ctx, int64_t cycles);
/*
 * Terms of the error monitor (no read of X) that the last persistent nmf_iterate / nmf_solve
 * left on this context, and the sums the last nmf_solve took of X. Synchronises the stream.
 *   terms[0] = <W_tld^T X_hat, H> (FP32; W_tld = Q_L^T W) at the last iteration's W, H
 *   terms[1] = <W^T W, H H^T>     (FP32) at the same W, H
 *   terms[2] = ||X||_F^2          (FP64) of the last nmf_solve
 *   terms[3] = <X - X_q, X>       (FP64) of the last nmf_solve with a BF16 copy X_q (else 0)
 * The solve's estimate of ||X - W H||^2 is terms[2] - 2 (terms[0] + terms[3]) + terms[1]
 * (Section 3, Eq. 3.4: X replaced by Q_L Q_L^T X in the cross term).
 */
nmf_status nmf_monitor_terms(nmf_ctx* ctx, double* terms);
nmf_status nmf_phase_times(nmf_ctx* ctx, double* ms, int64_t* counts, int32_t reset);
/* Bytes of device workspace nmf_solve needs for these parameters (other calls need less). */
nmf_status nmf_workspace_size(const nmf_params* p, size_t* bytes);

/*
 * Gaussian test matrix (Section 3: Omega has standard-normal entries), rows x cols row-major,
 * from Philox4x32-10 (Salmon et al., SC'11) and the Box-Muller transform: element e = i*cols + k
 * uses lane e % 4 of the generator output for counter (e/4 low word, e/4 high word, stream_id, 0)
 * and key (seed low word, seed high word); words map to uniforms ((x >> 8) + 1/2) 2^-24.
 * nmf_sketch uses stream_id 0 for Omega_L and 1 for Omega_R when they are not given.
 */
nmf_status nmf_gaussian(nmf_ctx* ctx, int64_t rows, int64_t cols, uint64_t seed,
                        uint32_t stream_id, float* out);

/*
 * Low-precision copy of X (FP32, m x n, leading dimension ldx) that the sketch and compression
 * read. `Xq` (device) must hold nmf_quantized_bytes(prec, m, n) bytes.
 *   prec = NMF_PREC_BF16: m*n BF16 codes, dense m x n, round to nearest even.
 *   prec = NMF_PREC_FP8_E4M3: OCP FP8 E4M3 codes, row pitch ldq = n rounded up to 16 bytes (the
 *     pad columns are zero), then, at byte offset ceil(m * ldq / 256) * 256, one E8M0 byte
 *     k + 127 for every 32 x 32 tile (ceil(m/32) rows of ceil(n/32), row-major). 2^k is the
 *     smallest power of two with amax / 2^k <= 448 over the tile (k = 0 for an all-zero tile,
 *     clamped to [-127, 127]); each code is round-to-nearest-even of x / 2^k, saturating, and
 *     the copy's value of x is code * 2^k.
 */
nmf_status nmf_quantize(nmf_ctx* ctx, int32_t prec, const float* X, int64_t m, int64_t n,
                        int64_t ldx, void* Xq);

/* Bytes of the nmf_quantize copy of an m x n matrix (0 for an unknown precision). */
size_t nmf_quantized_bytes(int32_t prec, int64_t m, int64_t n);

/*
 * One fused pass over X (the building block of every sketch and compression step):
 *   Y = X V   (m x l, reduction over n)   and   Z = X^T U   (n x l, reduction over m),
 * reading X once. V is n x l, U is m x l, all FP32 row-major; Y, Z are written (not accumulated).
 * `X` is FP32 (prec = NMF_PREC_FP32, leading dimension ldx) or the BF16 / FP8 copy from
 * nmf_quantize (prec = NMF_PREC_BF16 / NMF_PREC_FP8_E4M3, ldx must equal n; the FP8 copy's
 * values are code * 2^k of its tile scale). Either of V/Y or U/Z may be NULL
 * (both of a pair) to skip that product. 1 <= l <= 128.
 */
nmf_status nmf_dual_pass(nmf_ctx* ctx, int32_t prec, const void* X, int64_t m, int64_t n,
                         int64_t ldx, int32_t ell, const float* V, const float* U,
                         float* Y, float* Z);

/*
 * Thin QR of a tall FP32 matrix Y (rows x l, rows >= l): writes Q (rows x l, FP32, orthonormal
 * columns, the unique Q whose R has a positive diagonal; Section 3, Eq. 3.4-3.5). CholeskyQR2
 * (Fukaya et al. 2014): the Gram matrix Y^T Y, its factor and R^-1 are formed in float-float
 * arithmetic (about 48 significant bits) on the FP32 pipes; a non-positive pivot latches
 * NMF_ERR_QR_BREAKDOWN. Q may alias Y.
 */
nmf_status nmf_qr(nmf_ctx* ctx, const float* Y, int64_t rows, int32_t ell, float* Q);

/*
 * Two-sided sketch (Section 3 Eq. 3.5, Section 3.1): Q_L spans (X X^T)^w X Omega_L, Q_R spans
 * (X^T X)^w X^T Omega_R, orthonormalised after every application of X or X^T, both chains
 * advancing together so that 2w + 1 passes over X serve both. omega_L (n x l) / omega_R (m x l)
 * may be NULL: drawn with nmf_gaussian(seed = p->seed, stream_id 0 / 1).
 * `X` is FP32 with leading dimension ldx (p->prec = FP32), or the nmf_quantize copy of the
 * precision p->prec (BF16 or FP8, ldx = n).
 */
nmf_status nmf_sketch(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                      const float* omega_L, const float* omega_R, float* QL, float* QR);

/* Compression (Section 4, before Algorithm 4): X_hat = Q_L^T X (l x n), X_chk = X Q_R (m x l),
 * in one pass over X. X as for nmf_sketch. */
nmf_status nmf_compress(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                        const float* QL, const float* QR, float* Xhat, float* Xchk);

/*
 * `iters` iterations of the compressed updates on W (m x r) and H (r x n), in place.
 * FastHALS-RP (Eq. fastHALS_a, Section 4.1 form with p->alpha, p->beta): the whole W sweep over
 * components j = 1..r (Gauss-Seidel), normalisation of the columns of W with the scale moved to
 * the rows of H, then the whole H sweep. MU-RP (Algorithm 3): the semi-NMF multiplicative rule on
 * W, then on H. Never reads X.
 * Device arrays owned by the caller, row-major: QL (m x l), QR (n x l), Xhat (l x n), Xchk
 * (m x l), W (m x r), H (r x n). Asynchronous on the context's stream. r <= 48 with the
 * problem's slices fitting on chip runs as one persistent launch per call; otherwise (or with
 * NMF_FLAG_STAGED_ITERATE) one launch per stage and iteration. r > 64: NMF_ERR_UNSUPPORTED;
 * Invalid parameters (r > l, l > 128 or > min(m, n), ...): NMF_ERR_INVALID_ARG.
 */
nmf_status nmf_iterate(nmf_ctx* ctx, const nmf_params* p, const float* QL, const float* QR,
                       const float* Xhat, const float* Xchk, float* W, float* H, int32_t iters);

/*
 * Relative reconstruction error ||X - W H||_F / ||X||_F (the error of Eq. 2.2) written to
 * *rel_err_host; X FP32 with leading dimension ldx. Differences are formed in FP32 and summed in
 * FP64. Synchronises the stream. Returns NMF_ERR_NOT_FINITE if the sum is not finite.
 * `err2_host` / `x2_host` (may be NULL) receive ||X - W H||^2 and ||X||^2.
 */
nmf_status nmf_residual(nmf_ctx* ctx, const nmf_params* p, const float* X, int64_t ldx,
                        const float* W, const float* H, double* rel_err_host,
                        double* err2_host, double* x2_host);

/*
 * The residual sums of nmf_residual without a context and without allocating device memory.
 * The paper has no counterpart: this is a service entry point for callers that cannot allocate
 * when they need the residual, such as a serving loop whose device memory is all handed to its
 * own pools, or code that must not stall the device's other streams (cudaFree synchronises the
 * whole device). The per-block partial sums live in a fixed array of 33,024 bytes in the
 * library's global memory (two doubles per block plus 256 bytes of alignment slack; the grid is
 * at most 4 blocks per SM, so devices with up to 512 SMs fit) instead of a workspace. Nothing in
 * it has to start at zero.
 *
 * device: the CUDA device of X, W, H and out_dev; it is made current for the call.
 * stream: a cudaStream_t of that device (NULL = legacy default stream).
 * X: m x n FP32, row-major with leading dimension ldx >= n. W: m x r, H: r x n, contiguous
 * row-major FP32, 1 <= r <= 128. All device pointers, owned by the caller.
 * out_dev: 2 doubles of device memory: out_dev[0] = ||X - W H||_F^2, out_dev[1] = ||X||_F^2,
 * summed as in nmf_residual. The relative error is sqrt(out_dev[0] / out_dev[1]).
 * The call queues two kernels on `stream` and returns without synchronising.
 *
 * The first call on a device does a one-time set-up: it resolves the array's device address,
 * which can load the library's device code onto the device; make that first call before any
 * stream capture. The address is kept for the life of the process: after cudaDeviceReset on
 * that device it is stale, so do not call this entry point on a device that has been reset. Calls on one device share the array, so two calls in flight at the same time
 * (on different streams, or from different threads) race: order them on one stream or with
 * events.
 * Returns NMF_ERR_INVALID_ARG for NULL pointers, bad sizes or a device that cannot be made
 * current; NMF_ERR_UNSUPPORTED if the device needs more partial-sum slots than the array holds;
 * NMF_ERR_CUDA if the set-up or a launch fails.
 */
nmf_status nmf_residual_static(int32_t device, void* stream, const float* X, int64_t m,
                               int64_t n, int64_t ldx, int32_t r, const float* W, const float* H,
                               double* out_dev);

/*
 * `iters` iterations of the uncompressed methods on the full data X, the baselines the paper
 * compares against (Section 5, Tables 5.2 and 5.3), in place on W (m x r) and H (r x n):
 *   p->rule = NMF_RULE_FASTHALS_RP: FastHALS (Section 2.2): S_W = X H^T, G_W = H H^T, the W sweep
 *     w_j <- [w_j + (S_W[:,j] - W G_W[:,j]) / G_W[j,j]]_+ over j = 1..r (Gauss-Seidel), the
 *     normalisation w_j /= ||w_j|| with h_j *= ||w_j||, then S_H = W^T X, G_H = W^T W and the H
 *     sweep (Section 4.1 alpha / beta form; plain at alpha = beta = 0).
 *   p->rule = NMF_RULE_MU_RP: Lee-Seung multiplicative updates (Section 2.1, Algorithm 1):
 *     W <- W o (X H^T) / (W H H^T + eps), then H <- H o (W^T X) / (W^T W H + eps).
 * Two passes over X an iteration (the H step needs this iteration's W). X as for nmf_sketch:
 * FP32 with leading dimension ldx (p->prec = FP32), or the nmf_quantize copy of p->prec (ldx = n;
 * the BF16 / FP8 tensor-core pass keeps W and H as hi + lo BF16 pairs, so only X is rounded).
 * Uses p->m, n, r (1 <= r <= 64), rule, prec, alpha, beta, eps, flags; p->ell is not used.
 * Device arrays owned by the caller. Asynchronous on the context's stream.
 * Errors: NMF_ERR_INVALID_ARG (sizes, pointers, ldx, enums), NMF_ERR_UNSUPPORTED (r > 64).
 */
nmf_status nmf_iterate_full(nmf_ctx* ctx, const nmf_params* p, const void* X, int64_t ldx,
                            float* W, float* H, int32_t iters);

/*
 * Sparse X (Section 5.2 applies the methods to a sparse term-frequency matrix). X is m x n in CSR
 * form: row_ptr (m + 1 int64, row_ptr[0] = 0, row_ptr[m] = nnz), col (nnz int32 column indices,
 * distinct within a row, any order) and val (nnz FP32 values), all device arrays owned by the
 * caller; n < 2^31. Each call builds the transpose (CSC form, rows of a column in increasing
 * order) in the context's workspace, so X^T U is a gather like X V and every sum runs in a fixed
 * order (results are bit-identical between runs). The products, the QRs and the updates are
 * FP32 as for dense FP32 X; p->prec is not used.
 *   nmf_sketch_csr:   as nmf_sketch (Section 3 Eq. 3.5 with a QR after every application).
 *   nmf_compress_csr: as nmf_compress (X_hat = Q_L^T X, X_chk = X Q_R).
 *   nmf_residual_csr: ||X - W H||_F / ||X||_F from ||X||^2 - 2 <X, W H> + <W^T W, H H^T> (the
 *     first two over the nonzeros, FP64 sums; the Grams in FP32 within 256-row slabs, FP64 across
 *     them), O(nnz r + (m + n) r^2) work; 1 <= r <= 128. Synchronises the stream.
 *   nmf_solve_csr:    sketch (rank-deficient pass outputs repaired as with NMF_FLAG_ROBUST_QR),
 *     compression, initialisation, then iterations in chunks of p->residual_every with the exact
 *     sparse residual after each; stops at the first check <= p->target_rel_err (if > 0) or after
 *     p->iters iterations. Synchronises the stream.
 * Errors as for the dense calls; NMF_ERR_INVALID_ARG also for a NULL row_ptr, nnz < 0 or NULL
 * col / val with nnz > 0.
 */
nmf_status nmf_sketch_csr(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr,
                          const int32_t* col, const float* val, int64_t nnz,
                          const float* omega_L, const float* omega_R, float* QL, float* QR);
nmf_status nmf_compress_csr(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr,
                            const int32_t* col, const float* val, int64_t nnz, const float* QL,
                            const float* QR, float* Xhat, float* Xchk);
nmf_status nmf_residual_csr(nmf_ctx* ctx, const nmf_params* p, const int64_t* row_ptr,
                            const int32_t* col, const float* val, int64_t nnz, const float* W,
                            const float* H, double* rel_err_host, double* err2_host,
                            double* x2_host);
nmf_status nmf_solve_csr(nmf_ctx* ctx, const nmf_params* p, int32_t init, const int64_t* row_ptr,
                         const int32_t* col, const float* val, int64_t nnz, float* W, float* H,
                         double* rel_err_host, int32_t* iters_done_host);

/*
 * Singular values of the compressed data X_hat (ell x n, row-major FP32 device array owned by the
 * caller), descending, into sigma_host[0..ell). With X ~ Q_L X_hat (Section 3, Eq. 3.4) they are
 * the estimates the sketch gives of sigma_1..sigma_ell of X, whose decay sets how many power
 * iterations w the sketch needs (Section 5.2). Computed as sqrt(lambda_j(X_hat X_hat^T)) from a
 * float-float Gram and a cyclic Jacobi eigensolver in FP32: each lambda_j carries an absolute
 * error of about ell * 1.2e-7 * lambda_1. Synchronises the stream.
 * Errors: NMF_ERR_INVALID_ARG for NULL pointers or sizes outside 1 <= ell <= min(n, 128).
 */
nmf_status nmf_spectrum(nmf_ctx* ctx, int64_t n, int32_t ell, const float* Xhat,
                        double* sigma_host);
/*
 * Decay rate p of a singular-value spectrum (host arrays, no device work). Section 5.2 relates
 * the best number of power iterations to the decay rate p of the spectrum, which it writes as
 * sigma_j(X)^-p; the rates it reports (0.0012 and 0.0053 over spectra of 1000 and 400 values,
 * the slower decay needing more power iterations) fit an exponential decay sigma_j ~ C e^(-p j),
 * so p is taken as minus the least-squares slope of log sigma_j against j over the entries
 * with sigma_j > rel_floor * sigma_1 (sigma[0] = sigma_1 > 0, descending).
 * Errors: NMF_ERR_INVALID_ARG for NULL pointers, count < 2, sigma[0] <= 0, rel_floor < 0, or
 * fewer than two entries above the floor.
 */
nmf_status nmf_decay_rate(const double* sigma, int32_t count, double rel_floor, double* p_out);

/*
 * Gini coefficient of the `count` entries of B (Section 5.1, the sparsity measure of the factor
 * B = H^T in Figures 5.4 and 5.7): G = sum_{i=1..N} (2 i - N - 1) b_(i) / (N sum_i b_(i)) with
 * b_(1) <= ... <= b_(N) the entries in ascending order, N = count. B: device array of count
 * FP32 values (any layout: only the multiset of values matters), owned by the caller. The
 * entries are sorted on the device (bitonic network over order-preserving integer keys) and the
 * sums taken in FP64. G = 0 when the entries sum to zero. Synchronises the stream.
 * Errors: NMF_ERR_INVALID_ARG for NULL pointers or count < 1; NMF_ERR_NOT_FINITE if B holds a
 * NaN or an infinity.
 */
nmf_status nmf_gini(nmf_ctx* ctx, const float* B, int64_t count, double* gini_host);

/* NNDSVD initial factors (Boutsidis & Gallopoulos) from the compressed data: the top r singular
 * triplets of X ~ Q_L X_hat (Section 3, Eq. 3.4) come from the l x l eigenproblem of
 * X_hat X_hat^T (Gram in float-float arithmetic summed in FP64, cyclic Jacobi in FP32), with
 * u_j = Q_L u'_j and v_j = X_hat^T u'_j / sigma_j; each pair keeps its larger sign part.
 * QL: m x l, Xhat: l x n, W: m x r, H: r x n, all row-major FP32 device arrays owned by the
 * caller. Components whose eigenvector error matters are those with small eigenvalue gaps:
 * the FP32 eigensolver gives eigenvector j an error of about l * eps32 * lambda_1 / gap_j. */
nmf_status nmf_nndsvd(nmf_ctx* ctx, const nmf_params* p, const float* QL, const float* Xhat,
                      float* W, float* H);

/*
 * Learned warm start. The paper starts from random factors (Section 5); NNDSVD of the compressed
 * data (above) corrected row by row by a small network trained on solutions of the compressed NMF
 * itself is a faster start. Definitions (r components; u_j, v_j, s_j the singular triplets of
 * X ~ Q_L X_hat; p(x) the part of x NNDSVD keeps: |x| for j = 0, else x+ or x- by the larger
 * product of norms, or nothing):
 *   W_b[:, j] = p(u_j) / ||p(u_j)||,  H_b[j, :] = hscale_j p(v_j) / ||p(v_j)||,
 *   hscale_j = s_j ||p(u_j)|| ||p(v_j)||            (W_b H_b is the NNDSVD product)
 *   F_w[i] = [sqrt(m) c_j u_ij, sqrt(m) W_b[i, j], s_j / s_0]  (j < r; m x 3r, row-major)
 *   F_h[c] = [sqrt(n) c_j v_cj, sqrt(n) H_b[j, c] / hscale_j, s_j / s_0]  (n x 3r)
 *   with c_j u = |u| (j = 0), u (positive part kept), -u (negative part kept), 0 (none)
 *   W_0 = max(0, W_b + D_w / sqrt(m)),  H_0[j][c] = max(0, H_b[j][c] + hscale_j D_h[c][j] / sqrt(n))
 *   with D_w = net_W(F_w) (m x r) and D_h = net_H(F_h) (n x r).
 * A network (F inputs, two hidden ReLU layers of `hidden` units, r outputs) is one FP32 vector
 * [W1 (F x hidden), b1 (hidden), W2 (hidden x hidden), b2, W3 (hidden x r), b3 (r)], matrices
 * row-major, owned by the caller (device memory). The weight matrices are rounded to BF16 (round
 * to nearest even) wherever they enter a product; biases, activations and accumulation are FP32.
 * Loss: mean squared error over rows x r outputs; gradients are those of the rounded weights,
 * laid out like the parameters.
 */
/* Number of parameters of a network (F inputs, hidden units, r outputs); -1 for bad sizes. */
int64_t nmf_mlp_param_count(int32_t F, int32_t hidden, int32_t r);
/* W_b (m x r), H_b (r x n), hscale (r), F_w (m x 3r), F_h (n x 3r) from Q_L (m x l) and
 * X_hat (l x n); device arrays owned by the caller. r <= 64, l <= 128. */
nmf_status nmf_warmstart_features(nmf_ctx* ctx, const nmf_params* p, const float* QL,
                                  const float* Xhat, float* Wb, float* Hb, float* hscale,
                                  float* Fw, float* Fh);
/* Y (rows x r) = network(X) for X (rows x F); device arrays. */
nmf_status nmf_mlp_forward(nmf_ctx* ctx, int32_t F, int32_t hidden, int32_t r,
                           const float* params, const float* X, int64_t rows, float* Y);
/* grad (param_count floats, device) of the loss of network(X) against T (rows x r); the loss is
 * written to *loss_host when it is not NULL (this synchronises). */
nmf_status nmf_mlp_loss_grad(nmf_ctx* ctx, int32_t F, int32_t hidden, int32_t r,
                             const float* params, const float* X, const float* T, int64_t rows,
                             float* grad, double* loss_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias correction for step >= 1) on `count`
 * parameters with moment buffers m, v (device, zero before step 1). */
nmf_status nmf_mlp_adam(nmf_ctx* ctx, int64_t count, float* params, float* m, float* v,
                        const float* grad, int32_t step, float lr);
/* nmf_mlp_loss_grad into `grad` followed by nmf_mlp_adam. */
nmf_status nmf_mlp_train_step(nmf_ctx* ctx, int32_t F, int32_t hidden, int32_t r, float* params,
                              float* m, float* v, float* grad, int32_t step, float lr,
                              const float* X, const float* T, int64_t rows, double* loss_host);
/* W (m x r), H (r x n) from W_b, H_b, hscale and the two network outputs (definitions above). */
nmf_status nmf_warmstart_apply(nmf_ctx* ctx, int64_t m, int64_t n, int32_t r, const float* Wb,
                               const float* Dw, const float* Hb, const float* Dh,
                               const float* hscale, float* W, float* H);
/* Training targets of the two networks, the inverse of nmf_warmstart_apply where the solution is
 * positive: Tw = sqrt(m) (W* - W_b) (m x r) and Th (n x r) with Th[c][j] = sqrt(n) (H*[j][c] -
 * H_b[j][c]) / hscale_j (a zero hscale_j taken as 1). W_b, H_b, hscale as from
 * nmf_warmstart_features, (W*, H*) the solution the networks learn to reach; device arrays owned
 * by the caller. */
nmf_status nmf_warmstart_targets(nmf_ctx* ctx, int64_t m, int64_t n, int32_t r, const float* Wb,
                                 const float* Hb, const float* hscale, const float* Wstar,
                                 const float* Hstar, float* Tw, float* Th);
/* Copy the two networks (F = 3r inputs, host or device memory) into the context for
 * NMF_INIT_MLP; problems with another r are refused at solve time. */
nmf_status nmf_set_warmstart(nmf_ctx* ctx, int32_t hidden, int32_t r, const float* params_w,
                             const float* params_h);

/*
 * Whole pipeline on FP32 X (m x n, leading dimension ldx): sketch (Omega from p->seed), compress,
 * initialise (init), iterate. Every p->residual_every iterations (and after the last one) there
 * is a check; with p->target_rel_err > 0 the solve stops at the first check whose exact relative
 * residual is <= the target, else after p->iters iterations. The exact residual of a check is
 * computed only when an error monitor built from the compressed data alone (||X||^2 -
 * 2 <W_tld^T X_hat, H> + <W^T W, H H^T>) is within 5 % of the target before the first exact
 * check, and within 0.2 % once scaled by the ratio exact / estimate of the last exact check;
 * always for the last check. The decision is taken on the device: the persistent iteration
 * kernel (r <= 48) applies it at every check point itself and returns only when an exact
 * check is due. With p->prec = BF16 the X passes read a BF16
 * copy made in the workspace. W, H: in/out (read only for NMF_INIT_GIVEN). Synchronises the
 * stream. Outputs: *rel_err_host (the last exact relative residual), *iters_done_host
 * (iterations at that check; may be NULL).
 */
nmf_status nmf_solve(nmf_ctx* ctx, const nmf_params* p, int32_t init, const float* X, int64_t ldx,
                     float* W, float* H, double* rel_err_host, int32_t* iters_done_host);

/*
 * Many independent problems in one call (throughput mode; each problem is the computation of
 * nmf_solve with a fixed iteration count). Section 2, Eq. 2.2 per problem; Algorithms 3/4 loop.
 * count >= 1 problems; p[i] their parameters (m, n, r, ell, power_iters, iters, rule, prec,
 * seed, alpha, beta, eps; residual_every and target_rel_err are not used: every problem runs
 * p[i].iters iterations). X, ldx, W, H are HOST arrays of count entries holding DEVICE pointers
 * (X[i]: FP32 m x n, leading dimension ldx[i]; W[i]: m x r, H[i]: r x n in/out, read for
 * NMF_INIT_GIVEN). init applies to all problems. rows_per_block: rows of W a block of the
 * iteration kernel takes; each problem runs on ceil(m / rows_per_block) blocks (at least what its
 * shared-memory slices need, at most the number of SMs), and problems are packed into cooperative
 * launches that fill the SMs. rows_per_block = 0 lets the autotuner choose among 128, 256, 512
 * and 1024 rows: on the first call with a given list of (m, n, r, ell, rule) it times 4 iterations
 * of every candidate on scratch copies of W and H (stream-ordered cudaMallocAsync) and keeps the
 * fastest for later calls on this context (nmf_last_batch_info reports the choice). rel_err_host[i] receives ||X_i - W_i H_i||_F /
 * ||X_i||_F after the iterations. The sketch, compression and residuals of different problems
 * run concurrently on up to 8 internal streams. Synchronises the context stream.
 * Limits: r <= 48, ell <= 128 per problem. Errors as for nmf_solve; NMF_ERR_UNSUPPORTED if a
 * problem is outside the limits.
 */
nmf_status nmf_solve_batched(nmf_ctx* ctx, int32_t count, const nmf_params* p, int32_t init,
                             const float* const* X, const int64_t* ldx, float* const* W,
                             float* const* H, int32_t rows_per_block, double* rel_err_host);

/* Rows per block the last nmf_solve_batched on this context used (autotuned or given). */
nmf_status nmf_last_batch_info(const nmf_ctx* ctx, int32_t* rows_per_block);

/* Iterations and number of exact residual checks of the last nmf_solve on this context. */
nmf_status nmf_last_solve_info(const nmf_ctx* ctx, int32_t* iters, int32_t* exact_checks);

#ifdef __cplusplus
}
#endif

#endif /* NMF_RP_H */
