"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on identical seeded inputs.

Tolerances (relative Frobenius error unless stated):
  FP32 kernels, one step from the oracle's own state ............ 1e-5
  BF16 X contractions, against the oracle on the same BF16 X ..... 1e-5 (FP32 accumulation)
  QR (unique Q with positive R diagonal) ......................... 1e-5, orthogonality 1e-5
  whole runs: final rel_err within 1 % of the oracle's after the same iteration count
  BF16 / integer byte work (quantisation) ........................ bit-exact
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_02248_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def host(t):
    return t.detach().double().cpu().numpy()


def bf16_round(x):
    """Round-to-nearest-even of float32 values to bfloat16, returned as float32 (integer work)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32)


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


# ------------------------------------------------------------------ Omega generator

def test_gaussian_matches_oracle_philox(lib, ctx):
    Z = host(lib.nmf_gaussian(ctx, 37, 19, seed=123456789, stream_id=1))
    ref = O.philox_normal(37, 19, seed=123456789, stream=1)
    assert np.abs(Z - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())


# ------------------------------------------------------------------ quantisation

@pytest.mark.parametrize("shape", [(33, 70), (128, 256), (5, 3)])
def test_quantize_bf16_bit_exact(lib, ctx, shape):
    rng = np.random.default_rng(7)
    X = (rng.standard_normal(shape) * 10.0 ** rng.uniform(-3, 3, shape)).astype(np.float32)
    q = lib.nmf_quantize(ctx, cu(X))
    got = q.view(torch.int16).cpu().numpy().view(np.uint16)
    want = (bf16_round(X).view(np.uint32) >> 16).astype(np.uint16)
    assert np.array_equal(got, want)


# ------------------------------------------------------------------ dual pass (Eq. 3.5 step)

# FP32 X takes the tensor-core pass (hi + lo BF16 splits of X, V and U) when n is a multiple of 4
# and ell <= 80, else the SIMT pass; both are held to 1e-5 of the FP64 products.
DUAL_SHAPES = [(512, 256, 18), (300, 517, 18), (1000, 777, 40), (129, 130, 1), (257, 1025, 70),
               (64, 64, 64), (2000, 300, 128), (1000, 784, 40), (300, 1032, 70), (130, 132, 80),
               (5000, 3000, 48), (77, 4, 3), (4096, 1000, 80), (20000, 5000, 40)]


@pytest.mark.parametrize("m,n,ell", DUAL_SHAPES)
def test_dual_pass_fp32(lib, ctx, m, n, ell):
    rng = np.random.default_rng(m * 7 + n)
    X = rng.uniform(0, 1, (m, n)).astype(np.float32)
    V = rng.standard_normal((n, ell)).astype(np.float32)
    U = rng.standard_normal((m, ell)).astype(np.float32)
    Y, Z = lib.nmf_dual_pass(ctx, cu(X), cu(V), cu(U))
    X64 = X.astype(np.float64)
    ey, ez = rel(host(Y), X64 @ V), rel(host(Z), X64.T @ U)
    print(f"fp32 pass {m}x{n} l={ell} ({'tc' if n % 4 == 0 and ell <= 80 else 'simt'}): "
          f"{ey:.2e} {ez:.2e}")
    assert ey <= 1e-5 and ez <= 1e-5


def test_dual_pass_fp32_tensor_core_is_deterministic_and_handles_signs(lib, ctx):
    """Mixed signs and magnitudes spanning 2^-20 .. 2^20 (the split is relative per element),
    and two runs bit-identical (fixed slot order)."""
    rng = np.random.default_rng(5)
    m, n, ell = 3000, 1024, 40
    X = (rng.standard_normal((m, n)) * 2.0 ** rng.integers(-20, 21, (m, n))).astype(np.float32)
    V = rng.standard_normal((n, ell)).astype(np.float32)
    U = rng.standard_normal((m, ell)).astype(np.float32)
    Y, Z = lib.nmf_dual_pass(ctx, cu(X), cu(V), cu(U))
    Y2, Z2 = lib.nmf_dual_pass(ctx, cu(X), cu(V), cu(U))
    assert torch.equal(Y, Y2) and torch.equal(Z, Z2)
    X64 = X.astype(np.float64)
    # each product is off by at most ~3 * 2^-18 of sum |x| |v|: compare against that scale
    ay = np.abs(X64) @ np.abs(V.astype(np.float64))
    az = np.abs(X64).T @ np.abs(U.astype(np.float64))
    assert np.max(np.abs(host(Y) - X64 @ V) / ay) <= 2e-5
    assert np.max(np.abs(host(Z) - X64.T @ U) / az) <= 2e-5


def test_dual_pass_strided_x_and_single_sides(lib, ctx):
    rng = np.random.default_rng(3)
    big = rng.uniform(0, 1, (200, 333)).astype(np.float32)
    Xv = cu(big)[:, :301]                      # leading dimension 333 > n = 301
    V = rng.standard_normal((301, 24)).astype(np.float32)
    U = rng.standard_normal((200, 24)).astype(np.float32)
    Y, _ = lib.nmf_dual_pass(ctx, Xv, V=cu(V))
    _, Z = lib.nmf_dual_pass(ctx, Xv, U=cu(U))
    X64 = big[:, :301].astype(np.float64)
    assert rel(host(Y), X64 @ V) <= 1e-5
    assert rel(host(Z), X64.T @ U) <= 1e-5


@pytest.mark.parametrize("m,n,ell", [(512, 256, 18), (1000, 777, 40), (257, 1025, 70),
                                     (1000, 784, 40), (300, 1032, 70), (129, 136, 18),
                                     (2000, 520, 128), (5000, 3000, 40), (64, 8, 1),
                                     (3000, 4096, 100)])
def test_dual_pass_bf16(lib, ctx, m, n, ell):
    """BF16 X: n a multiple of 8 goes to the tcgen05/TMA kernel, which also rounds V and U to
    BF16 (one BF16 operand each, as in the sketch passes); other n to the SIMT kernel, which
    keeps V and U in FP32. Each is held to its own reference."""
    rng = np.random.default_rng(11 + m)
    X = rng.uniform(0, 1, (m, n)).astype(np.float32)
    V = rng.standard_normal((n, ell)).astype(np.float32)
    U = rng.standard_normal((m, ell)).astype(np.float32)
    Xq = lib.nmf_quantize(ctx, cu(X))
    Y, Z = lib.nmf_dual_pass(ctx, Xq, cu(V), cu(U), prec="bf16")
    Xb = bf16_round(X).astype(np.float64)
    if n % 8 == 0:
        Vb, Ub = bf16_round(V).astype(np.float64), bf16_round(U).astype(np.float64)
    else:
        Vb, Ub = V.astype(np.float64), U.astype(np.float64)
    assert rel(host(Y), Xb @ Vb) <= 1e-5
    assert rel(host(Z), Xb.T @ Ub) <= 1e-5


# ------------------------------------------------------------------ QR (Section 3)

@pytest.mark.parametrize("rows,ell", [(500, 18), (20000, 40), (1000, 1), (130, 128), (77, 70)])
def test_qr_matches_oracle(lib, ctx, rows, ell):
    rng = np.random.default_rng(rows + ell)
    # columns with a spread of scales: condition number ~ 1e3
    Y = (rng.standard_normal((rows, ell)) * np.logspace(0, -3, ell)).astype(np.float32)
    Q = host(lib.nmf_qr(ctx, cu(Y)))
    lib.nmf_sync(ctx)
    Qo = O.qr_orthonormal(Y.astype(np.float64))
    assert np.abs(Q.T @ Q - np.eye(ell)).max() <= 1e-5
    assert rel(Q, Qo) <= 1e-5


def test_qr_at_condition_1e6_matches_oracle_where_fp32_cholesky_qr2_fails(lib, ctx):
    """Singular values spread over six decades (condition ~1e6): the Gram matrix's condition
    (~1e12) is beyond FP32 (2^-24 ~ 6e-8), so CholeskyQR2 with FP32 Grams loses orthogonality
    or breaks down, while the float-float Gram, factor and first application (about 48
    significant bits) give the unique Q to FP32 accuracy. The FP32 variant is formed here in
    numpy float32 to show that the case does separate the two."""
    rng = np.random.default_rng(77)
    rows, ell = 20000, 40
    U, _ = np.linalg.qr(rng.standard_normal((rows, ell)))
    V, _ = np.linalg.qr(rng.standard_normal((ell, ell)))
    Y = ((U * np.logspace(0, -6, ell)) @ V.T).astype(np.float32)
    assert np.linalg.cond(Y.astype(np.float64)) > 5e5
    Q = host(lib.nmf_qr(ctx, cu(Y)))
    lib.nmf_sync(ctx)
    Qo = O.qr_orthonormal(Y.astype(np.float64))
    assert np.abs(Q.T @ Q - np.eye(ell)).max() <= 1e-5
    assert rel(Q, Qo) <= 1e-5

    def chol_qr_fp32(A):
        G = (A.T @ A).astype(np.float32)
        R = np.linalg.cholesky(G).T.astype(np.float32)
        return np.linalg.solve(R.T, A.T).T.astype(np.float32)

    try:
        Q32 = chol_qr_fp32(chol_qr_fp32(Y))
        fp32_err = float(np.abs(Q32.T.astype(np.float64) @ Q32 - np.eye(ell)).max())
        fp32_err = fp32_err if np.isfinite(fp32_err) else np.inf
    except np.linalg.LinAlgError:
        fp32_err = np.inf
    assert fp32_err > 1e-3


def test_qr_breakdown_is_reported(lib, ctx):
    Y = np.random.default_rng(0).standard_normal((100, 8)).astype(np.float32)
    Y[:, 3] = 0.0
    lib.nmf_qr(ctx, cu(Y))
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_sync(ctx)
    assert e.value.status == 4
    lib.nmf_sync(ctx)   # status cleared after being reported


def exact_rank_problem(seed, m, n, r, ell):
    """X = W0 H0 exactly (no noise, Exp(1) factors): rank r < ell, so every pass output of the
    sketch is numerically rank deficient."""
    rng = np.random.default_rng(seed)
    W0 = rng.exponential(1.0, (m, r))
    H0 = rng.exponential(1.0, (r, n))
    X = (W0 @ H0).astype(np.float32)
    return X, rng.standard_normal((n, ell)), rng.standard_normal((m, ell))


def test_sketch_of_exact_low_rank_x_breaks_down_without_repair(lib, ctx):
    """The SIMT pass keeps FP32 products (null directions of the pass output at ~1e-7 relative),
    so CholeskyQR2 meets the dependent columns and reports the breakdown."""
    X, oL, oR = exact_rank_problem(3, 600, 400, 5, 12)
    p = lib.params(600, 400, 5, 12, power_iters=2, flags=lib.FLAG_SIMT_DUAL_PASS)
    lib.nmf_sketch(ctx, p, cu(X), cu(oL), cu(oR))
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_sync(ctx)
    assert e.value.status == 4


def test_tensor_core_sketch_of_exact_low_rank_x_spans_x(lib, ctx):
    """The FP32 tensor-core pass (hi + lo BF16 splits) leaves noise of ~4e-6 relative in the
    null directions, above CholeskyQR2's pivot tolerance: the extra columns come out as
    orthonormal noise directions (what the repair would draw) and the bases still capture X."""
    m, n, r, ell = 600, 400, 5, 12
    X, oL, oR = exact_rank_problem(3, m, n, r, ell)
    p = lib.params(m, n, r, ell, power_iters=2)
    QL, QR = lib.nmf_sketch(ctx, p, cu(X), cu(oL), cu(oR))
    lib.nmf_sync(ctx)
    QL, QR, X64 = host(QL), host(QR), X.astype(np.float64)
    assert np.abs(QL.T @ QL - np.eye(ell)).max() <= 1e-5
    assert np.abs(QR.T @ QR - np.eye(ell)).max() <= 1e-5
    assert rel(QL @ (QL.T @ X64), X64) <= 1e-5 and rel(X64 @ QR @ QR.T, X64) <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_robust_sketch_repairs_rank_deficient_passes(lib, ctx, prec):
    """With NMF_FLAG_ROBUST_QR the dependent columns of each pass output are replaced by Gaussian
    draws and CholeskyQR2 repeated: Q_L, Q_R orthonormal, and (closed form for exact rank
    r <= ell) the projections reproduce X: Q_L Q_L^T X = X = X Q_R Q_R^T."""
    m, n, r, ell = 600, 400, 5, 12
    X, oL, oR = exact_rank_problem(3, m, n, r, ell)
    p = lib.params(m, n, r, ell, power_iters=2, prec=prec, flags=lib.FLAG_ROBUST_QR)
    Xd = cu(X)
    Xp = lib.nmf_quantize(ctx, Xd) if prec == "bf16" else Xd
    QL, QR = lib.nmf_sketch(ctx, p, Xp, cu(oL), cu(oR))
    lib.nmf_sync(ctx)
    QL, QR, Xh = host(QL), host(QR), X.astype(np.float64)
    assert np.abs(QL.T @ QL - np.eye(ell)).max() <= 1e-5
    assert np.abs(QR.T @ QR - np.eye(ell)).max() <= 1e-5
    tol = 1e-5 if prec == "fp32" else 2e-2      # BF16: the rounding of X moves its range
    assert rel(QL @ (QL.T @ Xh), Xh) <= tol
    assert rel((Xh @ QR) @ QR.T, Xh) <= tol


def test_solve_reruns_with_repaired_qr(lib, ctx):
    """nmf_solve on an exactly low-rank X: the first run meets the breakdown, the library
    restores the given factors and runs again with the repairing QR; the result is the solve of
    the rank-r problem (finite, non-negative, error far below the start's)."""
    m, n, r, ell = 600, 400, 5, 12
    X, _, _ = exact_rank_problem(4, m, n, r, ell)
    rng = np.random.default_rng(5)
    W0, H0 = rng.random((m, r)), rng.random((r, n))
    e0 = O.residual(X.astype(np.float64), W0, H0)[0]
    p = lib.params(m, n, r, ell, power_iters=2, iters=200, seed=8)
    W, H = cu(W0), cu(H0)
    e, it = lib.nmf_solve(ctx, p, cu(X), W, H)
    assert it == 200 and np.isfinite(e)
    assert (W >= 0).all() and (H >= 0).all()
    assert e <= 0.05 * e0
    # the solve's exact checks rebuild W H on the tensor cores: the same kernel through
    # nmf_residual gives the same value (the FP32 SIMT rebuild differs by ~5e-6 relative at a
    # residual this small, both being FP32-grade evaluations)
    ptc = lib.params(m, n, r, ell, flags=lib.FLAG_TC_RESIDUAL)
    assert abs(lib.nmf_residual(ctx, ptc, cu(X), W, H)[0] - e) <= 1e-6 * max(e, 1e-12)
    assert abs(lib.nmf_residual(ctx, p, cu(X), W, H)[0] - e) <= 3e-5 * max(e, 1e-12)


# ------------------------------------------------------------------ sketch and compression

def proj_diff(QL, QLo, X):
    X = X.astype(np.float64)
    return rel(QL @ (QL.T @ X), QLo @ (QLo.T @ X))


@pytest.mark.parametrize("seed,m,n,r,ell,w", [(0, 512, 256, 8, 18, 2), (1, 700, 450, 5, 12, 0),
                                              (2, 1000, 3001, 20, 40, 2), (3, 300, 300, 10, 20, 3)])
def test_sketch_fp32(lib, ctx, seed, m, n, r, ell, w):
    pr = inputs.random_problem(seed, m, n, r, ell, w=w)
    p = lib.params(m, n, r, ell, power_iters=w)
    QL, QR = lib.nmf_sketch(ctx, p, cu(pr.X), cu(pr.omega_L), cu(pr.omega_R))
    lib.nmf_sync(ctx)
    QLo, QRo = O.sketch(pr.X, pr.omega_L, pr.omega_R, w)
    QL, QR = host(QL), host(QR)
    assert np.abs(QL.T @ QL - np.eye(ell)).max() <= 1e-5
    assert proj_diff(QL, QLo, pr.X) <= 1e-5
    assert proj_diff(QR, QRo, pr.X.T) <= 1e-5


def test_sketch_bf16_within_low_precision_tolerance(lib, ctx):
    pr = inputs.random_problem(4, 2000, 1500, 20, 40, w=2)
    p = lib.params(2000, 1500, 20, 40, power_iters=2, prec="bf16")
    X = cu(pr.X)
    Xq = lib.nmf_quantize(ctx, X)
    QL, QR = lib.nmf_sketch(ctx, p, Xq, cu(pr.omega_L), cu(pr.omega_R))
    Xhat, Xchk = lib.nmf_compress(ctx, p, Xq, QL, QR)
    lib.nmf_sync(ctx)
    QLo, QRo = O.sketch(pr.X, pr.omega_L, pr.omega_R, 2)
    Xhat_o, _ = O.compress(pr.X, QLo, QRo)
    # basis-free form of "Q_L^T X within 2e-2": the projected data Q_L X_hat
    assert rel(host(QL) @ host(Xhat), QLo @ Xhat_o) <= 2e-2


@pytest.mark.parametrize("seed,m,n,r,ell", [(0, 512, 256, 8, 18), (5, 1001, 333, 4, 9)])
def test_compress_fp32(lib, ctx, seed, m, n, r, ell):
    pr = inputs.random_problem(seed, m, n, r, ell)
    QLo, QRo = O.sketch(pr.X, pr.omega_L, pr.omega_R, 1)
    QL32, QR32 = QLo.astype(np.float32), QRo.astype(np.float32)
    p = lib.params(m, n, r, ell, power_iters=1)
    Xhat, Xchk = lib.nmf_compress(ctx, p, cu(pr.X), cu(QL32), cu(QR32))
    Xh_o, Xc_o = O.compress(pr.X, QL32, QR32)
    assert rel(host(Xhat), Xh_o) <= 1e-5
    assert rel(host(Xchk), Xc_o) <= 1e-5


# ------------------------------------------------------------------ iterations (Section 4, 3.1)

def compressed_state(seed, m, n, r, ell, w=2):
    pr = inputs.random_problem(seed, m, n, r, ell, w=w)
    QL, QR = O.sketch(pr.X, pr.omega_L, pr.omega_R, w)
    QL, QR = QL.astype(np.float32), QR.astype(np.float32)
    Xhat, Xchk = O.compress(pr.X, QL, QR)
    return pr, QL, QR, Xhat.astype(np.float32), Xchk.astype(np.float32)


# r = 50 and 64 run on the per-stage kernels (above the persistent kernel's 48), the rest on
# the persistent kernel
ITER_CASES = [(0, 512, 256, 8, 18), (1, 1000, 777, 20, 40), (2, 333, 1201, 1, 6),
              (3, 600, 500, 40, 50), (4, 257, 129, 16, 16), (5, 400, 300, 33, 40),
              (7, 700, 901, 50, 70), (8, 300, 403, 64, 64)]


def fp32_model_step(W, H, QL, QR, Xhat, Xchk):
    """Error model, not the oracle: one FastHALS-RP step evaluated in numpy float32 (library
    order, every operation rounded to FP32). Its distance to the FP64 oracle is the error that
    FP32 arithmetic itself commits on these inputs."""
    t = np.float32
    W = W.astype(t).copy()
    H = H.astype(t).copy()
    Ht = H @ QR.astype(t)
    G = Ht @ Ht.T
    S = Xchk.astype(t) @ Ht.T
    for j in range(W.shape[1]):
        if G[j, j] > 0:
            W[:, j] = np.maximum(0, W[:, j] + (S[:, j] - W @ G[:, j]) / G[j, j])
    s = np.sqrt((W * W).sum(0))
    W /= np.where(s > 0, s, 1)
    H *= np.where(s > 0, s, 1)[:, None]
    Wt = QL.astype(t).T @ W
    Gh = Wt.T @ Wt
    P = Wt.T @ Xhat.astype(t)
    for j in range(H.shape[0]):
        if Gh[j, j] > 0:
            H[j] = np.maximum(0, H[j] + (P[j] - Gh[j] @ H) / Gh[j, j])
    return W, H


def fp32_model_mu_step(W, H, QL, QR, Xhat, Xchk, eps=O.EPS_MU):
    """Error model of one MU-RP step, as fp32_model_step (numpy float32, every operation
    rounded to FP32)."""
    t = np.float32
    W = W.astype(t)
    H = H.astype(t)
    pos = lambda a: np.maximum(a, t(0))
    neg = lambda a: np.maximum(-a, t(0))
    Ht = H @ QR.astype(t)
    G = Ht @ Ht.T
    S = Xchk.astype(t) @ Ht.T
    W = W * np.sqrt((pos(S) + W @ neg(G)) / (neg(S) + W @ pos(G) + t(eps)))
    Wt = QL.astype(t).T @ W
    Gh = Wt.T @ Wt
    P = Wt.T @ Xhat.astype(t)
    H = H * np.sqrt((pos(P) + neg(Gh) @ H) / (neg(P) + pos(Gh) @ H + t(eps)))
    return W, H


@pytest.mark.parametrize("rule", ["fasthals", "mu"])
@pytest.mark.parametrize("seed,m,n,r,ell", ITER_CASES)
def test_one_iteration_matches_oracle(lib, ctx, rule, seed, m, n, r, ell):
    """One GPU iteration from the oracle's own state, compared with one oracle iteration, from
    the U[0,1) start and from states of the oracle's trajectory (after 1 and 6 iterations).

    W, H and W H must each agree within max(1e-5, twice the distance of an FP32 evaluation of
    the same step to the oracle): the error FP32 arithmetic itself commits on these inputs. At
    small r that is 1e-5 throughout except for W from the random start (the first FastHALS-RP
    step nearly annihilates some columns of W and their normalisation to unit length magnifies
    FP32 rounding in them); at r = 50 and 64 the FP32 error alone reaches 1.2e-5 to 1.5e-5 for
    W and 1e-5 for H."""
    pr, QL, QR, Xhat, Xchk = compressed_state(seed, m, n, r, ell)
    step = O.fasthals_rp_step if rule == "fasthals" else O.mu_rp_step
    model = fp32_model_step if rule == "fasthals" else fp32_model_mu_step
    W0, H0 = pr.W0, pr.H0
    for k, advance in enumerate((1, 5, 0)):
        p = lib.params(m, n, r, ell, rule=rule)
        W, H = cu(W0), cu(H0)
        lib.nmf_iterate(ctx, p, cu(QL), cu(QR), cu(Xhat), cu(Xchk), W, H, 1)
        Wo, Ho = step(W0, H0, QL, QR, Xhat, Xchk)
        Wm, Hm = model(W0, H0, QL, QR, Xhat, Xchk)
        Wg, Hg = host(W), host(H)
        assert (Wg >= 0).all() and (Hg >= 0).all()
        for name, g, o, mdl in (("H", Hg, Ho, Hm), ("W", Wg, Wo, Wm),
                                ("WH", Wg @ Hg, Wo @ Ho, Wm @ Hm)):
            bound = max(1e-5, 2.0 * rel(mdl, o))
            assert rel(g, o) <= bound, f"{name}, state {k} (bound {bound:.2e})"
        if advance:
            W0, H0 = O.iterate(W0, H0, QL, QR, Xhat, Xchk, advance, rule=rule)
            W0, H0 = W0.astype(np.float32), H0.astype(np.float32)


def test_regularised_iteration_matches_oracle(lib, ctx):
    pr, QL, QR, Xhat, Xchk = compressed_state(6, 500, 400, 10, 20)
    p = lib.params(500, 400, 10, 20, alpha=0.05, beta=0.2)
    W, H = cu(pr.W0), cu(pr.H0)
    lib.nmf_iterate(ctx, p, cu(QL), cu(QR), cu(Xhat), cu(Xchk), W, H, 1)
    Wo, Ho = O.fasthals_rp_step(pr.W0, pr.H0, QL, QR, Xhat, Xchk, alpha=0.05, beta=0.2)
    assert rel(host(W), Wo) <= 1e-5 and rel(host(H), Ho) <= 1e-5


# ------------------------------------------------------------------ residual (Eq. 2.2)

@pytest.mark.parametrize("m,n,r", [(512, 256, 8), (1001, 777, 20), (64, 129, 1), (300, 200, 64)])
def test_residual_matches_oracle(lib, ctx, m, n, r):
    rng = np.random.default_rng(m + r)
    W = rng.uniform(0, 1, (m, r)).astype(np.float32)
    H = rng.uniform(0, 1, (r, n)).astype(np.float32)
    X = (W.astype(np.float64) @ H * (1 + 0.05 * rng.standard_normal((m, n)))).astype(np.float32)
    p = lib.params(m, n, r, min(r, m, n))
    relg, e2, x2 = lib.nmf_residual(ctx, p, cu(X), cu(W), cu(H))
    relo, e2o, x2o = O.residual(X, W, H)
    assert abs(x2 - x2o) <= 1e-6 * x2o
    assert abs(e2 - e2o) <= 1e-4 * e2o
    assert abs(relg - relo) <= 1e-4 * relo


@pytest.mark.parametrize("m,n,r", [(1000, 700, 20), (20000, 5000, 20), (333, 517, 1), (900, 1300, 16),
                                   (2049, 131, 17), (640, 1024, 32)])
def test_tensor_core_residual_matches_oracle(lib, ctx, m, n, r):
    """The residual with the W H rebuild on the tensor cores (BF16 hi + lo splits, three products):
    every product within about 2^-17 of FP32, so at a residual of 5 % (and 1 % for the dense
    workload's shape) the squared error agrees with the oracle to 1e-5 relative and ||X||^2 (FP32
    sums of 128 squares a tile, float-float across tiles, FP64 across blocks) to 1e-7; ragged
    tiles (m, n not multiples of 128) and r = 1, 16, 17, 32 (one or two K steps) included."""
    rng = np.random.default_rng(m + 3 * r)
    W = rng.uniform(0, 1, (m, r)).astype(np.float32)
    H = rng.uniform(0, 1, (r, n)).astype(np.float32)
    noise = 0.01 if (m, n) == (20000, 5000) else 0.05
    X = (W.astype(np.float64) @ H * (1 + noise * rng.standard_normal((m, n)))).astype(np.float32)
    p = lib.params(m, n, r, min(r, m, n), flags=lib.FLAG_TC_RESIDUAL)
    relg, e2, x2 = lib.nmf_residual(ctx, p, cu(X), cu(W), cu(H))
    relo, e2o, x2o = O.residual(X, W, H)
    print(f"tc residual {m}x{n} r={r}: e2 {e2 / e2o - 1:+.2e}, x2 {x2 / x2o - 1:+.2e}")
    assert abs(x2 - x2o) <= 1e-7 * x2o
    assert abs(e2 - e2o) <= 1e-5 * e2o
    assert abs(relg - relo) <= 1e-5 * relo


# ------------------------------------------------------------------ whole runs

def test_planted_small_mu_rp_200_iterations(lib, ctx):
    """512 x 256, r = 8, l = 18, w = 2, 200 MU-RP iterations from U[0,1) factors."""
    pr = inputs.planted_small(seed=0)
    m, n = pr.X.shape
    p = lib.params(m, n, pr.r, pr.ell, power_iters=pr.w, rule="mu")
    X = cu(pr.X)
    QL, QR = lib.nmf_sketch(ctx, p, X, cu(pr.omega_L), cu(pr.omega_R))
    Xhat, Xchk = lib.nmf_compress(ctx, p, X, QL, QR)
    W, H = cu(pr.W0), cu(pr.H0)
    lib.nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, W, H, 200)
    relg, _, _ = lib.nmf_residual(ctx, p, X, W, H)
    _, _, _, _, hist = O.solve(pr.X, pr.omega_L, pr.omega_R, pr.W0, pr.H0, pr.w, 200, rule="mu")
    relo = hist[-1][1]
    print(f"planted_small MU-RP: gpu {relg:.6g} oracle {relo:.6g}")
    assert abs(relg - relo) <= 0.01 * relo


def test_solve_matches_stepwise_path(lib, ctx):
    pr = inputs.random_problem(9, 800, 600, 10, 20)
    p = lib.params(800, 600, 10, 20, power_iters=2, iters=60, residual_every=20, seed=5)
    X = cu(pr.X)
    W, H = cu(pr.W0), cu(pr.H0)
    relg, it = lib.nmf_solve(ctx, p, X, W, H)
    assert it == 60
    # Omega from the oracle's own generator (same definition as the library's, seed 5)
    oL = O.philox_normal_np(600, 20, 5, 0)
    oR = O.philox_normal_np(800, 20, 5, 1)
    _, _, _, _, hist = O.solve(pr.X, oL, oR, pr.W0, pr.H0, 2, 60)
    assert abs(relg - hist[-1][1]) <= 0.01 * hist[-1][1]


def test_solve_stops_at_target(lib, ctx):
    pr = inputs.random_problem(10, 600, 500, 8, 16)
    p = lib.params(600, 500, 8, 16, iters=400, residual_every=10, target_rel_err=0.5, seed=1)
    relg, it = lib.nmf_solve(ctx, p, cu(pr.X), cu(pr.W0), cu(pr.H0))
    assert relg <= 0.5 and it < 400 and it % 10 == 0


def test_solve_budget_not_a_multiple_of_the_check_interval(lib, ctx):
    """25 iterations with a check every 10 and no target: the persistent kernel stops for the
    checks at 10 and 20 and for the forced one at the end of the budget (25), resuming from the
    count it left on the device; every check is exact (no target), the reported iterations are
    the budget, and W, H are the factors that last check measured. The same run as one launch
    (a single check at the end) lands on the same error up to the FP32 rounding that the
    relaunches reorder."""
    pr = inputs.random_problem(12, 700, 500, 6, 14)
    X = cu(pr.X)
    p = lib.params(700, 500, 6, 14, power_iters=2, iters=25, residual_every=10, seed=2)
    W, H = cu(pr.W0), cu(pr.H0)
    e, it = lib.nmf_solve(ctx, p, X, W, H)
    its, checks = lib.nmf_last_solve_info(ctx)
    assert it == 25 and its == 25 and checks == 3
    assert abs(lib.nmf_residual(ctx, p, X, W, H)[0] - e) <= 1e-6 * e
    p1 = lib.params(700, 500, 6, 14, power_iters=2, iters=25, residual_every=0, seed=2)
    W1, H1 = cu(pr.W0), cu(pr.H0)
    e1, it1 = lib.nmf_solve(ctx, p1, X, W1, H1)
    assert it1 == 25 and lib.nmf_last_solve_info(ctx)[1] == 1
    assert abs(e - e1) <= 1e-3 * e1


def test_invalid_arguments_are_rejected(lib, ctx):
    X = torch.zeros((10, 10), device=DEV)
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_sketch(ctx, lib.params(10, 10, 5, 11), X)      # ell > min(m, n)
    assert e.value.status == 1
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_sketch(ctx, lib.params(10, 10, 6, 5), X)       # r > ell
    assert e.value.status == 1
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_qr(ctx, torch.zeros((3, 5), device=DEV))      # rows < ell
    assert e.value.status == 1


def test_degenerate_square_full_width(lib, ctx):
    """l = m = n: the sketch spans everything and the compressed iteration is full FastHALS."""
    pr = inputs.random_problem(11, 48, 48, 4, 48, w=1)
    p = lib.params(48, 48, 4, 48, power_iters=1)
    X = cu(pr.X)
    QL, QR = lib.nmf_sketch(ctx, p, X, cu(pr.omega_L), cu(pr.omega_R))
    Xhat, Xchk = lib.nmf_compress(ctx, p, X, QL, QR)
    W, H = cu(pr.W0), cu(pr.H0)
    lib.nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, W, H, 3)
    Wo, Ho = pr.W0.astype(np.float64), pr.H0.astype(np.float64)
    for _ in range(3):
        Wo, Ho = O.fasthals_step(Wo, Ho, pr.X)
    assert rel(host(W) @ host(H), Wo @ Ho) <= 1e-4


@pytest.mark.parametrize("rule", ["fasthals", "mu"])
@pytest.mark.parametrize("seed,m,n,r,ell", [(0, 512, 256, 8, 18), (1, 3000, 1777, 20, 40),
                                            (2, 100, 5001, 32, 48), (3, 600, 500, 40, 50)])
def test_persistent_and_staged_iterations_agree(lib, ctx, rule, seed, m, n, r, ell):
    """The one-launch persistent kernel and the one-launch-per-stage kernels run the same
    arithmetic (they differ only in the order of cross-block sums): 30 iterations agree, and
    both stay within 1% of the oracle's relative error."""
    pr, QL, QR, Xhat, Xchk = compressed_state(seed, m, n, r, ell)
    outs = []
    for flags in (0, lib.FLAG_STAGED_ITERATE):
        p = lib.params(m, n, r, ell, rule=rule, flags=flags)
        W, H = cu(pr.W0), cu(pr.H0)
        lib.nmf_iterate(ctx, p, cu(QL), cu(QR), cu(Xhat), cu(Xchk), W, H, 30)
        lib.nmf_sync(ctx)
        outs.append((host(W), host(H)))
    (Wp, Hp), (Ws, Hs) = outs
    assert rel(Wp @ Hp, Ws @ Hs) <= 1e-4
    Wo, Ho = O.iterate(pr.W0, pr.H0, QL, QR, Xhat, Xchk, 30, rule=rule)
    ro = O.residual(pr.X, Wo, Ho)[0]
    for Wg, Hg in outs:
        assert abs(O.residual(pr.X, Wg, Hg)[0] - ro) <= 0.01 * ro


def test_iterate_zero_iterations_is_identity(lib, ctx):
    pr, QL, QR, Xhat, Xchk = compressed_state(3, 300, 200, 5, 10)
    p = lib.params(300, 200, 5, 10)
    W, H = cu(pr.W0), cu(pr.H0)
    lib.nmf_iterate(ctx, p, cu(QL), cu(QR), cu(Xhat), cu(Xchk), W, H, 0)
    assert np.array_equal(host(W), pr.W0) and np.array_equal(host(H), pr.H0)


def test_bf16_sketch_tensor_core_and_simt_agree(lib, ctx):
    """The tcgen05 pass rounds V, U to BF16, the SIMT pass keeps them FP32; both sketches of the
    same BF16 X agree within the low-precision tolerance and span the same subspace as the FP64
    oracle's on the exact X to within 2e-2 in projected data."""
    pr = inputs.random_problem(12, 3000, 2048, 20, 40, w=2)
    X = cu(pr.X)
    Xq = lib.nmf_quantize(ctx, X)
    outs = []
    for flags in (0, lib.FLAG_SIMT_DUAL_PASS):
        p = lib.params(3000, 2048, 20, 40, power_iters=2, prec="bf16", flags=flags)
        QL, QR = lib.nmf_sketch(ctx, p, Xq, cu(pr.omega_L), cu(pr.omega_R))
        Xhat, Xchk = lib.nmf_compress(ctx, p, Xq, QL, QR)
        lib.nmf_sync(ctx)
        outs.append((host(QL), host(Xhat)))
    (QLt, Xht), (QLs, Xhs) = outs
    QLo, QRo = O.sketch(pr.X, pr.omega_L, pr.omega_R, 2)
    Xho, _ = O.compress(pr.X, QLo, QRo)
    ref = QLo @ Xho
    assert rel(QLt @ Xht, ref) <= 2e-2
    assert rel(QLs @ Xhs, ref) <= 2e-2
    assert rel(QLt @ Xht, QLs @ Xhs) <= 2e-2


def test_solve_monitor_gates_exact_checks(lib, ctx):
    """With a target, the device-side loop runs the exact residual only when the compressed
    error monitor is within 5 % of the target (0.2 % once an exact check has calibrated it); the
    stopping iteration equals the one found by checking the exact residual at every check (the
    staged kernels, which never use the monitor)."""
    pr = inputs.random_problem(13, 2000, 1500, 10, 20, w=2)
    X = cu(pr.X)
    res = {}
    for flags in (0, lib.FLAG_STAGED_ITERATE):
        p = lib.params(2000, 1500, 10, 20, power_iters=2, iters=300, residual_every=10,
                       target_rel_err=0.0, seed=3, flags=flags)
        W, H = cu(pr.W0), cu(pr.H0)
        e_final, _ = lib.nmf_solve(ctx, p, X, W, H)
        target = 1.01 * e_final
        p = lib.params(2000, 1500, 10, 20, power_iters=2, iters=300, residual_every=10,
                       target_rel_err=target, seed=3, flags=flags)
        W, H = cu(pr.W0), cu(pr.H0)
        e, it = lib.nmf_solve(ctx, p, X, W, H)
        its, checks = lib.nmf_last_solve_info(ctx)
        assert e <= target and its == it
        assert abs(lib.nmf_residual(ctx, p, X, W, H)[0] - e) <= 1e-6 * e   # W, H match the check
        res[flags] = (it, checks)
    (it_mon, checks_mon), (it_all, checks_all) = res[0], res[lib.FLAG_STAGED_ITERATE]
    assert checks_all == it_all // 10
    assert checks_mon < checks_all
    assert abs(it_mon - it_all) <= 10


# ------------------------------------------------------------------ NNDSVD from compressed data

def designed_compressed(seed, m, n, ell, decay):
    """Q_L with orthonormal columns and X_hat = A diag(s) B^T with s_j = decay^j: a compressed
    pair whose singular values are known and separated."""
    rng = np.random.default_rng(seed)
    QL = np.linalg.qr(rng.standard_normal((m, ell)))[0]
    A = np.linalg.qr(rng.standard_normal((ell, ell)))[0]
    B = np.linalg.qr(rng.standard_normal((n, ell)))[0]
    s = decay ** np.arange(ell)
    return QL.astype(np.float32), ((A * s) @ B.T).astype(np.float32), s


@pytest.mark.parametrize("seed,m,n,r,ell,decay", [(0, 1001, 333, 4, 9, 0.7),
                                                  (1, 3000, 1200, 20, 40, 0.85),
                                                  (2, 256, 4100, 1, 16, 0.5)])
def test_nndsvd_matches_oracle(lib, ctx, seed, m, n, r, ell, decay):
    """Each column of W and row of H against the oracle's LAPACK-SVD NNDSVD on the same FP32
    inputs. The kernel's eigensolver runs in FP32, so component j carries the eigenvector error
    ell * eps32 * lambda_1 / gap_j with lambda = s^2 and gap_j the distance of lambda_j to its
    neighbours."""
    QL, Xhat, s = designed_compressed(seed, m, n, ell, decay)
    Wo, Ho = O.nndsvd_compressed(QL, Xhat, r)
    # precondition: no component is close to a tie between its two sign parts
    U1, _, Vt = np.linalg.svd(Xhat.astype(np.float64), full_matrices=False)
    U = QL.astype(np.float64) @ U1[:, :r]
    for j in range(1, r):
        x, y = U[:, j], Vt[j]
        mp = np.linalg.norm(np.maximum(x, 0)) * np.linalg.norm(np.maximum(y, 0))
        mn = np.linalg.norm(np.minimum(x, 0)) * np.linalg.norm(np.minimum(y, 0))
        assert abs(mp - mn) > 1e-3 * (mp + mn)
    p = lib.params(m, n, r, ell)
    W, H = lib.nmf_nndsvd(ctx, p, cu(QL), cu(Xhat))
    W, H = host(W), host(H)
    lam = s ** 2
    eps32 = 2.0 ** -24
    for j in range(r):
        gap = min(lam[j - 1] - lam[j] if j > 0 else np.inf, lam[j] - lam[j + 1])
        tol = 1e-5 + ell * eps32 * lam[0] / gap
        assert rel(W[:, j], Wo[:, j]) <= tol, (j, rel(W[:, j], Wo[:, j]), tol)
        assert rel(H[j], Ho[j]) <= tol, (j, rel(H[j], Ho[j]), tol)
    assert (W >= 0).all() and (H >= 0).all()


def test_nndsvd_rejects_rank_above_sketch(lib, ctx):
    QL, Xhat, _ = designed_compressed(0, 100, 80, 8, 0.5)
    with pytest.raises(lib.NmfError):
        lib.nmf_nndsvd(ctx, lib.params(100, 80, 9, 8), cu(QL), cu(Xhat))
