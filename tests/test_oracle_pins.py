"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it pins. None of them re-types the oracle's formula: they use closed
forms, invariants, special cases that reduce to a textbook method, brute force on tiny inputs and
values the paper prints.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s):
    return np.random.default_rng(1000 + s)


def _planted(rng, m, n, r, noise=0.0):
    W0 = rng.exponential(1.0, (m, r))
    H0 = rng.exponential(1.0, (r, n))
    X = W0 @ H0
    if noise:
        X = np.maximum(0.0, X + noise * X.std() * rng.standard_normal(X.shape))
    return X, W0, H0


# ---------------------------------------------------------------- QR (Section 3, Eq. 3.4-3.5)

def _mgs2(Y):
    """Modified Gram-Schmidt applied twice: an independent QR with positive R diagonal."""
    Q = np.array(Y, dtype=np.float64)
    for _ in range(2):
        for j in range(Q.shape[1]):
            for i in range(j):
                Q[:, j] -= (Q[:, i] @ Q[:, j]) * Q[:, i]
            Q[:, j] /= np.linalg.norm(Q[:, j])
    return Q


@pytest.mark.parametrize("shape", [(50, 8), (200, 18), (33, 33)])
def test_qr_orthonormal_and_reconstructs(shape):
    Y = _rng(0).standard_normal(shape)
    Q = O.qr_orthonormal(Y)
    assert np.abs(Q.T @ Q - np.eye(shape[1])).max() <= 1e-12
    R = Q.T @ Y
    assert np.abs(np.tril(R, -1)).max() <= 1e-12          # R upper triangular
    assert (np.diag(R) >= 0).all()                          # sign convention
    assert np.linalg.norm(Q @ R - Y) / np.linalg.norm(Y) <= 1e-13


def test_qr_unique_positive_diagonal_matches_gram_schmidt():
    Y = _rng(1).standard_normal((60, 10))
    assert np.abs(O.qr_orthonormal(Y) - _mgs2(Y)).max() <= 1e-12


# ---------------------------------------------------------------- sketch (Section 3, 3.1)

def test_power_product_singular_values_are_raised_to_2w_plus_1():
    """Section 3: sigma_j((X X^T)^w X) = sigma_j(X)^(2w+1). With Omega = I the oracle's
    literal Eq. 3.5 product must show exactly this spectrum."""
    X = _rng(2).uniform(0.0, 1.0, (30, 20)) / 3.0
    s = np.linalg.svd(X, compute_uv=False)
    for w in (0, 1, 2, 3):
        P = O.power_product(X, np.eye(20), w)
        sp = np.linalg.svd(P, compute_uv=False)
        # SVD is accurate to eps * sigma_1 in absolute terms
        np.testing.assert_allclose(sp, s ** (2 * w + 1), rtol=1e-10, atol=1e-14 * sp[0])


@pytest.mark.parametrize("w", [0, 1, 2, 3])
def test_sketch_captures_exact_low_rank(w):
    """Closed form: for X of exact rank r <= l, range(Q_L) contains range(X) and range(Q_R)
    contains range(X^T), so both projections reproduce X (Section 3.1: min(d,n) >> l > k)."""
    rng = _rng(3)
    X, _, _ = _planted(rng, 120, 90, 5)
    oL, oR = rng.standard_normal((90, 9)), rng.standard_normal((120, 9))
    QL, QR = O.sketch(X, oL, oR, w)
    assert QL.shape == (120, 9) and QR.shape == (90, 9)
    nx = np.linalg.norm(X)
    assert np.linalg.norm(QL @ (QL.T @ X) - X) / nx <= 1e-12
    assert np.linalg.norm((X @ QR) @ QR.T - X) / nx <= 1e-12


def test_sketch_span_equals_literal_power_product():
    """The re-orthonormalised chain spans the same subspace as Eq. 3.5's literal product
    (well-conditioned case, where the literal product keeps all directions)."""
    rng = _rng(4)
    X = rng.uniform(0.5, 1.0, (40, 30)) + 3.0 * np.eye(40, 30)
    oL, oR = rng.standard_normal((30, 6)), rng.standard_normal((40, 6))
    for w in (0, 1):
        QL, QR = O.sketch(X, oL, oR, w)
        PL = O.qr_orthonormal(O.power_product(X, oL, w))
        PR = O.qr_orthonormal(O.power_product(X.T, oR, w))
        assert np.abs(QL @ QL.T - PL @ PL.T).max() <= 1e-9
        assert np.abs(QR @ QR.T - PR @ PR.T).max() <= 1e-9


def test_sketch_right_chain_is_left_chain_of_transpose():
    """Section 3.1: R comes from P(X^T). A transposed operand in either chain breaks this."""
    rng = _rng(5)
    X = rng.uniform(0, 1, (70, 50))
    oL, oR = rng.standard_normal((50, 7)), rng.standard_normal((70, 7))
    QL, QR = O.sketch(X, oL, oR, 2)
    QL2, QR2 = O.sketch(X.T, oR, oL, 2)
    assert np.abs(QR - QL2).max() <= 1e-10
    assert np.abs(QL - QR2).max() <= 1e-10


def test_power_iterations_reduce_tail_error():
    """Section 3: power iterations sharpen the spectrum, so the projection error of a matrix
    with a slowly decaying spectrum does not grow with w (median over seeds)."""
    rng = _rng(6)
    U, _ = np.linalg.qr(rng.standard_normal((200, 60)))
    V, _ = np.linalg.qr(rng.standard_normal((150, 60)))
    X = (U * (np.arange(1, 61) ** -0.5)) @ V.T
    errs = {w: [] for w in (0, 1, 3)}
    for s in range(20):
        oL = np.random.default_rng(s).standard_normal((150, 12))
        oR = np.random.default_rng(100 + s).standard_normal((200, 12))
        for w in errs:
            QL, _ = O.sketch(X, oL, oR, w)
            errs[w].append(np.linalg.norm(X - QL @ (QL.T @ X)))
    med = {w: np.median(v) for w, v in errs.items()}
    assert med[3] <= med[1] <= med[0]
    # and never below the optimal rank-12 error (Eckart-Young)
    s = np.linalg.svd(X, compute_uv=False)
    assert med[3] >= np.sqrt(np.sum(s[12:] ** 2)) * (1 - 1e-12)


def test_compress_with_square_projections_is_lossless():
    """l = min(m, n) = m = n: Q_L, Q_R are orthogonal, so Q_L X_hat = X and X_chk Q_R^T = X."""
    rng = _rng(7)
    X = rng.uniform(0, 1, (16, 16))
    QL, QR = O.sketch(X, rng.standard_normal((16, 16)), rng.standard_normal((16, 16)), 1)
    Xhat, Xchk = O.compress(X, QL, QR)
    assert np.abs(QL @ Xhat - X).max() <= 1e-12
    assert np.abs(Xchk @ QR.T - X).max() <= 1e-12


# ---------------------------------------------------------------- FastHALS-RP (Section 4)

def _compressed(seed, m=40, n=30, r=4, ell=9, w=2, noise=0.05):
    rng = _rng(seed)
    X, _, _ = _planted(rng, m, n, r, noise)
    QL, QR = O.sketch(X, rng.standard_normal((n, ell)), rng.standard_normal((m, ell)), w)
    Xhat, Xchk = O.compress(X, QL, QR)
    W = rng.uniform(0, 1, (m, r))
    H = rng.uniform(0, 1, (r, n))
    return X, QL, QR, Xhat, Xchk, W, H


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fasthals_rp_equals_hals_rp_with_explicit_residuals(seed):
    """Eq. fastHALS_a is Eq. hals_update with Eq. 4.6 substituted: the two forms agree."""
    _, QL, QR, Xhat, Xchk, W, H = _compressed(seed)
    for _ in range(5):
        Wf, Hf = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk)
        Wh, Hh = O.hals_rp_step(W, H, QL, QR, Xhat, Xchk, order="block")
        assert np.abs(Wf - Wh).max() <= 1e-12 * max(1.0, np.abs(Wh).max())
        assert np.abs(Hf - Hh).max() <= 1e-11 * max(1.0, np.abs(Hh).max())
        W, H = Wf, Hf


def test_fasthals_rp_with_square_projections_is_fasthals():
    """l = m = n: the compressed problem is the full one; FastHALS-RP reduces to FastHALS,
    which in turn equals HALS (Algorithm 2, Eq. 2.2_3) with explicit component residuals."""
    rng = _rng(8)
    X, _, _ = _planted(rng, 14, 14, 3, 0.05)
    QL, QR = O.sketch(X, rng.standard_normal((14, 14)), rng.standard_normal((14, 14)), 1)
    Xhat, Xchk = O.compress(X, QL, QR)
    W, H = rng.uniform(0, 1, (14, 3)), rng.uniform(0, 1, (3, 14))
    for _ in range(5):
        Wc, Hc = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk)
        Wf, Hf = O.fasthals_step(W, H, X)
        assert np.abs(Wc - Wf).max() <= 1e-11 and np.abs(Hc - Hf).max() <= 1e-10
        # HALS with explicit X_j = X - A B^T + a_j b_j^T (identity projections)
        I = np.eye(14)
        Wh, Hh = O.hals_rp_step(W, H, I, I, X, X, order="block")
        assert np.abs(Wh - Wf).max() <= 1e-11 and np.abs(Hh - Hf).max() <= 1e-10
        W, H = Wf, Hf


def _golden_min(f, lo, hi, tol=1e-13):
    g = (np.sqrt(5) - 1) / 2
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    while b - a > tol * max(1.0, abs(b)):
        if f(c) < f(d):
            b, d = d, c
            c = b - g * (b - a)
        else:
            a, c = c, d
            d = a + g * (b - a)
    return 0.5 * (a + b)


def test_fasthals_rp_step_matches_brute_force_minimisers():
    """Algorithm 4 lines 3-4 define each update as the argmin over a_j >= 0 (b_j >= 0) of the
    compressed component cost. Solve every scalar sub-problem by golden-section search on the
    cost itself (no closed form), in block order with the compensated normalisation, and compare
    with one oracle step."""
    _, QL, QR, Xhat, Xchk, W, H = _compressed(3, m=12, n=10, r=3, ell=6)
    A, B = W.copy(), H.T.copy()
    R = QR.T
    k = A.shape[1]
    for j in range(k):
        Bc = R @ B
        Xc_j = Xchk - A @ Bc.T + np.outer(A[:, j], Bc[:, j])
        for i in range(A.shape[0]):
            f = lambda a: np.sum((Xc_j[i] - a * Bc[:, j]) ** 2)
            A[i, j] = _golden_min(f, 0.0, 50.0)
    s = np.linalg.norm(A, axis=0)
    A /= s
    B *= s
    for j in range(k):
        Ah = QL.T @ A
        Xh_j = Xhat - Ah @ B.T + np.outer(Ah[:, j], B[:, j])
        for c in range(B.shape[0]):
            f = lambda b: np.sum((Xh_j[:, c] - b * Ah[:, j]) ** 2)
            B[c, j] = _golden_min(f, 0.0, 200.0)
    Wo, Ho = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk)
    np.testing.assert_allclose(A, Wo, atol=1e-6)
    np.testing.assert_allclose(B.T, Ho, atol=1e-5)


def test_each_component_update_satisfies_kkt():
    """Eq. hals_a / hals_b: the update zeroes the gradient where the entry is positive and
    leaves it non-negative where the entry is clamped. In an interleaved Algorithm 4 sweep the
    last update (b_k) is an exact minimiser given everything else; the gradient is formed from
    the explicit residual of Eq. 4.6."""
    _, QL, QR, Xhat, Xchk, W, H = _compressed(4)
    for _ in range(3):
        A2, H2 = O.hals_rp_step(W, H, QL, QR, Xhat, Xchk, order="interleaved", normalize=False)
        B2 = H2.T
        jl = A2.shape[1] - 1
        Ah = QL.T @ A2
        Xh = Xhat - Ah @ B2.T + np.outer(Ah[:, jl], B2[:, jl])
        gb = B2[:, jl] * (Ah[:, jl] @ Ah[:, jl]) - Xh.T @ Ah[:, jl]      # Eq. hals_b
        pos = B2[:, jl] > 0
        scale = np.abs(Xh.T @ Ah[:, jl]).max()
        assert np.abs(gb[pos]).max(initial=0) <= 1e-11 * scale
        assert (gb[~pos] >= -1e-11 * scale).all()
        W, H = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk)
    # W half-step of a single component (r = 1) is an exact NNLS solve, Eq. hals_a
    _, QL, QR, Xhat, Xchk, W, H = _compressed(5, r=1)
    Wn, _ = O.hals_rp_step(W, H, QL, QR, Xhat, Xchk, order="block", normalize=False)
    bc = (H @ QR)[0]
    ga = Wn[:, 0] * (bc @ bc) - Xchk @ bc
    pos = Wn[:, 0] > 0
    sc = np.abs(Xchk @ bc).max()
    assert np.abs(ga[pos]).max(initial=0) <= 1e-11 * sc and (ga[~pos] >= -1e-11 * sc).all()


def test_normalisation_keeps_product_and_unit_columns():
    """Section 4 (after Eq. fastHALS_a): a_j <- a_j / ||a_j||. With the scale moved to b_j, the
    iteration is invariant: W H after one step is the same with or without normalisation, and
    the normalised W has unit columns."""
    _, QL, QR, Xhat, Xchk, W, H = _compressed(6)
    for _ in range(4):
        Wn, Hn = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk, normalize=True)
        Wu, Hu = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk, normalize=False)
        assert np.abs(Wn @ Hn - Wu @ Hu).max() <= 1e-11 * np.abs(Wu @ Hu).max()
        nz = np.linalg.norm(Wn, axis=0) > 0
        np.testing.assert_allclose(np.linalg.norm(Wn, axis=0)[nz], 1.0, atol=1e-14)
        W, H = Wn, Hn


def test_regularised_update_reduces_to_plain_and_sparsifies():
    """Section 4.1: alpha = beta = 0 is Eq. fastHALS_a; a large alpha zeroes H (the l1 term's
    soft threshold exceeds every correlation)."""
    _, QL, QR, Xhat, Xchk, W, H = _compressed(7)
    W1, H1 = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk)
    W2, H2 = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk, alpha=0.0, beta=0.0)
    assert np.array_equal(W1, W2) and np.array_equal(H1, H2)
    _, H3 = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk, alpha=1e6)
    assert np.all(H3 == 0.0)
    # the regularised b_j minimises 1/2||X_hat_j - a b^T||^2 + alpha|b|_1 + beta/2|b|^2 per entry
    alpha, beta = 0.3, 0.7
    _, QL, QR, Xhat, Xchk, W, H = _compressed(8, r=1)
    Wn, Hn = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk, alpha=alpha, beta=beta)
    ah = (QL.T @ Wn)[:, 0]
    for c in range(Xhat.shape[1]):
        f = lambda b: 0.5 * np.sum((Xhat[:, c] - b * ah) ** 2) + alpha * abs(b) + 0.5 * beta * b * b
        assert abs(_golden_min(f, 0.0, 100.0) - Hn[0, c]) <= 1e-6


def test_planted_exact_recovery():
    """North-star pin: X = W0 H0 exactly, separable W0 (an r x r identity block), recovered by
    FastHALS-RP to relative residual < 1e-8 from the best of a few random starts."""
    rng = _rng(9)
    m, n, r, ell = 40, 30, 3, 8
    W0 = rng.uniform(0.0, 1.0, (m, r))
    W0[:r] = 2.0 * np.eye(r)
    H0 = rng.uniform(0.0, 1.0, (r, n))
    H0[:, :r] += np.eye(r)
    X = W0 @ H0
    QL, QR = O.sketch(X, rng.standard_normal((n, ell)), rng.standard_normal((m, ell)), 2)
    Xhat, Xchk = O.compress(X, QL, QR)
    best = np.inf
    for s in range(5):
        g = np.random.default_rng(s)
        W, H = g.uniform(0, 1, (m, r)), g.uniform(0, 1, (r, n))
        for it in range(4000):
            W, H = O.fasthals_rp_step(W, H, QL, QR, Xhat, Xchk)
            if it % 200 == 199 and O.residual(X, W, H)[0] < 1e-9:
                break
        best = min(best, O.residual(X, W, H)[0])
        if best < 1e-8:
            break
    assert best < 1e-8
    assert (W >= 0).all() and (H >= 0).all()


# ---------------------------------------------------------------- MU, MU-RP (Sections 2.1, 3.1)

def test_lee_seung_mu_is_monotone():
    """Multiplicative updates on the full data never increase J (Lee & Seung 2001, cited in
    Section 2.1)."""
    rng = _rng(10)
    X, _, _ = _planted(rng, 30, 25, 4, 0.1)
    W, H = rng.uniform(0.1, 1, (30, 4)), rng.uniform(0.1, 1, (4, 25))
    J = O.objective(X, W, H)
    for _ in range(200):
        W, H = O.mu_step(W, H, X)
        Jn = O.objective(X, W, H)
        assert Jn <= J * (1 + 1e-12)
        J = Jn
    assert (W >= 0).all() and (H >= 0).all()


def test_mu_rp_half_steps_are_monotone_in_their_own_objectives():
    """Algorithm 3: line 2 minimises ||X R^T - A (R B)^T|| over A >= 0, line 3 minimises
    ||L^T X - (L^T A) B^T|| over B >= 0. The semi-NMF rule (Ding, Li & Jordan 2010) never
    increases the objective of the half-step it performs."""
    _, QL, QR, Xhat, Xchk, W, H = _compressed(11, m=60, n=50, r=5, ell=12)
    for _ in range(100):
        Ht = H @ QR
        jw0 = np.sum((Xchk - W @ Ht) ** 2)
        Wn, Hn = O.mu_rp_step(W, H, QL, QR, Xhat, Xchk)
        jw1 = np.sum((Xchk - Wn @ Ht) ** 2)
        assert jw1 <= jw0 * (1 + 1e-12)
        Wt = QL.T @ Wn
        jh0 = np.sum((Xhat - Wt @ H) ** 2)
        jh1 = np.sum((Xhat - Wt @ Hn) ** 2)
        assert jh1 <= jh0 * (1 + 1e-12)
        assert (Wn >= 0).all() and (Hn >= 0).all()
        W, H = Wn, Hn


def test_mu_rp_fixed_point_at_exact_factorisation():
    """At X = W0 H0 (exact, positive factors) both semi-NMF ratios are 1: one step moves
    neither factor."""
    rng = _rng(12)
    m, n, r, ell = 30, 20, 3, 8
    W0, H0 = rng.uniform(0.5, 1.5, (m, r)), rng.uniform(0.5, 1.5, (r, n))
    X = W0 @ H0
    QL, QR = O.sketch(X, rng.standard_normal((n, ell)), rng.standard_normal((m, ell)), 1)
    Xhat, Xchk = O.compress(X, QL, QR)
    W1, H1 = O.mu_rp_step(W0, H0, QL, QR, Xhat, Xchk)
    assert np.abs(W1 - W0).max() <= 1e-12 * 10 and np.abs(H1 - H0).max() <= 1e-12 * 10


# ---------------------------------------------------------------- residual, monitor, init, Gini

def test_residual_closed_form():
    """Eq. 2.2 on a constructed case: X = 2 * ones, W H = ones -> ||X - WH||^2 = m n,
    ||X||^2 = 4 m n, rel = 1/2, J = m n / 2."""
    m, n = 7, 5
    X = 2.0 * np.ones((m, n))
    W, H = np.ones((m, 1)), np.ones((1, n))
    rel, e2, x2 = O.residual(X, W, H)
    assert rel == 0.5 and e2 == m * n and x2 == 4 * m * n
    assert O.objective(X, W, H) == m * n / 2


def test_compressed_error_estimate_is_exact_with_square_projection():
    rng = _rng(13)
    X = rng.uniform(0, 1, (12, 12))
    QL, QR = O.sketch(X, rng.standard_normal((12, 12)), rng.standard_normal((12, 12)), 0)
    Xhat, _ = O.compress(X, QL, QR)
    W, H = rng.uniform(0, 1, (12, 3)), rng.uniform(0, 1, (3, 12))
    _, e2, x2 = O.residual(X, W, H)
    assert abs(O.compressed_sq_error(x2, QL, Xhat, W, H) - e2) <= 1e-10 * x2


def test_compressed_error_estimate_identity_for_any_projection():
    """For any orthonormal Q_L (P = Q_L Q_L^T) the compressed estimate is
    ||X||^2 - 2 <P X, W H> + ||W H||^2 = ||X - W H||^2 + 2 <(I - P) X, W H>: the cross term sees
    only the projected data. Checked against the exact residual of the full X and the
    complementary projector, with l well below the rank of X so that the correction is large."""
    rng = _rng(14)
    m, n, ell, r = 50, 30, 8, 4
    X = rng.uniform(0, 1, (m, n))
    QL, _ = np.linalg.qr(rng.standard_normal((m, ell)))
    Xhat = QL.T @ X
    W, H = rng.uniform(0, 1, (m, r)), rng.uniform(0, 1, (r, n))
    _, e2, x2 = O.residual(X, W, H)
    corr = 2.0 * float(np.sum((X - QL @ (QL.T @ X)) * (W @ H)))
    assert abs(corr) > 1e-3 * x2
    assert abs(O.compressed_sq_error(x2, QL, Xhat, W, H) - (e2 + corr)) <= 1e-10 * x2


def test_nndsvd_rank_one_and_nonnegative():
    """NNDSVD of a positive rank-1 matrix reproduces it with its first component."""
    rng = _rng(14)
    u, v = rng.uniform(0.5, 2, 25), rng.uniform(0.5, 2, 18)
    X = np.outer(u, v)
    QL, QR = O.sketch(X, rng.standard_normal((18, 6)), rng.standard_normal((25, 6)), 1)
    Xhat, _ = O.compress(X, QL, QR)
    W, H = O.nndsvd_compressed(QL, Xhat, 3)
    assert np.abs(np.outer(W[:, 0], H[0]) - X).max() <= 1e-10
    X2, _, _ = _planted(rng, 40, 30, 4, 0.1)
    QL, QR = O.sketch(X2, rng.standard_normal((30, 10)), rng.standard_normal((40, 10)), 2)
    Xhat, _ = O.compress(X2, QL, QR)
    W, H = O.nndsvd_compressed(QL, Xhat, 4)
    assert (W >= 0).all() and (H >= 0).all()
    assert O.residual(X2, W, H)[0] < 0.9


def test_nndsvd_block_diagonal_is_exact_for_every_component():
    """NNDSVD (Boutsidis & Gallopoulos 2008) on X = sum_k s_k a_k b_k^T with non-negative a_k, b_k
    on disjoint row and column blocks: the singular pairs are (a_k, b_k) up to a joint sign, each
    has one non-zero sign part, so every component j >= 1 must reproduce its block exactly and
    W H = X. The block scales are distinct so the singular values are simple."""
    rng = _rng(15)
    rows, cols = [9, 7, 11, 6, 8], [5, 8, 4, 7, 6]
    m, n, r = sum(rows), sum(cols), len(rows)
    X = np.zeros((m, n))
    i0 = c0 = 0
    for k in range(r):
        a = rng.uniform(0.2, 1.0, rows[k])
        b = rng.uniform(0.2, 1.0, cols[k])
        X[i0:i0 + rows[k], c0:c0 + cols[k]] = (5.0 - k) * np.outer(a, b) / (
            np.linalg.norm(a) * np.linalg.norm(b))
        i0 += rows[k]
        c0 += cols[k]
    X = X[rng.permutation(m)][:, rng.permutation(n)]
    ell = r + 3
    QL, QR = O.sketch(X, rng.standard_normal((n, ell)), rng.standard_normal((m, ell)), 1)
    Xhat, _ = O.compress(X, QL, QR)
    W, H = O.nndsvd_compressed(QL, Xhat, r)
    assert (W >= 0).all() and (H >= 0).all()
    assert np.abs(W @ H - X).max() <= 1e-12 * np.abs(X).max()
    # component j carries the block of singular value 5 - j (the j-th largest)
    for j in range(r):
        assert abs(np.linalg.norm(np.outer(W[:, j], H[j])) - (5.0 - j)) <= 1e-12


def test_nndsvd_component_is_dominant_quadrant_of_singular_pair():
    """Mixed signs. NNDSVD keeps, for each singular triplet (s_j, u_j, v_j) with j >= 1, the larger
    (in Frobenius norm) of the two non-negative quadrants of s_j u_j v_j^T: the part on rows with
    u > 0 and columns with v > 0, or the part on rows with u < 0 and columns with v < 0 (negated).
    The quadrants are cut from the m x n rank-1 matrix itself and the triplets come from an SVD
    of the full Q_L X_hat (not of X_hat); component 0 is s_0 |u_0| |v_0|^T."""
    rng = _rng(16)
    m, n, ell, r = 40, 30, 9, 6
    X = rng.uniform(0, 1, (m, n))
    QL, QR = O.sketch(X, rng.standard_normal((n, ell)), rng.standard_normal((m, ell)), 1)
    Xhat, _ = O.compress(X, QL, QR)
    W, H = O.nndsvd_compressed(QL, Xhat, r)
    U, s, Vt = np.linalg.svd(QL @ Xhat)
    both = 0
    for j in range(r):
        C = s[j] * np.outer(U[:, j], Vt[j])
        got = np.outer(W[:, j], H[j])
        if j == 0:
            want = s[0] * np.outer(np.abs(U[:, 0]), np.abs(Vt[0]))
        else:
            pp = np.where((U[:, j] > 0)[:, None] & (Vt[j] > 0)[None, :], C, 0.0)
            nn = np.where((U[:, j] < 0)[:, None] & (Vt[j] < 0)[None, :], C, 0.0)
            want = pp if np.linalg.norm(pp) >= np.linalg.norm(nn) else nn
            both += np.linalg.norm(pp) > 0 and np.linalg.norm(nn) > 0
        assert np.abs(got - want).max() <= 1e-10 * s[0]
    assert both >= r - 2  # the mixed-sign branch is exercised, not only one-signed pairs


def test_monitor_estimate_identity_with_square_projection():
    """With Q_L square (P = I) the monitor of a solve on a copy X_q of X is
    ||X||^2 - 2 <X_q, W H> - 2 <X - X_q, X> + ||W H||^2 = ||X - W H||^2 + 2 <X - X_q, W H - X>
    (expand both sides); it is exact at W H = X, and equals the compressed estimate for X_q = X."""
    rng = _rng(17)
    m, n, r = 14, 14, 3
    X = rng.uniform(0, 1, (m, n))
    Xq = X + 1e-2 * rng.standard_normal((m, n))
    QL, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Xhat = QL.T @ Xq
    W, H = rng.uniform(0, 1, (m, r)), rng.uniform(0, 1, (r, n))
    _, e2, x2 = O.residual(X, W, H)
    t = O.rounding_term(X, Xq)
    want = e2 + 2.0 * float(np.sum((X - Xq) * (W @ H - X)))
    assert abs(O.monitor_estimate(x2, QL, Xhat, W, H, t) - want) <= 1e-10 * x2
    Wx, Hx = X.copy(), np.eye(n)
    assert abs(O.monitor_estimate(x2, QL, Xhat, Wx, Hx, t)) <= 1e-10 * x2
    assert O.monitor_estimate(x2, QL, QL.T @ X, W, H, 0.0) == O.compressed_sq_error(
        x2, QL, QL.T @ X, W, H)


def test_rounding_term_closed_form():
    """<X - X_q, X> for a copy that moves every entry by the same fraction: X_q = (1 - d) X gives
    d ||X||^2; an exact copy gives 0."""
    X = np.arange(1.0, 13.0).reshape(3, 4)
    assert O.rounding_term(X, X) == 0.0
    assert abs(O.rounding_term(X, 0.75 * X) - 0.25 * float(np.sum(X * X))) <= 1e-12


def test_solve_to_target_stops_where_every_check_is_exact():
    """The estimate only skips exact residuals that cannot meet the target: the stop is the first
    check of `solve` (an exact residual at every check) whose error is at or below the target,
    with the same factors; a target no check meets runs all iterations."""
    rng = _rng(18)
    X, _, _ = _planted(rng, 60, 45, 4, 0.05)
    oL, oR = rng.standard_normal((45, 10)), rng.standard_normal((60, 10))
    W0, H0 = rng.uniform(0, 1, (60, 4)), rng.uniform(0, 1, (4, 45))
    _, _, _, _, hist = O.solve(X, oL, oR, W0, H0, 2, 200, residual_every=10)
    target = hist[6][1] * 1.0000001
    it_ref = next(i for i, e in hist if e <= target)
    W, H, it, rel, checks = O.solve_to_target(X, oL, oR, W0, H0, 2, 200, target)
    assert it == it_ref and rel <= target and checks < it // 10
    Wr, Hr, _, _, _ = O.solve(X, oL, oR, W0, H0, 2, it, residual_every=0)
    assert np.array_equal(W, Wr) and np.array_equal(H, Hr)
    _, _, it, rel, checks = O.solve_to_target(X, oL, oR, W0, H0, 2, 50, 1e-9)
    assert it == 50 and checks == 1 and rel == O.solve(X, oL, oR, W0, H0, 2, 50)[4][-1][1]


def test_spectrum_of_exact_rank_sketch_equals_singular_values():
    """For X of exact rank r <= l the sketch captures range(X), so X_hat = Q_L^T X has the nonzero
    singular values of X (Section 3, Eq. 3.4 holds with equality); the rest are zero."""
    rng = _rng(19)
    X, _, _ = _planted(rng, 60, 45, 5)
    QL, QR = O.sketch(X, rng.standard_normal((45, 9)), rng.standard_normal((60, 9)), 1)
    Xhat, _ = O.compress(X, QL, QR)
    s = O.spectrum(Xhat)
    want = np.linalg.svd(X, compute_uv=False)
    assert np.allclose(s[:5], want[:5], rtol=1e-12)
    assert np.all(np.abs(s[5:]) <= 1e-10 * s[0])


def test_decay_rate_recovers_exponential_spectrum():
    """sigma_j = C exp(-p j) is fitted exactly, for any C; entries below the floor are ignored."""
    j = np.arange(40)
    for p, C in ((0.0053, 7.0), (0.0012, 0.3), (0.25, 1e4)):
        s = C * np.exp(-p * j)
        assert abs(O.decay_rate(s, 0.0) - p) <= 1e-12 * max(1.0, p)
    s = np.exp(-0.1 * j)
    s[30:] = 1e-9                       # a noise floor the fit must skip
    assert abs(O.decay_rate(s, 1e-3) - 0.1) <= 1e-12


def test_gini_closed_forms():
    """Section 5.1 Gini formula: all-equal entries give 0, a single non-zero gives 1 - 1/N."""
    assert abs(O.gini(np.ones((4, 5)))) <= 1e-15
    B = np.zeros((4, 5))
    B[2, 3] = 7.0
    assert abs(O.gini(B) - (1 - 1 / 20)) <= 1e-15
    # half zeros, half equal values: the Lorenz-curve area gives exactly 1/2
    assert abs(O.gini(np.array([[0.0, 3.0], [3.0, 0.0]])) - 0.5) <= 1e-15
    # order of entries does not matter (the formula sorts)
    B = np.random.default_rng(0).exponential(1.0, (6, 7))
    assert O.gini(B) == O.gini(B.T[::-1])


def test_memory_formula_matches_printed_tables():
    """Section 4.2 Table 4.1 memory (2(r+r_ov)+k)(d+n) and (dn+dk+nk) against the values printed
    in Tables 5.2 and 5.3 (tests/golden/table_memory.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "table_memory.txt")) if l[0] != "#"]
    for d, n, k, ell, p_rp, p_full, unit in rows:
        d, n, k, ell = int(d), int(n), int(k), int(ell)
        unit = float(unit)
        # the tables print two significant digits, truncated (e.g. 172.8 -> 170, 53.6 -> 53)
        def two_sig(v):
            e = int(np.floor(np.log10(v)))
            return int(np.floor(v / 10.0 ** (e - 1)) * 10 ** (e - 1))
        assert two_sig(O.memory_floats_rp(d, n, k, ell) / unit) == int(p_rp)
        assert two_sig((d * n + d * k + n * k) / unit) == int(p_full)


# ---------------------------------------------------------------- generator for Omega

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt")) if l[0] != "#"]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        assert O.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_philox_normal_box_muller_pairs():
    """Box-Muller invariant: z0^2 + z1^2 = -2 ln u0 for the pair drawn from one Philox block;
    sample moments of a few thousand draws are those of N(0,1)."""
    Z = O.philox_normal(64, 40, seed=7, stream=1).ravel()
    x = O.philox4x32_10((0, 0, 1, 0), (7, 0))
    u0 = ((x[0] >> 8) + 0.5) * 2.0 ** -24
    assert abs(Z[0] ** 2 + Z[1] ** 2 + 2 * np.log(u0)) <= 1e-12
    assert abs(Z.mean()) < 0.06 and abs(Z.std() - 1) < 0.05


def test_philox_normal_np_equals_scalar_definition():
    """The array form of the generator gives the scalar definition's values element for element,
    including a seed above 2^32, a non-multiple-of-4 size and both streams."""
    for rows, cols, seed, stream in [(13, 7, (1 << 40) + 99, 1), (5, 3, 0, 0), (31, 9, 123, 5)]:
        a = O.philox_normal(rows, cols, seed=seed, stream=stream)
        b = O.philox_normal_np(rows, cols, seed=seed, stream=stream)
        assert np.array_equal(a, b)


# ---------------------------------------------------------------- learned warm start

from oracle import warmstart_oracle as WS  # noqa: E402


def test_bf16_round_exact_values():
    """Round to nearest, ties to even, at the 8-bit significand of bfloat16."""
    u = 2.0 ** -7    # spacing of bfloat16 in [1, 2)
    x = np.array([1.0, 1 + u / 2, 1 + 3 * u / 2, 1 + u / 4, 1 + 3 * u / 4, -3.0, 1 + u])
    want = np.array([1.0, 1.0, 1 + 2 * u, 1.0, 1 + u, -3.0, 1 + u])
    assert np.array_equal(WS.bf16_round(x), want)


def test_mlp_gradient_matches_finite_differences():
    """Every component of the gradient against a central difference of the loss (on the
    unrounded network, where the loss is smooth away from ReLU kinks)."""
    F, Hd, r, B = 5, 7, 3, 6
    rng = np.random.default_rng(0)
    p = rng.standard_normal(WS.mlp_param_count(F, Hd, r)) * 0.5
    X = rng.standard_normal((B, F))
    T = rng.standard_normal((B, r))
    _, g = WS.mlp_loss_grad(p, X, T, F, Hd, r, round_weights=False)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = WS.mlp_loss_grad(p + e, X, T, F, Hd, r, round_weights=False)
        lm, _ = WS.mlp_loss_grad(p - e, X, T, F, Hd, r, round_weights=False)
        fd[k] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_mlp_rounded_gradient_is_gradient_at_rounded_weights():
    F, Hd, r = 4, 6, 2
    rng = np.random.default_rng(1)
    p = rng.standard_normal(WS.mlp_param_count(F, Hd, r))
    X, T = rng.standard_normal((5, F)), rng.standard_normal((5, r))
    W1, b1, W2, b2, W3, b3 = WS.mlp_unpack(p, F, Hd, r)
    q = np.concatenate([WS.bf16_round(W1).ravel(), b1, WS.bf16_round(W2).ravel(), b2,
                        WS.bf16_round(W3).ravel(), b3])
    l1, g1 = WS.mlp_loss_grad(p, X, T, F, Hd, r)
    l2, g2 = WS.mlp_loss_grad(q, X, T, F, Hd, r, round_weights=False)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_adam_first_step_closed_form():
    """Step 1 of Adam moves every parameter by lr * g / (|g| + eps) (bias correction makes the
    moment estimates g and g^2)."""
    rng = np.random.default_rng(2)
    p, g = rng.standard_normal(9), rng.standard_normal(9)
    q, m, v = WS.adam_step(p, np.zeros(9), np.zeros(9), g, 1, 1e-3)
    assert np.allclose(q, p - 1e-3 * g / (np.abs(g) + WS.ADAM_EPS), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_warmstart_features_reproduce_nndsvd():
    """W_b has unit (or zero) columns, W_b H_b is the NNDSVD product, and an untrained network
    (zero last layer) returns exactly W_b, H_b."""
    rng = np.random.default_rng(3)
    m, n, ell, r = 300, 200, 12, 5
    QL = np.linalg.qr(rng.standard_normal((m, ell)))[0]
    Xhat = rng.standard_normal((ell, n)) * (0.7 ** np.arange(ell))[:, None]
    Wb, Hb, hs, Fw, Fh = WS.warmstart_features(QL, Xhat, r)
    Wn, Hn = O.nndsvd_compressed(QL, Xhat, r)
    norms = np.linalg.norm(Wb, axis=0)
    assert np.all((np.abs(norms - 1) < 1e-12) | (norms == 0))
    assert np.allclose(Wb @ Hb, Wn @ Hn, rtol=0, atol=1e-12 * np.abs(Wn @ Hn).max())
    assert np.allclose(np.linalg.norm(Hb, axis=1), hs)
    assert Fw.shape == (m, 3 * r) and Fh.shape == (n, 3 * r)
    F, Hd = 3 * r, 16
    p = WS.mlp_init(F, Hd, r, seed=4)
    Dw, _ = WS.mlp_forward(p, Fw, F, Hd, r)
    Dh, _ = WS.mlp_forward(p, Fh, F, Hd, r)
    W0, H0 = WS.warmstart_apply(Wb, Hb, hs, Dw, Dh)
    assert np.array_equal(W0, Wb) and np.array_equal(H0, Hb)
    # targets invert the map where the solution is positive
    Ws = np.abs(Wb + 0.01 * rng.standard_normal(Wb.shape)) + 0.1
    Hs = np.abs(Hb + 0.01 * rng.standard_normal(Hb.shape)) + 0.1
    Tw, Th = WS.warmstart_targets(Wb, Hb, hs, Ws, Hs)
    W1, H1 = WS.warmstart_apply(Wb, Hb, hs, Tw, Th)
    assert np.allclose(W1, Ws) and np.allclose(H1[hs > 0], Hs[hs > 0])


# ------------------------------------------------------------------ FP8 E4M3 copy of X

def test_e4m3_decode_matches_the_format_definition():
    """Codes the OCP E4M3 definition names: 1.0 = 0 0111 000, the largest finite 448 =
    0 1111 110, the smallest normal 2^-6 = 0 0001 000, the smallest subnormal 2^-9 = 0 0000 001,
    NaN = s 1111 111, and the sign bit."""
    d = O.e4m3_decode
    assert d(np.uint8(0x38)) == 1.0 and d(np.uint8(0xB8)) == -1.0
    assert d(np.uint8(0x7E)) == 448.0 and d(np.uint8(0x08)) == 2.0 ** -6
    assert d(np.uint8(0x01)) == 2.0 ** -9 and d(np.uint8(0x07)) == 7 / 8 * 2.0 ** -6
    assert d(np.uint8(0x00)) == 0.0 and d(np.uint8(0x3C)) == 1.5
    assert np.isnan(d(np.uint8(0x7F))) and np.isnan(d(np.uint8(0xFF)))
    v = d(np.arange(127, dtype=np.uint8))
    assert np.all(np.diff(v) > 0)                       # 127 increasing finite magnitudes
    assert np.isfinite(d(np.arange(256, dtype=np.uint8))).sum() == 254


def test_e4m3_encode_rounds_to_nearest_even_and_saturates():
    e = O.e4m3_encode
    assert e(1.0 + 1 / 16) == 0x38            # tie between 1 (mantissa 000) and 1.125: even
    assert e(1.0 + 3 / 16) == 0x3A            # tie between 1.125 and 1.25 (mantissa 010)
    assert e(1.0 + 1 / 16 + 1e-9) == 0x39     # just above the tie
    assert e(2.0 ** -10) == 0x00              # tie between 0 and 2^-9: zero (even)
    assert e(3 * 2.0 ** -10) == 0x02          # tie between 2^-9 and 2^-8: 2^-8 (even)
    assert e(500.0) == 0x7E and e(-1e6) == 0xFE
    assert e(-0.0) == 0x80 and e(-1e-6) == 0x80   # sign bit kept when rounding to zero
    rng = np.random.default_rng(0)
    v = np.exp(rng.uniform(np.log(2.0 ** -6), np.log(448.0), 100000))
    q = O.e4m3_decode(e(v))
    assert np.max(np.abs(q - v) / v) <= 2.0 ** -4   # half an ulp of a 3-bit mantissa
    # nearest: no other finite code is closer
    grid = O.e4m3_decode(np.arange(127, dtype=np.uint8))
    w = rng.uniform(0, 448, 2000)
    best = np.min(np.abs(grid[None, :] - w[:, None]), axis=1)
    assert np.all(np.abs(O.e4m3_decode(e(w)) - w) <= best)


def test_e8m0_tile_scale_is_the_smallest_power_of_two_that_fits():
    rng = np.random.default_rng(1)
    X = rng.exponential(1.0, (70, 45)) * np.exp(rng.uniform(-20, 20, (70, 45)))
    X[32:64, 32:45] = 0.0                                # an all-zero edge tile
    k = O.e8m0_tile_exponents(X)
    assert k.shape == (3, 2) and k[1, 1] == 0
    for a in range(3):
        for b in range(2):
            amax = np.abs(X[32 * a:32 * a + 32, 32 * b:32 * b + 32]).max()
            if amax > 0:
                assert amax / 2.0 ** k[a, b] <= 448.0 < amax / 2.0 ** (k[a, b] - 1)
    codes, kk = O.fp8_quantize(X)
    Xq = O.fp8_dequantize(codes, kk)
    big = X >= 2.0 ** -6 * 2.0 ** np.repeat(np.repeat(kk, 32, 0), 32, 1)[:70, :45]
    assert np.max(np.abs(Xq - X)[big] / X[big]) <= 2.0 ** -4
    assert np.all(np.abs(Xq) <= 448.0 * 2.0 ** np.repeat(np.repeat(kk, 32, 0), 32, 1)[:70, :45])


def test_fp8_layout_pads_rows_to_16_bytes():
    assert O.fp8_layout(100, 5000) == (5008, 500992, 500992 + 4 * 157)
    assert O.fp8_layout(64, 32) == (32, 2048, 2048 + 2)
