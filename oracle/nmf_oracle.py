"""FP64 CPU oracle: randomized two-sided sketch, compression, compressed NMF updates, residual.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the product path.

Notation (paper -> here). The paper factors X (d x n) as A B^T with A (d x k), B (n x k); here
X is m x n, W = A (m x r), H = B^T (r x n). The paper's left/right projections L (d x l) and
R (l x n) are Q_L (m x l) and Q_R^T (Q_R is n x l). Compressed data X_hat = Q_L^T X (l x n) and
X_chk = X Q_R (m x l), Section 4 (text before Algorithm 4). Compressed factors: W_tld = Q_L^T W
(the paper's A_hat, l x r) and H_tld = H Q_R (the transpose of the paper's B_chk, r x l).

Citations name the paper's section, equation or algorithm.

Functions and their pins (tests/test_oracle_pins.py):
  qr_orthonormal            orthonormality, reconstruction, uniqueness of the R>=0 factor
  sketch / power_product    exact-rank capture (closed form), singular-value identity (Sec. 3)
  compress                  special case l = min(m, n) (orthogonal Q)
  fasthals_rp_step          == hals_rp_step with explicit Eq. 4.6 residuals; KKT of each block;
                            == textbook FastHALS when Q_L, Q_R are square; brute-force minimiser
  hals_rp_step              KKT of each rank-1 sub-problem; golden-section brute force
  mu_rp_step                each half-step non-increasing in its own compressed objective
  mu_step                   Lee-Seung monotonicity on full data
  residual / objective      closed forms on constructed inputs
  compressed_sq_error       equals the exact squared error when Q_L is square
  nndsvd_compressed         exact for a rank-1 non-negative matrix; exact for a block-diagonal
                            non-negative matrix (every component j >= 1 reached); each component
                            equals the dominant quadrant of s_j u_j v_j^T (mixed signs)
  monitor_estimate          equals ||X - W H||^2 + 2 <X - X_q, W H - X> when Q_L is square
  rounding_term             closed form on a constructed copy; vanishes for an exact copy
  gini                      closed forms (uniform -> 0, one-hot -> 1 - 1/N)
  spectrum                  equals sigma_j(X) for exact-rank X (Q_L X_hat = X)
  decay_rate                recovers p of an exactly exponential spectrum; scale-invariant
  philox4x32_10             published known-answer vectors of the generator
  philox_normal_np          element for element equal to philox_normal (the scalar definition)
  solve_to_target           stops at the same check as `solve` with a residual at every check
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "qr_orthonormal", "sketch", "power_product", "compress",
    "fasthals_rp_step", "hals_rp_step", "mu_rp_step",
    "fasthals_step", "mu_step", "semi_nmf_mu_step",
    "residual", "objective", "compressed_sq_error", "monitor_estimate", "rounding_term",
    "nndsvd_compressed", "gini", "spectrum", "decay_rate", "solve", "solve_to_target", "iterate",
    "philox4x32_10", "philox_normal", "philox_normal_np", "memory_floats_rp",
    "EPS_MU",
]

# Reading: the multiplicative rule needs a guard in its denominator; the paper is silent.
EPS_MU = 1e-12


def _f64(a):
    return np.array(a, dtype=np.float64, copy=True)


def _pos(M):
    """Positive part (|M| + M) / 2, as in the semi-NMF rule of Ding, Li & Jordan (2010)."""
    return (np.abs(M) + M) * 0.5


def _neg(M):
    """Negative part (|M| - M) / 2 (non-negative entries)."""
    return (np.abs(M) - M) * 0.5


# --------------------------------------------------------------------------------------------
# Section 3: random projection
# --------------------------------------------------------------------------------------------

def qr_orthonormal(Y):
    """Q of the thin QR factorisation Y = Q R (Section 3, Eq. 3.4-3.5: "Q is defined by the QR
    decomposition of P(X)").

    One LAPACK Householder QR (numpy) as a single step. Columns are sign-flipped so that R has a
    non-negative diagonal; for a full-column-rank Y this makes Q unique, so any correct QR
    algorithm (e.g. Cholesky-based) must produce the same Q.
    """
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def power_product(X, omega, w):
    """P(X) = (X X^T)^w X Omega, Section 3 Eq. 3.5, formed literally (no re-orthonormalisation).

    Only for the singular-value identity of Section 3 on small inputs; the sketch itself uses
    the numerically stable subspace form below.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = X @ np.asarray(omega, dtype=np.float64)
    for _ in range(w):
        Y = X @ (X.T @ Y)
    return Y


def sketch(X, omega_L, omega_R, w):
    """Two-sided randomized range finder (Section 3 Eq. 3.5; Section 3.1 defines L from P(X)
    and R from P(X^T)).

    Left chain:  Q_L spans (X X^T)^w X Omega_L    (m x l), Omega_L is n x l.
    Right chain: Q_R spans (X^T X)^w X^T Omega_R  (n x l), Omega_R is m x l. The paper's R = Q_R^T.

    Reading (the paper shows no intermediate step): orthonormalise after every application of X
    or X^T. In exact arithmetic the span equals that of Eq. 3.5's product; in floating point the
    plain product loses every direction but the top one.
    """
    X = np.asarray(X, dtype=np.float64)
    QL = qr_orthonormal(X @ np.asarray(omega_L, dtype=np.float64))
    for _ in range(w):
        QL = qr_orthonormal(X.T @ QL)
        QL = qr_orthonormal(X @ QL)
    QR = qr_orthonormal(X.T @ np.asarray(omega_R, dtype=np.float64))
    for _ in range(w):
        QR = qr_orthonormal(X @ QR)
        QR = qr_orthonormal(X.T @ QR)
    return QL, QR


def compress(X, QL, QR):
    """Left- and right-projected data (Section 4, before Algorithm 4):
    X_hat = L^T X = Q_L^T X (l x n) and X_chk = X R^T = X Q_R (m x l)."""
    X = np.asarray(X, dtype=np.float64)
    return np.asarray(QL, np.float64).T @ X, X @ np.asarray(QR, np.float64)


def memory_floats_rp(m, n, r, ell):
    """Memory of the compressed methods, Section 4.2 Table 4.1: (2 l + k)(d + n) floats."""
    return (2 * ell + r) * (m + n)


# --------------------------------------------------------------------------------------------
# Section 4: FastHALS-RP, HALS-RP; Section 3.1: semi-NMF with random projection (MU-RP)
# --------------------------------------------------------------------------------------------

def _w_sweep(W, S, G):
    """Gauss-Seidel sweep over components j = 1..r of the first line of Eq. fastHALS_a:
    w_j <- [ w_j + (S_j - W G_j) / G_jj ]_+ with S = X_chk B_chk and G = B_chk^T B_chk.
    W is updated in place, so component j sees the already-updated components 1..j-1.
    Reading: a zero pivot G_jj leaves w_j unchanged (the paper is silent)."""
    r = W.shape[1]
    for j in range(r):
        if G[j, j] > 0.0:
            W[:, j] = np.maximum(0.0, W[:, j] + (S[:, j] - W @ G[:, j]) / G[j, j])
    return W


def _h_sweep(H, P, G, alpha=0.0, beta=0.0):
    """Gauss-Seidel sweep of the second line of Eq. fastHALS_a (rows of H = columns of B), in the
    regularised form of Section 4.1:
    h_j <- [ (h_j G_jj + P_j - G_j^T H - alpha) / (G_jj + beta) ]_+,
    with P = A_hat^T X_hat (r x n) and G = A_hat^T A_hat. alpha = beta = 0 gives Eq. fastHALS_a.
    """
    r = H.shape[0]
    for j in range(r):
        if alpha == 0.0 and beta == 0.0:
            if G[j, j] > 0.0:
                H[j, :] = np.maximum(0.0, H[j, :] + (P[j, :] - G[j, :] @ H) / G[j, j])
        elif G[j, j] + beta > 0.0:
            num = H[j, :] * G[j, j] + P[j, :] - G[j, :] @ H - alpha
            H[j, :] = np.maximum(0.0, num / (G[j, j] + beta))
    return H


def _normalise(W, H):
    """Section 4 after Eq. fastHALS_a: a_j <- a_j / ||a_j||_2. Reading: the scale moves to the
    matching row of H so that W H is unchanged; a zero column is left as it is."""
    s = np.sqrt(np.sum(W * W, axis=0))
    for j in range(W.shape[1]):
        if s[j] > 0.0:
            W[:, j] /= s[j]
            H[j, :] *= s[j]
    return W, H


def fasthals_rp_step(W, H, QL, QR, Xhat, Xchk, normalize=True, alpha=0.0, beta=0.0):
    """One FastHALS-RP iteration (Section 4, Eq. fastHALS_a; regularised form Section 4.1).

    Block order (reading): the whole W sweep over j, then the normalisation, then the whole H
    sweep, each sweep using the products S, G formed once before it (the quantities the paper
    names H, G, W, P in Section 4.1). Algorithm 4's per-j interleaving is `hals_rp_step(...,
    order="interleaved")`.
    """
    W = _f64(W)
    H = _f64(H)
    QL = np.asarray(QL, np.float64)
    QR = np.asarray(QR, np.float64)
    # W half-step: B_chk = R B, i.e. H_tld = H Q_R (r x l)
    Ht = H @ QR
    G_W = Ht @ Ht.T                      # B_chk^T B_chk  (paper's G)
    S_W = np.asarray(Xchk, np.float64) @ Ht.T   # X_chk B_chk (paper's H), m x r
    _w_sweep(W, S_W, G_W)
    if normalize:
        _normalise(W, H)
    # H half-step: A_hat = L^T A, i.e. W_tld = Q_L^T W (l x r)
    Wt = QL.T @ W
    G_H = Wt.T @ Wt                      # A_hat^T A_hat (paper's W)
    S_H = Wt.T @ np.asarray(Xhat, np.float64)   # (X_hat^T A_hat)^T (paper's P^T), r x n
    _h_sweep(H, S_H, G_H, alpha, beta)
    return W, H


def hals_rp_step(W, H, QL, QR, Xhat, Xchk, order="block", normalize=True):
    """One HALS-RP iteration with the component residuals formed explicitly
    (Algorithm 4, Eq. 4.6 and Eq. hals_update): a_j <- [X_chk_j b_chk_j / b_chk_j^T b_chk_j]_+ and
    b_j <- [X_hat_j^T a_hat_j / a_hat_j^T a_hat_j]_+, where
    X_hat_j = X_hat - A_hat B^T + a_hat_j b_j^T and X_chk_j = X_chk - A B_chk^T + a_j b_chk_j^T.

    order="block": all a_j, then all b_j (the order fasthals_rp_step uses);
    order="interleaved": a_j then b_j for each j, as Algorithm 4 is printed.
    The normalisation is applied right after each a_j update (compensated in b_j).
    Costs O(m n l k) per iteration; for pins on small inputs only.
    """
    A = _f64(W)
    B = _f64(H).T.copy()        # n x k
    L = np.asarray(QL, np.float64)
    R = np.asarray(QR, np.float64).T     # l x n, the paper's R
    Xhat = np.asarray(Xhat, np.float64)
    Xchk = np.asarray(Xchk, np.float64)
    k = A.shape[1]

    def update_a(j):
        Bc = R @ B                                              # B_chk (l x k)
        Xc_j = Xchk - A @ Bc.T + np.outer(A[:, j], Bc[:, j])    # Eq. 4.6, second line
        den = Bc[:, j] @ Bc[:, j]
        if den > 0.0:
            A[:, j] = np.maximum(0.0, (Xc_j @ Bc[:, j]) / den)
        if normalize:
            s = np.linalg.norm(A[:, j])
            if s > 0.0:
                A[:, j] /= s
                B[:, j] *= s

    def update_b(j):
        Ah = L.T @ A                                            # A_hat (l x k)
        Xh_j = Xhat - Ah @ B.T + np.outer(Ah[:, j], B[:, j])    # Eq. 4.6, first line
        den = Ah[:, j] @ Ah[:, j]
        if den > 0.0:
            B[:, j] = np.maximum(0.0, (Xh_j.T @ Ah[:, j]) / den)

    if order == "block":
        for j in range(k):
            update_a(j)
        for j in range(k):
            update_b(j)
    elif order == "interleaved":
        for j in range(k):
            update_a(j)
            update_b(j)
    else:
        raise ValueError(order)
    return A, B.T.copy()


def mu_rp_step(W, H, QL, QR, Xhat, Xchk, eps=EPS_MU):
    """One iteration of semi-NMF with random projection (Section 3.1, Algorithm 3): the W
    sub-problem min ||X R^T - A (R B)^T|| and the H sub-problem min ||L^T X - (L^T A) B^T||, each
    with only the unprojected factor kept non-negative.

    Reading: the paper names the semi-NMF method of Ding, Li & Jordan (2010) for both
    sub-problems but prints no rule; this is their multiplicative rule for the non-negative factor
    of X ~ F G^T, G <- G o sqrt(((X^T F)^+ + G (F^T F)^-) / ((X^T F)^- + G (F^T F)^+)):
      W <- W o sqrt((S_W^+ + W G_W^-) / (S_W^- + W G_W^+ + eps)),  S_W = X_chk H_tld^T, G_W = H_tld H_tld^T
      H <- H o sqrt((S_H^+ + G_H^- H) / (S_H^- + G_H^+ H + eps)),  S_H = W_tld^T X_hat, G_H = W_tld^T W_tld
    W first, then H (Algorithm 3 order); no normalisation.
    """
    W = _f64(W)
    H = _f64(H)
    QL = np.asarray(QL, np.float64)
    QR = np.asarray(QR, np.float64)
    Ht = H @ QR
    G_W = Ht @ Ht.T
    S_W = np.asarray(Xchk, np.float64) @ Ht.T
    W = W * np.sqrt((_pos(S_W) + W @ _neg(G_W)) / (_neg(S_W) + W @ _pos(G_W) + eps))
    Wt = QL.T @ W
    G_H = Wt.T @ Wt
    S_H = Wt.T @ np.asarray(Xhat, np.float64)
    H = H * np.sqrt((_pos(S_H) + _neg(G_H) @ H) / (_neg(S_H) + _pos(G_H) @ H + eps))
    return W, H


def semi_nmf_mu_step(X, F, G, eps=EPS_MU):
    """The semi-NMF rule alone on X ~ F G^T (Ding, Li & Jordan 2010), G >= 0, F fixed:
    G <- G o sqrt(((X^T F)^+ + G (F^T F)^-) / ((X^T F)^- + G (F^T F)^+ + eps)).
    Used by the monotonicity pin of each MU-RP half-step."""
    X = np.asarray(X, np.float64)
    F = np.asarray(F, np.float64)
    G = _f64(G)
    XtF = X.T @ F
    FtF = F.T @ F
    return G * np.sqrt((_pos(XtF) + G @ _neg(FtF)) / (_neg(XtF) + G @ _pos(FtF) + eps))


# --------------------------------------------------------------------------------------------
# Section 2: uncompressed methods (pins and special cases)
# --------------------------------------------------------------------------------------------

def fasthals_step(W, H, X, normalize=True):
    """One FastHALS iteration on the full data (Section 2.2, Cichocki & Phan): the same sweeps
    as fasthals_rp_step with S_W = X H^T, G_W = H H^T, S_H = W^T X, G_H = W^T W."""
    W = _f64(W)
    H = _f64(H)
    X = np.asarray(X, np.float64)
    _w_sweep(W, X @ H.T, H @ H.T)
    if normalize:
        _normalise(W, H)
    _h_sweep(H, W.T @ X, W.T @ W)
    return W, H


def mu_step(W, H, X, eps=0.0):
    """Lee & Seung multiplicative update on the full data (Section 2.1, Algorithm 1 order: A
    first, then B): W <- W o (X H^T) / (W H H^T), H <- H o (W^T X) / (W^T W H)."""
    W = _f64(W)
    H = _f64(H)
    X = np.asarray(X, np.float64)
    W = W * (X @ H.T) / (W @ (H @ H.T) + eps)
    H = H * (W.T @ X) / ((W.T @ W) @ H + eps)
    return W, H


# --------------------------------------------------------------------------------------------
# Objective and residual (Section 2, Eq. 2.2)
# --------------------------------------------------------------------------------------------

def objective(X, W, H):
    """J = 1/2 ||X - A B^T||_F^2 (Section 2, Eq. 2.2)."""
    D = np.asarray(X, np.float64) - np.asarray(W, np.float64) @ np.asarray(H, np.float64)
    return 0.5 * float(np.sum(D * D))


def residual(X, W, H):
    """Relative reconstruction error ||X - W H||_F / ||X||_F (the error of Eq. 2.2, normalised).
    Returns (rel_err, ||X - W H||_F^2, ||X||_F^2)."""
    X = np.asarray(X, np.float64)
    D = X - np.asarray(W, np.float64) @ np.asarray(H, np.float64)
    e2 = float(np.sum(D * D))
    x2 = float(np.sum(X * X))
    return float(np.sqrt(e2 / x2)) if x2 > 0 else float(np.sqrt(e2)), e2, x2


def compressed_sq_error(x2, QL, Xhat, W, H):
    """Estimate of ||X - W H||_F^2 from compressed data only (a monitor, no X read):
    ||X||^2 - 2 <W_tld^T X_hat, H> + <W^T W, H H^T>, using X ~ Q_L X_hat (Section 3, Eq. 3.4).
    With P = Q_L Q_L^T it equals ||X - W H||^2 + 2 <(I - P) X, W H> for any inputs (the cross
    term sees only P X), hence exact when P X = X; both are pinned."""
    W = np.asarray(W, np.float64)
    H = np.asarray(H, np.float64)
    Wt = np.asarray(QL, np.float64).T @ W
    cross = float(np.sum((Wt.T @ np.asarray(Xhat, np.float64)) * H))
    quad = float(np.sum((W.T @ W) * (H @ H.T)))
    return x2 - 2.0 * cross + quad


def rounding_term(X, Xq):
    """<X - X_q, X>: how far a low-precision copy X_q of X moves the cross term <X, W H> of the
    error when the compressed data are made from X_q (plain FP64 sum over all entries)."""
    X = np.asarray(X, np.float64)
    return float(np.sum((X - np.asarray(Xq, np.float64)) * X))


def monitor_estimate(x2, QL, Xhat, W, H, xq_term=0.0):
    """Error monitor of a solve whose compressed data X_hat = Q_L^T X_q come from a copy X_q of X:
    ||X - W H||^2 ~ ||X||^2 - 2 (<W_tld^T X_hat, H> + <X - X_q, X>) + <W^T W, H H^T>.
    The cross term <X, W H> is split as <X_q, W H> + <X - X_q, W H>; the first is replaced by its
    projection (Section 3, Eq. 3.4), the second by <X - X_q, X> (W H ~ X near a solution).
    With Q_L square the estimate equals ||X - W H||^2 + 2 <X - X_q, W H - X> exactly (pinned)."""
    return compressed_sq_error(x2, QL, Xhat, W, H) - 2.0 * float(xq_term)


# --------------------------------------------------------------------------------------------
# Initialisation and diagnostics
# --------------------------------------------------------------------------------------------

def nndsvd_compressed(QL, Xhat, r):
    """NNDSVD initialisation (Boutsidis & Gallopoulos 2008) from compressed data: the truncated
    SVD of X ~ Q_L X_hat is Q_L U' S V^T with X_hat = U' S V^T (LAPACK SVD as one step). For each
    component the larger-norm sign part of the singular-vector pair is kept; the first pair is
    taken in absolute value. Zeros are kept as zeros. Sign-invariant in each (u_j, v_j) pair."""
    QL = np.asarray(QL, np.float64)
    Xhat = np.asarray(Xhat, np.float64)
    U1, s, Vt = np.linalg.svd(Xhat, full_matrices=False)
    U = QL @ U1[:, :r]
    V = Vt[:r].T
    m, n = QL.shape[0], Xhat.shape[1]
    W = np.zeros((m, r))
    H = np.zeros((r, n))
    W[:, 0] = np.sqrt(s[0]) * np.abs(U[:, 0])
    H[0, :] = np.sqrt(s[0]) * np.abs(V[:, 0])
    for j in range(1, r):
        x, y = U[:, j], V[:, j]
        xp, xn, yp, yn = _pos(x), _neg(x), _pos(y), _neg(y)
        nxp, nxn = np.linalg.norm(xp), np.linalg.norm(xn)
        nyp, nyn = np.linalg.norm(yp), np.linalg.norm(yn)
        mp, mn = nxp * nyp, nxn * nyn
        if mp >= mn:
            if mp == 0.0:
                continue
            u, v, sig = xp / nxp, yp / nyp, mp
        else:
            u, v, sig = xn / nxn, yn / nyn, mn
        W[:, j] = np.sqrt(s[j] * sig) * u
        H[j, :] = np.sqrt(s[j] * sig) * v
    return W, H


def spectrum(Xhat):
    """Singular values of the compressed data X_hat (LAPACK SVD as one step), descending: with
    X ~ Q_L X_hat (Section 3, Eq. 3.4) they estimate sigma_1..sigma_l of X."""
    return np.linalg.svd(np.asarray(Xhat, np.float64), compute_uv=False)


def decay_rate(sigma, rel_floor=1e-3):
    """Decay rate p of a spectrum, Section 5.2. Reading: the paper writes the spectrum as
    sigma_j(X)^-p, but its values (p = 0.0012 and 0.0053 for spectra of 1000 and 400 values) fit
    an exponential decay sigma_j ~ C exp(-p j); p = minus the least-squares slope of log sigma_j
    against j (j from 0) over the entries above rel_floor * sigma_1."""
    s = np.asarray(sigma, np.float64)
    j = np.arange(s.size, dtype=np.float64)
    keep = s > rel_floor * s[0]
    slope, _ = np.polyfit(j[keep], np.log(s[keep]), 1)
    return float(-slope)


def gini(B):
    """Gini coefficient of the entries of B (Section 5.1):
    G = sum_i (2 i - N - 1) b_i / (N sum_i b_i), b sorted ascending, i = 1..N, N = n k."""
    b = np.sort(np.asarray(B, np.float64).ravel())
    N = b.size
    i = np.arange(1, N + 1, dtype=np.float64)
    tot = b.sum()
    return float(np.sum((2.0 * i - N - 1.0) * b) / (N * tot)) if tot > 0 else 0.0


# --------------------------------------------------------------------------------------------
# Whole solve (Algorithm 3 / Algorithm 4 loops with a fixed iteration count)
# --------------------------------------------------------------------------------------------

def iterate(W, H, QL, QR, Xhat, Xchk, iters, rule="fasthals", alpha=0.0, beta=0.0, eps=EPS_MU):
    """Run `iters` iterations of the compressed updates. Reading: the paper's "convergence
    criterion" (Algorithms 1-4) is never defined, so the count is fixed by the caller."""
    for _ in range(iters):
        if rule == "fasthals":
            W, H = fasthals_rp_step(W, H, QL, QR, Xhat, Xchk, alpha=alpha, beta=beta)
        elif rule == "mu":
            W, H = mu_rp_step(W, H, QL, QR, Xhat, Xchk, eps=eps)
        else:
            raise ValueError(rule)
    return W, H


def solve(X, omega_L, omega_R, W0, H0, w, iters, rule="fasthals", residual_every=0):
    """Sketch, compress, iterate, residual: the whole compressed-NMF pipeline in FP64.
    Returns (W, H, QL, QR, history) with history a list of (iteration, rel_err) taken every
    `residual_every` iterations (and at the end)."""
    QL, QR = sketch(X, omega_L, omega_R, w)
    Xhat, Xchk = compress(X, QL, QR)
    W, H = _f64(W0), _f64(H0)
    hist = []
    step = residual_every if residual_every > 0 else iters
    done = 0
    while done < iters:
        k = min(step, iters - done)
        W, H = iterate(W, H, QL, QR, Xhat, Xchk, k, rule=rule)
        done += k
        hist.append((done, residual(X, W, H)[0]))
    return W, H, QL, QR, hist


def solve_to_target(X, omega_L, omega_R, W0, H0, w, iters, target, check_every=10,
                    rule="fasthals", margin=0.05):
    """Whole solve with the stopping rule of a timed run (the paper leaves the convergence
    criterion undefined; reading: stop at the first check whose exact relative residual is at or
    below `target`). Sketch and compression as in `solve`; every `check_every` iterations the
    compressed error estimate (`compressed_sq_error`, no read of X) is formed, and the exact
    residual of X is computed only when that estimate is within `margin` of the target, or at the
    last check. The estimate only decides whether the exact residual is worth computing; the stop
    itself is decided by the exact residual alone.

    Returns (W, H, iters_done, rel_err, exact_checks); rel_err is the last exact residual (at
    iters_done when the target was met)."""
    X = np.asarray(X, np.float64)
    QL, QR = sketch(X, omega_L, omega_R, w)
    Xhat, Xchk = compress(X, QL, QR)
    x2 = float(np.sum(X * X))
    W, H = _f64(W0), _f64(H0)
    done, checks, rel = 0, 0, float("nan")
    while done < iters:
        k = min(check_every, iters - done)
        W, H = iterate(W, H, QL, QR, Xhat, Xchk, k, rule=rule)
        done += k
        est = np.sqrt(max(compressed_sq_error(x2, QL, Xhat, W, H), 0.0) / x2)
        if done >= iters or est <= target * (1.0 + margin):
            rel = residual(X, W, H)[0]
            checks += 1
            if rel <= target:
                break
    return W, H, done, rel, checks


# --------------------------------------------------------------------------------------------
# Counter-based generator for the Gaussian test matrix (Section 3: Omega ~ N(0,1))
# --------------------------------------------------------------------------------------------

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11), written from the
    published definition: each round multiplies words 0 and 2 by the two multipliers, takes
    the 64-bit products' halves, XORs the high halves with words 1, 3 and the key; the key is
    bumped by the two Weyl constants between rounds. ctr: 4 uint32, key: 2 uint32."""
    c0, c1, c2, c3 = (int(x) & _MASK32 for x in ctr)
    k0, k1 = (int(x) & _MASK32 for x in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _PHILOX_W0) & _MASK32
            k1 = (k1 + _PHILOX_W1) & _MASK32
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = (p0 >> 32) & _MASK32, p0 & _MASK32
        hi1, lo1 = (p1 >> 32) & _MASK32, p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox_normal(rows, cols, seed, stream):
    """rows x cols standard normals from Philox4x32-10 and the Box-Muller transform.

    Element e = i * cols + k (row-major) uses block b = e // 4 and lane e % 4 of the Philox
    output for counter (b mod 2^32, b >> 32, stream, 0) and key (seed mod 2^32, seed >> 32).
    Words are mapped to uniforms u = (x >> 8 + 1/2) 2^-24 in (0, 1); the pair (u0, u1) gives
    z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1), likewise (u2, u3).
    Pure Python: for small matrices only (the generator pin)."""
    total = rows * cols
    out = np.empty(total, dtype=np.float64)
    key = (seed & _MASK32, (seed >> 32) & _MASK32)
    nblk = (total + 3) // 4
    for b in range(nblk):
        x = philox4x32_10((b & _MASK32, (b >> 32) & _MASK32, stream, 0), key)
        u = [((xi >> 8) + 0.5) * 2.0 ** -24 for xi in x]
        rad0 = np.sqrt(-2.0 * np.log(u[0]))
        rad1 = np.sqrt(-2.0 * np.log(u[2]))
        z = (rad0 * np.cos(2 * np.pi * u[1]), rad0 * np.sin(2 * np.pi * u[1]),
             rad1 * np.cos(2 * np.pi * u[3]), rad1 * np.sin(2 * np.pi * u[3]))
        for t in range(4):
            e = 4 * b + t
            if e < total:
                out[e] = z[t]
    return out.reshape(rows, cols)


def philox_normal_np(rows, cols, seed, stream):
    """philox_normal for large matrices: the same definition (counter, key, rounds, uniform map,
    Box-Muller) evaluated on numpy arrays of counters at once. Pinned element for element
    against the scalar philox_normal."""
    total = rows * cols
    nblk = (total + 3) // 4
    b = np.arange(nblk, dtype=np.uint64)
    m32 = np.uint64(_MASK32)
    c0 = b & m32
    c1 = b >> np.uint64(32)
    c2 = np.full(nblk, np.uint64(stream & _MASK32))
    c3 = np.zeros(nblk, dtype=np.uint64)
    k0 = np.uint64(seed & _MASK32)
    k1 = np.uint64((seed >> 32) & _MASK32)
    M0, M1 = np.uint64(_PHILOX_M0), np.uint64(_PHILOX_M1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & m32
            k1 = (k1 + np.uint64(_PHILOX_W1)) & m32
        p0 = M0 * c0          # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & m32
        hi1, lo1 = p1 >> np.uint64(32), p1 & m32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    u = [((x >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24 for x in (c0, c1, c2, c3)]
    rad0 = np.sqrt(-2.0 * np.log(u[0]))
    rad1 = np.sqrt(-2.0 * np.log(u[2]))
    z = np.empty((nblk, 4), dtype=np.float64)
    z[:, 0] = rad0 * np.cos(2 * np.pi * u[1])
    z[:, 1] = rad0 * np.sin(2 * np.pi * u[1])
    z[:, 2] = rad1 * np.cos(2 * np.pi * u[3])
    z[:, 3] = rad1 * np.sin(2 * np.pi * u[3])
    return z.ravel()[:total].reshape(rows, cols)
