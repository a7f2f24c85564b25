"""Sparse X (CSR) through the C ABI against the FP64 oracle on the densified matrix.

Term-count matrices from the topic model of the inputs module stand in for the 20 Newsgroups
frequency matrix of Section 5.2 (documents x words, empty rows and columns included).

Tolerances: the CSR products are FP32 sums in a fixed order, against FP64 products at 1e-5
relative Frobenius; two runs are bit-identical (the transpose keeps row order within each
column). The FP32 sketch is compared in the basis-free projected form (1e-4, as the dense FP32
sketch) and the compression from the oracle's Q at 1e-5; the residual (expanded form, FP64
sums of FP32 dot products) at 1e-6 relative on the error; the whole solve within 1 % of the
oracle after the same iterations (Section 5.2's k = 60, r + r_ov = 72, w = 9, 150 iterations).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_02248_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_csr(lib, sp):
    return lib.Csr(torch.from_numpy(sp.row_ptr).cuda(), torch.from_numpy(sp.col).cuda(),
                   cu(sp.val), sp.shape)


@pytest.fixture(scope="module")
def small():
    sp = inputs.sparse_counts(3, m=1301, n=517, r=12, ell=24, w=2, mean_len=40)
    return sp, sp.dense()


@pytest.mark.parametrize("ell", [7, 40, 100])
def test_csr_pass_matches_dense_products(lib, ctx, small, ell):
    sp, X = small
    rng = np.random.default_rng(ell)
    m, n = sp.shape
    V, U = rng.standard_normal((n, ell)), rng.standard_normal((m, ell))
    p = lib.params(m, n, min(ell, 12), ell, power_iters=0)
    Xs = to_csr(lib, sp)
    # a sketch with w = 0 is one pass: Q_L = qr(X Omega_L), Q_R = qr(X^T Omega_R)
    QL, QR = lib.nmf_sketch_csr(ctx, p, Xs, cu(V), cu(U))
    oQL = O.qr_orthonormal(X @ V.astype(np.float32).astype(np.float64))
    oQR = O.qr_orthonormal(X.T @ U.astype(np.float32).astype(np.float64))
    assert rel(host(QL) @ (host(QL).T @ X), oQL @ (oQL.T @ X)) <= 1e-4
    assert rel(X @ host(QR) @ host(QR).T, X @ oQR @ oQR.T) <= 1e-4
    # the products themselves: compression with arbitrary (non-orthonormal) V, U
    Xhat, Xchk = lib.nmf_compress_csr(ctx, p, Xs, cu(U), cu(V))
    assert rel(host(Xchk), X @ V.astype(np.float32)) <= 1e-5
    assert rel(host(Xhat), U.astype(np.float32).T @ X) <= 1e-5
    Xhat2, Xchk2 = lib.nmf_compress_csr(ctx, p, Xs, cu(U), cu(V))
    assert torch.equal(Xhat, Xhat2) and torch.equal(Xchk, Xchk2)


def test_csr_edge_cases(lib, ctx):
    """Empty rows, empty columns, a row holding every column, one nonzero in all."""
    m, n = 70, 45
    rng = np.random.default_rng(9)
    X = np.zeros((m, n), np.float32)
    X[3, :] = rng.random(n)                       # a full row
    X[10:60:7, 5] = 2.0                           # column 5 in a few rows
    X[64, 44] = 7.0
    rows, cols = np.nonzero(X)
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=m))]).astype(np.int64)
    sp = inputs.SparseProblem(row_ptr, cols.astype(np.int32), X[rows, cols], (m, n), 2, 4, 0,
                              None, None, None, None, 0)
    Xs = to_csr(lib, sp)
    V, U = rng.standard_normal((n, 4)), rng.standard_normal((m, 4))
    p = lib.params(m, n, 2, 4)
    Xhat, Xchk = lib.nmf_compress_csr(ctx, p, Xs, cu(U), cu(V))
    Xd = X.astype(np.float64)
    assert rel(host(Xchk), Xd @ V.astype(np.float32)) <= 1e-6
    assert rel(host(Xhat), U.astype(np.float32).T @ Xd) <= 1e-6
    W, H = rng.random((m, 2)), rng.random((2, n))
    r_g = lib.nmf_residual_csr(ctx, p, Xs, cu(W), cu(H))[0]
    r_o = O.residual(Xd, W.astype(np.float32), H.astype(np.float32))[0]
    assert abs(r_g - r_o) <= 1e-6 * r_o


def test_csr_sketch_compress_residual_match_oracle(lib, ctx, small):
    sp, X = small
    m, n = sp.shape
    p = lib.params(m, n, sp.r, sp.ell, power_iters=2)
    Xs = to_csr(lib, sp)
    QL, QR = lib.nmf_sketch_csr(ctx, p, Xs, cu(sp.omega_L), cu(sp.omega_R))
    oQL, oQR = O.sketch(X, sp.omega_L, sp.omega_R, 2)
    assert rel(host(QL) @ (host(QL).T @ X), oQL @ (oQL.T @ X)) <= 1e-4
    assert rel(X @ host(QR) @ host(QR).T, X @ oQR @ oQR.T) <= 1e-4
    Xhat, Xchk = lib.nmf_compress_csr(ctx, p, Xs, cu(oQL), cu(oQR))
    oXhat, oXchk = O.compress(X, oQL.astype(np.float32), oQR.astype(np.float32))
    assert rel(host(Xhat), oXhat) <= 1e-5 and rel(host(Xchk), oXchk) <= 1e-5
    W, H = cu(sp.W0), cu(sp.H0)
    rg, e2, x2 = lib.nmf_residual_csr(ctx, p, Xs, W, H)
    ro, oe2, ox2 = O.residual(X, sp.W0, sp.H0)
    assert abs(x2 - ox2) <= 1e-12 * ox2
    assert abs(e2 - oe2) <= 1e-6 * oe2 and abs(rg - ro) <= 1e-6 * ro


def test_csr_solve_matches_oracle_section_5_2_settings(lib, ctx):
    """5000 documents x 1000 words, k = 60, r + r_ov = 72, w = 9, 150 FastHALS-RP iterations
    (Section 5.2), U[0,1) start; Omega from the oracle's own Philox with the solve's seed."""
    sp = inputs.sparse_counts(4, m=5000, n=1000, r=60, ell=72, w=9)
    X = sp.dense()
    m, n = sp.shape
    iters = 150
    p = lib.params(m, n, 60, 72, power_iters=9, iters=iters, seed=31, residual_every=50)
    W, H = cu(sp.W0), cu(sp.H0)
    e, it = lib.nmf_solve_csr(ctx, p, to_csr(lib, sp), W, H)
    assert it == iters and bool((W >= 0).all()) and bool((H >= 0).all())
    oL = O.philox_normal_np(n, 72, 31, 0)
    oR = O.philox_normal_np(m, 72, 31, 1)
    _, _, _, _, hist = O.solve(X, oL, oR, sp.W0, sp.H0, 9, iters)
    print(f"sparse 5000x1000 k=60: gpu {e:.6f} oracle {hist[-1][1]:.6f}")
    assert abs(e - hist[-1][1]) <= 0.01 * hist[-1][1]


def test_csr_arguments_are_checked(lib, ctx, small):
    sp, _ = small
    m, n = sp.shape
    Xs = to_csr(lib, sp)
    with pytest.raises(ValueError):
        lib.nmf_sketch_csr(ctx, lib.params(m + 1, n, 4, 8), Xs)
    with pytest.raises(ValueError):
        lib.Csr(torch.from_numpy(sp.row_ptr[:-1]).cuda(), torch.from_numpy(sp.col).cuda(),
                cu(sp.val), sp.shape)
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_residual_csr(ctx, lib.params(m, n, 129, 129), Xs, cu(np.zeros((m, 129))),
                             cu(np.zeros((129, n))))
    assert e.value.status == 1
