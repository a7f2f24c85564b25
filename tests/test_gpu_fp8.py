"""FP8 copy of X (OCP E4M3 codes, one E8M0 scale a 32 x 32 tile) and the contractions that read it.

The quantization is integer work decided in FP32 on both sides (the scale exponent from frexp of
the tile maximum, the code by round-to-nearest-even of an exact power-of-two scaling), so the
codes, the pad bytes and the scale bytes are compared bit for bit with the oracle. The dual pass
on the FP8 copy is compared with the FP64 oracle applied to the dequantised values: exactly
(1e-5, the library's FP32 accumulation) once the basis operands are rounded to BF16 as the
tensor-core pass rounds them (RNE, relative error <= 2^-9; the SIMT pass keeps them in FP32).
The sketch and compression through the SIMT pass match the oracle on the dequantised copy to
1e-4; through the tensor cores, whose bases are BF16, to the 2e-2 of the BF16 sketch. The solve
with an FP8 sketch compresses from the FP32 X and must end within 1 % of the oracle taking the
same steps.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_02248_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda")


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def split_copy(q, m, n):
    """(codes m x n, pad bytes, scale bytes) of the library's FP8 layout."""
    buf = q.buf.cpu().numpy()
    ldq, off, total = O.fp8_layout(m, n)
    assert buf.size >= total
    rows = buf[:m * ldq].reshape(m, ldq)
    tm, tn = -(-m // 32), -(-n // 32)
    return rows[:, :n], rows[:, n:], buf[off:off + tm * tn].reshape(tm, tn)


def bf16(a):
    """Round to the nearest BF16 (ties to even), as the tensor-core pass rounds V and U."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def varied_matrix(seed, m, n):
    """Entries over many binades, tile by tile, with negative values, an all-zero tile and exact
    ties of the E4M3 grid (x / 2^k = 1 + 1/16)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, n)) * np.exp(rng.uniform(-12, 12, (m, n)))
    X[:32, :32] = 0.0
    if m > 40 and n >= 48:
        # x / 2^k = (1 + 1/16) 2^j: a tie of the E4M3 grid whatever the tile's power of two
        X[40, 40:48] = (1.0 + 1.0 / 16.0) * 2.0 ** np.arange(8)
    return X.astype(np.float32)


@pytest.mark.parametrize("shape", [(300, 517), (64, 32), (97, 1000), (1, 7)])
def test_quantize_fp8_is_bit_exact(lib, ctx, shape):
    m, n = shape
    X = varied_matrix(7, m, n)
    q = lib.nmf_quantize(ctx, cu(X), prec="fp8")
    lib.nmf_sync(ctx)
    codes, pad, scales = split_copy(q, m, n)
    c_ref, k_ref = O.fp8_quantize(X.astype(np.float64))
    assert np.array_equal(scales.astype(np.int64) - 127, k_ref)
    assert np.array_equal(codes, c_ref)
    assert not pad.any()
    assert q.buf.numel() == lib.nmf_quantized_bytes("fp8", m, n) == O.fp8_layout(m, n)[2]


def test_quantize_fp8_full_size_sampled_tiles(lib, ctx):
    """The dense 20000 x 5000 workload (Exp(1) factors, 1 % noise): 200 random tiles against the
    oracle, and the relative error of the whole copy within the E4M3 bound."""
    pr = inputs.dense_20k_5k(seed=3)
    X = pr.X
    m, n = X.shape
    Xd = cu(X)
    q = lib.nmf_quantize(ctx, Xd, prec="fp8")
    lib.nmf_sync(ctx)
    codes, pad, scales = split_copy(q, m, n)
    assert not pad.any()
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = rng.integers(0, -(-m // 32)), rng.integers(0, -(-n // 32))
        T = X[32 * a:32 * a + 32, 32 * b:32 * b + 32].astype(np.float64)
        c_ref, k_ref = O.fp8_quantize(T)
        assert int(scales[a, b]) - 127 == k_ref[0, 0]
        assert np.array_equal(codes[32 * a:32 * a + 32, 32 * b:32 * b + 32], c_ref)
    rows = slice(0, 2048)     # the relative error of a 2048-row block of the copy
    Xq = O.fp8_dequantize(codes[rows], scales[:64].astype(np.int64) - 127)
    assert rel(Xq, X[rows]) <= 2.0 ** -4


def test_fp8_dual_pass_matches_the_dequantised_oracle(lib, ctx):
    m, n, ell = 700, 333, 24
    rng = np.random.default_rng(2)
    X = (rng.exponential(1.0, (m, n)) * rng.uniform(0.1, 10.0, (m, 1))).astype(np.float32)
    V = rng.standard_normal((n, ell)).astype(np.float32)
    U = rng.standard_normal((m, ell)).astype(np.float32)
    q = lib.nmf_quantize(ctx, cu(X), prec="fp8")
    Y, Z = lib.nmf_dual_pass(ctx, q, cu(V), cu(U), prec="fp8")   # tensor cores (m, n >= 128)
    codes, _, scales = split_copy(q, m, n)
    Xq = O.fp8_dequantize(codes, scales.astype(np.int64) - 127)
    assert rel(Y.cpu().numpy(), Xq @ bf16(V)) <= 1e-5
    assert rel(Z.cpu().numpy(), Xq.T @ bf16(U)) <= 1e-5
    # small enough for the SIMT pass only (fewer than 128 columns): FP32 bases
    Xs = X[:, :100]
    q2 = lib.nmf_quantize(ctx, cu(Xs), prec="fp8")
    Y2, Z2 = lib.nmf_dual_pass(ctx, q2, cu(V[:100]), cu(U), prec="fp8")
    codes2, _, scales2 = split_copy(q2, m, 100)
    Xq2 = O.fp8_dequantize(codes2, scales2.astype(np.int64) - 127)
    assert rel(Y2.cpu().numpy(), Xq2 @ V[:100]) <= 1e-5
    assert rel(Z2.cpu().numpy(), Xq2.T @ U) <= 1e-5


@pytest.mark.parametrize("m,n,ell", [(1000, 3001, 40), (4096, 700, 70), (256, 128, 16)])
def test_fp8_tensor_core_pass_matches_simt_and_oracle(lib, ctx, m, n, ell):
    """The tensor-core pass (codes converted to BF16 in shared memory, exact) against the SIMT
    pass on the same copy (the sketch with the SIMT flag) and against the FP64 oracle applied
    to the dequantised values."""
    rng = np.random.default_rng(m + n)
    X = (rng.exponential(1.0, (m, n)) * np.exp(rng.uniform(-3, 3, (m, 1)))).astype(np.float32)
    V = rng.standard_normal((n, ell)).astype(np.float32)
    U = rng.standard_normal((m, ell)).astype(np.float32)
    q = lib.nmf_quantize(ctx, cu(X), prec="fp8")
    Y, Z = lib.nmf_dual_pass(ctx, q, cu(V), cu(U), prec="fp8")
    codes, _, scales = split_copy(q, m, n)
    Xq = O.fp8_dequantize(codes, scales.astype(np.int64) - 127)
    assert rel(Y.cpu().numpy(), Xq @ bf16(V)) <= 1e-5
    assert rel(Z.cpu().numpy(), Xq.T @ bf16(U)) <= 1e-5
    pr = inputs.random_problem(9, m, n, min(10, ell - 4), ell, w=1)
    q2 = lib.nmf_quantize(ctx, cu(pr.X), prec="fp8")
    out = []
    for flags in (0, lib.FLAG_SIMT_DUAL_PASS):
        p = lib.params(m, n, pr.r, ell, power_iters=1, prec="fp8", flags=flags)
        QL, QR = lib.nmf_sketch(ctx, p, q2, cu(pr.omega_L), cu(pr.omega_R))
        out.append((QL.double().cpu().numpy(), QR.double().cpu().numpy()))
    (a, b), (c, d) = out     # BF16 bases on the tensor cores, FP32 on the SIMT pass
    assert rel(a @ a.T, c @ c.T) <= 2e-2 and rel(b @ b.T, d @ d.T) <= 2e-2


def test_fp8_tensor_core_pass_full_size_sampled(lib, ctx):
    """The dense 20000 x 5000 workload at its sketch width: Y = X_q V on 300 sampled rows and
    Z = X_q^T U on 300 sampled columns against the dequantised oracle."""
    pr = inputs.dense_20k_5k(seed=4)
    X = pr.X
    m, n = X.shape
    ell = 40
    rng = np.random.default_rng(5)
    V = rng.standard_normal((n, ell)).astype(np.float32)
    U = rng.standard_normal((m, ell)).astype(np.float32)
    q = lib.nmf_quantize(ctx, cu(X), prec="fp8")
    Y, Z = lib.nmf_dual_pass(ctx, q, cu(V), cu(U), prec="fp8")
    codes, _, scales = split_copy(q, m, n)
    k = scales.astype(np.int64) - 127
    rows = rng.choice(m, 300, replace=False)
    cols = rng.choice(n, 300, replace=False)
    kr = np.repeat(k, 32, axis=1)[:, :n]                 # tile exponent of every column
    Xr = O.e4m3_decode(codes[rows]) * 2.0 ** kr[rows // 32]
    assert rel(Y.cpu().numpy()[rows], Xr @ bf16(V)) <= 1e-5
    kc = np.repeat(k, 32, axis=0)[:m]                    # tile exponent of every row
    Xc = O.e4m3_decode(codes[:, cols]) * 2.0 ** kc[:, cols // 32]
    assert rel(Z.cpu().numpy()[cols], Xc.T @ bf16(U)) <= 1e-5


def test_fp8_sketch_and_compression_match_the_dequantised_oracle(lib, ctx):
    pr = inputs.random_problem(21, 1200, 900, 10, 20, w=2)
    m, n = pr.X.shape
    q = lib.nmf_quantize(ctx, cu(pr.X), prec="fp8")
    codes, _, scales = split_copy(q, m, n)
    Xq = O.fp8_dequantize(codes, scales.astype(np.int64) - 127)
    QLo, QRo = O.sketch(Xq, pr.omega_L, pr.omega_R, 2)
    Xho, Xco = O.compress(Xq, QLo, QRo)
    for flags, tol in ((lib.FLAG_SIMT_DUAL_PASS, 1e-4), (0, 2e-2)):
        p = lib.params(m, n, pr.r, pr.ell, power_iters=2, prec="fp8", flags=flags)
        QL, QR = lib.nmf_sketch(ctx, p, q, cu(pr.omega_L), cu(pr.omega_R))
        Xhat, Xchk = lib.nmf_compress(ctx, p, q, QL, QR)
        # basis-free forms: Q_L X_hat = Q_L Q_L^T X_q and X_chk Q_R^T = X_q Q_R Q_R^T
        QLh, QRh = QL.double().cpu().numpy(), QR.double().cpu().numpy()
        assert rel(QLh @ Xhat.double().cpu().numpy(), QLo @ Xho) <= tol
        assert rel(Xchk.double().cpu().numpy() @ QRh.T, Xco @ QRo.T) <= tol


def test_fp8_solve_ends_within_one_percent_of_the_oracle(lib, ctx):
    """FP8 sketch, FP32 compression (precision recovery), FastHALS-RP iterations, against the
    oracle taking the same steps in FP64: its own FP8 quantization of X (bit-identical to the
    library's, test_quantize_fp8_is_bit_exact), the sketch of that copy, the compression and the
    residual of X itself. Final relative error within 1 % after the same iterations. (A sketch
    of X itself spans a slightly different subspace, so its unconverged error after 60 iterations
    is no reference for this path.)"""
    pr = inputs.random_problem(31, 1500, 1000, 12, 24, w=2)
    m, n = pr.X.shape
    iters = 60
    p = lib.params(m, n, pr.r, pr.ell, power_iters=2, iters=iters, prec="fp8", seed=5)
    W, H = cu(pr.W0), cu(pr.H0)
    e, it = lib.nmf_solve(ctx, p, cu(pr.X), W, H)
    assert it == iters and (W >= 0).all() and (H >= 0).all()
    oL = O.philox_normal_np(n, pr.ell, 5, 0)
    oR = O.philox_normal_np(m, pr.ell, 5, 1)
    X = pr.X.astype(np.float64)
    Xq = O.fp8_dequantize(*O.fp8_quantize(X))
    QL, QR = O.sketch(Xq, oL, oR, 2)
    Xhat, Xchk = O.compress(X, QL, QR)
    Wo, Ho = O.iterate(pr.W0.astype(np.float64), pr.H0.astype(np.float64), QL, QR, Xhat, Xchk,
                       iters)
    ro = O.residual(X, Wo, Ho)[0]
    assert abs(e - ro) <= 0.01 * ro, f"fp8 {e} vs oracle {ro}"


def test_fp8_arguments_are_checked(lib, ctx):
    pr = inputs.random_problem(5, 300, 200, 4, 10)
    X = cu(pr.X)
    q = lib.nmf_quantize(ctx, X, prec="fp8")
    p = lib.params(300, 200, 4, 10, iters=5, prec="fp8")
    with pytest.raises(ValueError):
        lib.nmf_sketch(ctx, p, X)                      # an FP32 tensor is not the FP8 copy
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_solve_batched(ctx, [p], [X], [cu(pr.W0)], [cu(pr.H0)])
    assert e.value.status == 7                         # FP8 copies are single-solve only
    assert lib.nmf_quantized_bytes("fp8", 300, 200) == O.fp8_layout(300, 200)[2]
    QL, QR = lib.nmf_sketch(ctx, p, q)                 # Omega drawn by the library
    assert torch.isfinite(QL).all() and torch.isfinite(QR).all()
