"""Full-data FastHALS and Lee-Seung MU on the GPU (nmf_iterate_full) against the oracle.

These are the uncompressed methods the paper compares its compressed ones with (Section 2.1
Algorithm 1, Section 2.2; Tables 5.2 and 5.3). FP32 X: one step from the same state within 1e-5
relative (Frobenius) of the oracle's fasthals_step / mu_step, for W, H and W H; 30 steps within
1e-4 on W H (FP32 rounding carried through the sweeps). BF16 X (the nmf_quantize copy, W and H
entering the tensor-core pass as hi + lo pairs): against the oracle on the dequantised copy, the
same 1e-5 / 1e-4 bars. The FastHALS step is also checked to keep W H's error non-increasing on a
planted problem (each block update is an exact minimisation).
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import warmstart_oracle as WS
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


def oracle_step(rule, W, H, X):
    if rule == "fasthals":
        return O.fasthals_step(W, H, X)
    return O.mu_step(W, H, X, eps=1e-12)


SHAPES = [(700, 450, 8), (1999, 1301, 20), (3000, 600, 33), (640, 2048, 48)]


@pytest.mark.parametrize("m,n,r", SHAPES)
@pytest.mark.parametrize("rule", ["fasthals", "mu"])
def test_one_full_step_fp32(lib, ctx, m, n, r, rule):
    pr = inputs.random_problem(81 + r, m, n, r, min(2 * r, 128))
    X = pr.X.astype(np.float64)
    # start from a state of the oracle's own trajectory (away from the U[0,1) start)
    W0, H0 = pr.W0.astype(np.float64), pr.H0.astype(np.float64)
    for _ in range(3):
        W0, H0 = oracle_step(rule, W0, H0, X)
    Wo, Ho = oracle_step(rule, W0, H0, X)
    p = lib.params(m, n, r, min(2 * r, 128), rule=rule)
    W, H = cu(W0), cu(H0)
    lib.nmf_iterate_full(ctx, p, cu(pr.X), W, H, 1)
    Wg, Hg = host(W), host(H)
    assert rel(Wg, Wo) <= 1e-5 and rel(Hg, Ho) <= 1e-5
    assert rel(Wg @ Hg, Wo @ Ho) <= 1e-5


@pytest.mark.parametrize("rule", ["fasthals", "mu"])
def test_thirty_full_steps_fp32_and_bf16(lib, ctx, rule):
    pr = inputs.random_problem(91, 2500, 1700, 16, 32)
    m, n = pr.X.shape
    X = pr.X.astype(np.float64)
    W0, H0 = pr.W0.astype(np.float64), pr.H0.astype(np.float64)
    p32 = lib.params(m, n, 16, 32, rule=rule)
    W, H = cu(W0), cu(H0)
    lib.nmf_iterate_full(ctx, p32, cu(pr.X), W, H, 30)
    Wo, Ho = W0, H0
    for _ in range(30):
        Wo, Ho = oracle_step(rule, Wo, Ho, X)
    assert rel(host(W) @ host(H), Wo @ Ho) <= 1e-4
    # BF16 copy of X on the tensor-core pass: against the oracle on the rounded X
    Xq = lib.nmf_quantize(ctx, cu(pr.X), prec="bf16")
    Xb = WS.bf16_round(pr.X)
    pb = lib.params(m, n, 16, 32, rule=rule, prec="bf16")
    W, H = cu(W0), cu(H0)
    lib.nmf_iterate_full(ctx, pb, Xq, W, H, 1)
    Wb, Hb = oracle_step(rule, W0, H0, Xb)
    assert rel(host(W) @ host(H), Wb @ Hb) <= 1e-5
    W, H = cu(W0), cu(H0)
    lib.nmf_iterate_full(ctx, pb, Xq, W, H, 30)
    Wb, Hb = W0, H0
    for _ in range(30):
        Wb, Hb = oracle_step(rule, Wb, Hb, Xb)
    assert rel(host(W) @ host(H), Wb @ Hb) <= 1e-4


def test_full_fasthals_error_never_increases(lib, ctx):
    pr = inputs.random_problem(93, 1800, 1200, 12, 24)
    m, n = pr.X.shape
    p = lib.params(m, n, 12, 24)
    W, H = cu(pr.W0), cu(pr.H0)
    Xd = cu(pr.X)
    last = lib.nmf_residual(ctx, p, Xd, W, H)[0]
    for _ in range(15):
        lib.nmf_iterate_full(ctx, p, Xd, W, H, 2)
        e = lib.nmf_residual(ctx, p, Xd, W, H)[0]
        assert e <= last * (1 + 1e-5)
        last = e
    assert bool((W >= 0).all()) and bool((H >= 0).all())


def test_full_iterations_reject_bad_arguments(lib, ctx):
    pr = inputs.random_problem(94, 300, 200, 4, 10)
    p = lib.params(300, 200, 65, 65)
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_iterate_full(ctx, p, cu(pr.X), cu(np.zeros((300, 65))), cu(np.zeros((65, 200))), 1)
    assert e.value.status == 7                       # r > 64
    with pytest.raises(ValueError):
        lib.nmf_iterate_full(ctx, lib.params(300, 200, 4, 10), cu(pr.X), cu(pr.W0), cu(pr.W0), 1)
