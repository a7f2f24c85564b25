"""Failure detection without a GPU fault, and the error monitor's terms against the oracle.

Time-outs: the persistent iteration kernel bounds every grid-barrier wait. The test gives the
context a budget of one SM cycle (nmf_set_wait_limit), so the first barrier runs out in every
block but the last to arrive; the kernel latches NMF_ERR_TIMEOUT, raises its abort flag and every
block leaves (no asynchronous copies are in flight in that kernel). The next synchronising call
reports the status; the context then runs the same iterations cleanly with the default budget.
Nothing waits without a limit, nothing traps.

Non-finite input: a NaN or an infinity planted in X on the host is reported as
NMF_ERR_NOT_FINITE by nmf_residual and by nmf_solve (from ||X||^2), and the context stays usable.

Monitor (Section 3, Eq. 3.4): the cross and quadratic terms the persistent kernel leaves after
its last iteration equal the oracle's <W_tld^T X_hat, H> and <W^T W, H H^T> at the returned
factors (FP32 sums: 1e-5 relative); ||X||^2 and the BF16 copy's rounding term <X - X_q, X> of a
solve equal the oracle's plain FP64 sums (1e-9 and 1e-4 relative: the rounding term is a sum of
terms of both signs, formed in FP32 products).
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import warmstart_oracle as WS
from paper_1712_02248_gb300 import inputs

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda")


@pytest.fixture
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


def oracle_state(pr):
    QL, QR = O.sketch(pr.X.astype(np.float64), pr.omega_L, pr.omega_R, pr.w)
    Xhat, Xchk = O.compress(pr.X.astype(np.float64), QL, QR)
    return QL, QR, Xhat, Xchk


def test_grid_barrier_timeout_is_reported_and_context_recovers(lib, ctx):
    pr = inputs.random_problem(51, 3000, 1200, 12, 24)
    m, n = pr.X.shape
    QL, QR, Xhat, Xchk = (cu(a) for a in oracle_state(pr))
    p = lib.params(m, n, pr.r, pr.ell)
    lib.nmf_set_wait_limit(ctx, 1)
    W, H = cu(pr.W0), cu(pr.H0)
    lib.nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, W, H, 5)
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_sync(ctx)
    assert e.value.status == 6                      # NMF_ERR_TIMEOUT
    lib.nmf_sync(ctx)                               # the status was cleared by the report
    lib.nmf_set_wait_limit(ctx, 0)
    W, H = cu(pr.W0), cu(pr.H0)
    lib.nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, W, H, 5)
    lib.nmf_sync(ctx)
    Wo, Ho = O.iterate(pr.W0, pr.H0, *oracle_state(pr)[:4], 5)
    got = W.double().cpu().numpy() @ H.double().cpu().numpy()
    assert np.linalg.norm(got - Wo @ Ho) <= 1e-5 * np.linalg.norm(Wo @ Ho)
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_set_wait_limit(ctx, -1)
    assert e.value.status == 1


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_x_is_reported(lib, ctx, prec, bad):
    pr = inputs.random_problem(52, 900, 700, 6, 16)
    m, n = pr.X.shape
    Xbad = pr.X.copy()
    Xbad[417, 233] = bad
    p = lib.params(m, n, pr.r, pr.ell, iters=20, residual_every=10, prec=prec, seed=3)
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_solve(ctx, p, cu(Xbad), cu(pr.W0), cu(pr.H0))
    assert e.value.status == 5                      # NMF_ERR_NOT_FINITE
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_residual(ctx, p, cu(Xbad), cu(pr.W0), cu(pr.H0))
    assert e.value.status == 5
    # the context is still usable: the clean X solves and matches the oracle's residual
    W, H = cu(pr.W0), cu(pr.H0)
    rel, it = lib.nmf_solve(ctx, p, cu(pr.X), W, H)
    assert it == 20 and np.isfinite(rel)
    ro = O.residual(pr.X, W.double().cpu().numpy(), H.double().cpu().numpy())[0]
    assert abs(rel - ro) <= 1e-6 * ro


@pytest.mark.parametrize("rule", ["fasthals", "mu"])
def test_monitor_terms_match_oracle(lib, ctx, rule):
    pr = inputs.random_problem(53, 4000, 1500, 16, 32)
    m, n = pr.X.shape
    QL, QR, Xhat, Xchk = oracle_state(pr)
    p = lib.params(m, n, pr.r, pr.ell, rule=rule)
    W, H = cu(pr.W0), cu(pr.H0)
    lib.nmf_iterate(ctx, p, cu(QL), cu(QR), cu(Xhat), cu(Xchk), W, H, 7)
    cross, quad, _, _ = lib.nmf_monitor_terms(ctx)
    Wg, Hg = W.double().cpu().numpy(), H.double().cpu().numpy()
    want_cross = float(np.sum(((QL.T @ Wg).T @ Xhat) * Hg))
    want_quad = float(np.sum((Wg.T @ Wg) * (Hg @ Hg.T)))
    assert abs(cross - want_cross) <= 1e-5 * abs(want_cross)
    assert abs(quad - want_quad) <= 1e-5 * abs(want_quad)
    # the three terms and ||X||^2 give the oracle's compressed estimate
    x2 = float(np.sum(pr.X.astype(np.float64) ** 2))
    est = x2 - 2 * cross + quad
    assert abs(est - O.compressed_sq_error(x2, QL, Xhat, Wg, Hg)) <= 1e-5 * x2


def test_solve_sums_of_x_match_oracle(lib, ctx):
    pr = inputs.random_problem(54, 2500, 1700, 10, 20)
    m, n = pr.X.shape
    X = pr.X.astype(np.float64)
    x2_want = float(np.sum(X * X))
    for prec in ("fp32", "bf16"):
        p = lib.params(m, n, pr.r, pr.ell, iters=10, prec=prec, seed=8)
        lib.nmf_solve(ctx, p, cu(pr.X), cu(pr.W0), cu(pr.H0))
        _, _, x2, rt = lib.nmf_monitor_terms(ctx)
        assert abs(x2 - x2_want) <= 1e-9 * x2_want
        if prec == "bf16":
            want = O.rounding_term(X, WS.bf16_round(pr.X))
            assert want != 0.0
            assert abs(rt - want) <= 1e-4 * abs(want), (rt, want)
        else:
            assert rt == 0.0
