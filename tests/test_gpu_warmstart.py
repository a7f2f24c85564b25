"""Learned warm start: features, network forward / gradient / Adam against the FP64 oracle
(oracle/warmstart_oracle.py), the untrained network's equivalence with NNDSVD, and what a trained
network gains over NNDSVD on held-out matrices.

Tolerances: FP32 network arithmetic against FP64 with the same BF16-rounded weights, 1e-5
relative (forward), 1e-4 (gradients: sums over the batch rows); features from the FP32
eigensolver, 1e-4 on designed inputs with separated singular values.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import warmstart_oracle as WS
from paper_1712_02248_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def designed(seed, m, n, ell, decay):
    rng = np.random.default_rng(seed)
    QL = np.linalg.qr(rng.standard_normal((m, ell)))[0]
    A = np.linalg.qr(rng.standard_normal((ell, ell)))[0]
    B = np.linalg.qr(rng.standard_normal((n, ell)))[0]
    s = decay ** np.arange(ell)
    return QL.astype(np.float32), ((A * s) @ B.T).astype(np.float32), s


@pytest.mark.parametrize("seed,m,n,r,ell", [(0, 1000, 300, 4, 9), (1, 2500, 700, 12, 24)])
def test_features_match_oracle(lib, ctx, seed, m, n, r, ell):
    """Component j carries the FP32 eigensolver's eigenvector error ell * eps32 * lambda_1 /
    gap_j (lambda = s^2, gap_j the distance of lambda_j to its neighbours), as for NNDSVD."""
    QL, Xhat, s = designed(seed, m, n, ell, 0.6)
    p = lib.params(m, n, r, ell)
    Wb, Hb, hs, Fw, Fh = lib.nmf_warmstart_features(ctx, p, cu(QL), cu(Xhat))
    oWb, oHb, ohs, oFw, oFh = WS.warmstart_features(QL, Xhat, r)
    lam = s ** 2
    eps32 = 2.0 ** -24
    for j in range(r):
        gap = min(lam[j - 1] - lam[j] if j > 0 else np.inf, lam[j] - lam[j + 1])
        tol = 1e-5 + ell * eps32 * lam[0] / gap
        assert abs(host(hs)[j] - ohs[j]) <= tol * ohs[j], f"hscale {j}"
        assert rel(host(Wb)[:, j], oWb[:, j]) <= tol, f"W_b column {j}"
        assert rel(host(Hb)[j], oHb[j]) <= tol, f"H_b row {j}"
        for blk in range(3):
            assert rel(host(Fw)[:, blk * r + j], oFw[:, blk * r + j]) <= tol
            assert rel(host(Fh)[:, blk * r + j], oFh[:, blk * r + j]) <= tol


def random_net(seed, F, Hd, r, rows):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(WS.mlp_param_count(F, Hd, r)) * 0.3).astype(np.float32)
    X = rng.standard_normal((rows, F)).astype(np.float32)
    T = rng.standard_normal((rows, r)).astype(np.float32)
    return p, X, T


@pytest.mark.parametrize("F,Hd,r,rows", [(15, 32, 5, 1000), (60, 128, 20, 4099), (3, 8, 1, 65)])
def test_forward_and_gradient_match_oracle(lib, ctx, F, Hd, r, rows):
    p, X, T = random_net(F + Hd + r, F, Hd, r, rows)
    Y = lib.nmf_mlp_forward(ctx, cu(p), cu(X), Hd, r)
    Yo, _ = WS.mlp_forward(p, X, F, Hd, r)
    assert rel(host(Y), Yo) <= 1e-5
    loss, g = lib.nmf_mlp_loss_grad(ctx, cu(p), cu(X), cu(T), Hd, r)
    lo, go = WS.mlp_loss_grad(p, X, T, F, Hd, r)
    assert abs(loss - lo) <= 1e-5 * lo
    gh = host(g)
    sizes = [F * Hd, Hd, Hd * Hd, Hd, Hd * r, r]
    at = 0
    for name, s in zip(["W1", "b1", "W2", "b2", "W3", "b3"], sizes):
        assert rel(gh[at:at + s], go[at:at + s]) <= 1e-4, name
        at += s


def test_adam_steps_match_oracle(lib, ctx):
    rng = np.random.default_rng(7)
    n = 10007
    p = rng.standard_normal(n).astype(np.float32)
    pd, m, v = cu(p), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    po, mo, vo = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        lib.nmf_mlp_adam(ctx, pd, m, v, cu(g), step, 1e-2)
        po, mo, vo = WS.adam_step(po, mo, vo, g.astype(np.float64), step, 1e-2)
    assert rel(host(pd), po) <= 1e-6
    assert rel(host(m), mo) <= 1e-6 and rel(host(v), vo) <= 1e-5


def test_apply_matches_oracle(lib, ctx):
    rng = np.random.default_rng(8)
    m, n, r = 700, 300, 6
    Wb, Hb = rng.random((m, r)), rng.random((r, n))
    hs = rng.random(r) + 0.5
    Dw, Dh = rng.standard_normal((m, r)), rng.standard_normal((n, r))
    W, H = lib.nmf_warmstart_apply(ctx, cu(Wb), cu(Dw), cu(Hb), cu(Dh), cu(hs))
    Wo, Ho = WS.warmstart_apply(Wb.astype(np.float32), Hb.astype(np.float32),
                                hs.astype(np.float32), Dw.astype(np.float32),
                                Dh.astype(np.float32))
    assert rel(host(W), Wo) <= 1e-6 and rel(host(H), Ho) <= 1e-6


def test_targets_match_oracle_and_invert_apply(lib, ctx):
    """nmf_warmstart_targets against the oracle's warmstart_targets (a zero scale included), and
    apply(targets) returns the solution where it is positive (the targets invert the map)."""
    rng = np.random.default_rng(9)
    m, n, r = 900, 333, 7
    Wb, Hb = rng.random((m, r)), rng.random((r, n))
    hs = rng.random(r) + 0.5
    hs[3] = 0.0
    Ws, Hs = rng.random((m, r)) + 0.1, rng.random((r, n)) + 0.1
    f = [a.astype(np.float32) for a in (Wb, Hb, hs, Ws, Hs)]
    Tw, Th = lib.nmf_warmstart_targets(ctx, *[cu(a) for a in f])
    Two, Tho = WS.warmstart_targets(*f)
    assert rel(host(Tw), Two) <= 1e-6 and rel(host(Th), Tho) <= 1e-6
    keep = np.ones(r, bool)
    keep[3] = False                     # a zero scale maps the correction to nothing
    W, H = lib.nmf_warmstart_apply(ctx, cu(f[0]), Tw, cu(f[1]), Th, cu(f[2]))
    assert rel(host(W), f[3]) <= 1e-6
    assert rel(host(H)[keep], f[4][keep]) <= 1e-6


def test_untrained_network_solve_equals_nndsvd_solve(lib, ctx):
    """A zero output layer returns (W_b, H_b), which differ from NNDSVD's factors only by a
    scaling of each component; the FastHALS-RP sweep is equivariant to that scaling, so whole
    solves agree."""
    pr = inputs.random_problem(21, 1500, 800, 10, 20)
    m, n = pr.X.shape
    F, Hd = 30, 64
    z = cu(WS.mlp_init(F, Hd, 10, seed=3))
    lib.nmf_set_warmstart(ctx, Hd, 10, z, z)
    X = cu(pr.X)
    p = lib.params(m, n, 10, 20, power_iters=2, iters=60, seed=4)
    out = {}
    for init in ("nndsvd", "mlp"):
        W = torch.empty((m, 10), device="cuda")
        H = torch.empty((10, n), device="cuda")
        out[init] = lib.nmf_solve(ctx, p, X, W, H, init=init)[0]
    assert abs(out["mlp"] - out["nndsvd"]) <= 1e-4 * out["nndsvd"]


def test_solve_without_network_is_refused(lib, ctx):
    pr = inputs.random_problem(22, 300, 200, 4, 10)
    p = lib.params(300, 200, 4, 10, iters=5)
    with pytest.raises(lib.NmfError):
        lib.nmf_solve(ctx, p, cu(pr.X), cu(pr.W0), cu(pr.H0), init="mlp")


def test_trained_warm_start_gain_over_nndsvd(lib, ctx):
    """Train both networks on 48 planted 1024 x 256 (r = 8) matrices through the library's own
    kernels; on 12 held-out matrices report iterations to 1.01 x the error of a 600-iteration
    NNDSVD-started solve for random, NNDSVD and learned starts. The training loss must fall
    below the targets' variance (the networks explain part of the correction), the learned start
    must begin closer than NNDSVD and need fewer iterations than NNDSVD on average."""
    from paper_1712_02248_gb300 import warmstart as WSM
    cfg = WSM.WarmStartConfig(m=1024, n=256, r=8, ell=16, noise=0.02, steps=800)
    pw, ph, info = WSM.train_warmstart(ctx, cfg, count=48, seed=5)
    assert info["loss_w"][-1][1] < 0.9 * info["target_var_w"]
    assert info["loss_h"][-1][1] < 0.9 * info["target_var_h"]
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev)
    gen.manual_seed(77)
    its = {"random": [], "nndsvd": [], "mlp": []}
    e0 = {"random": [], "nndsvd": [], "mlp": []}
    for k in range(12):
        X = WSM.planted(cfg.m, cfg.n, cfg.r, cfg.noise, gen, dev)
        p, QL, QR, Xhat, Xchk = WSM.compressed(ctx, cfg, X, 900 + k)
        Wb, Hb, hs, Fw, Fh = lib.nmf_warmstart_features(ctx, p, QL, Xhat)
        Wr, Hr = Wb.clone(), Hb.clone()
        lib.nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, Wr, Hr, 600)
        ref = lib.nmf_residual(ctx, p, X, Wr, Hr)[0]
        Dw = lib.nmf_mlp_forward(ctx, pw, Fw, cfg.hidden, cfg.r)
        Dh = lib.nmf_mlp_forward(ctx, ph, Fh, cfg.hidden, cfg.r)
        starts = {"random": (torch.rand(cfg.m, cfg.r, device=dev, generator=gen),
                             torch.rand(cfg.r, cfg.n, device=dev, generator=gen)),
                  "nndsvd": (Wb.clone(), Hb.clone()),
                  "mlp": lib.nmf_warmstart_apply(ctx, Wb, Dw, Hb, Dh, hs)}
        for name, (W, H) in starts.items():
            e0[name].append(lib.nmf_residual(ctx, p, X, W, H)[0])
            it = WSM.iterations_to_target(ctx, p, X, QL, QR, Xhat, Xchk, W, H, 1.01 * ref,
                                          every=10, max_iters=600)
            its[name].append(600 if it is None else it)
    summary = {k: (float(np.median(e0[k])), float(np.mean(v))) for k, v in its.items()}
    print("initial error (median), iterations to target (mean):", summary)
    assert summary["mlp"][0] < summary["nndsvd"][0]
    assert summary["mlp"][1] < summary["nndsvd"][1]
