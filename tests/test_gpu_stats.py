"""The Gini coefficient of a factor on the GPU (Section 5.1) against the oracle.

nmf_gini sorts on the device and sums in FP64, so it agrees with the oracle's sort-based formula
to FP64 rounding (1e-11 absolute: G lies in [0, 1]) on inputs with ties, exact zeros, negative
values and sizes that are not powers of two, from one entry to several million. The α-weighted
FastHALS-RP solves (Section 4.1) then show the sparsity effect of Figure 5.4a on the device: the
Gini of H from the GPU solve equals the oracle's Gini of that H, follows the oracle's own solve
to 2e-3, and grows with α.
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


def cases():
    rng = np.random.default_rng(71)
    e = rng.exponential(1.0, (37, 1000)).astype(np.float32)
    e[rng.random(e.shape) < 0.6] = 0.0                      # exact zeros: ties at the bottom
    yield "sparse exponential", e
    yield "few levels", rng.integers(0, 4, 5001).astype(np.float32)   # many ties, ragged size
    yield "one entry", np.array([3.5], np.float32)
    yield "2048 entries", rng.random(2048).astype(np.float32)
    yield "signed", rng.standard_normal(4097).astype(np.float32) + 0.5
    yield "all zero", np.zeros(300, np.float32)
    big = rng.exponential(1.0, 3_300_001).astype(np.float32)
    big[rng.random(big.size) < 0.3] = 0.0
    yield "3.3M entries", big


@pytest.mark.parametrize("name,B", list(cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_gini_matches_oracle(lib, ctx, name, B):
    g = lib.nmf_gini(ctx, cu(B))
    want = O.gini(B.astype(np.float64))
    assert abs(g - want) <= 1e-11, f"{name}: {g} vs {want}"


def test_gini_rejects_non_finite(lib, ctx):
    B = np.ones(100, np.float32)
    B[7] = np.nan
    with pytest.raises(lib.NmfError) as e:
        lib.nmf_gini(ctx, cu(B))
    assert e.value.status == 5


def test_gini_of_alpha_regularised_solves(lib, ctx):
    """Section 4.1 / Figure 5.4a: FastHALS-RP with the sparsity weight alpha on H, from the same
    sketch and start on both sides; the Gini of the GPU's H against the oracle's Gini of the same
    H (1e-11) and of the oracle's own solve (2e-3), growing with alpha."""
    pr = inputs.planted_exp(73, m=1200, n=900, r=10, ell=20, w=2, noise=0.05)
    m, n = pr.X.shape
    X = pr.X.astype(np.float64)
    QL, QR = O.sketch(X, pr.omega_L, pr.omega_R, pr.w)
    Xhat, Xchk = O.compress(X, QL, QR)
    scale = float(np.mean(X)) * m      # alpha in units of a typical column sum of X
    ginis = []
    for a in (0.0, 1e-3, 1e-2):      # (at 1e-1 every entry of H is driven to zero)
        alpha = a * scale
        p = lib.params(m, n, pr.r, pr.ell, alpha=alpha)
        W, H = cu(pr.W0), cu(pr.H0)
        lib.nmf_iterate(ctx, p, cu(QL), cu(QR), cu(Xhat), cu(Xchk), W, H, 60)
        g = lib.nmf_gini(ctx, H)
        Hh = H.double().cpu().numpy()
        assert abs(g - O.gini(Hh)) <= 1e-11
        _, Ho = O.iterate(pr.W0, pr.H0, QL, QR, Xhat, Xchk, 60, alpha=alpha)
        go = O.gini(Ho)
        print(f"alpha {alpha:.4g}: gini gpu {g:.6f} oracle {go:.6f}")
        assert abs(g - go) <= 2e-3
        ginis.append(g)
    assert ginis[-1] > ginis[0] + 0.2
    assert all(b >= a - 1e-3 for a, b in zip(ginis, ginis[1:]))


def test_spectrum_matches_oracle(lib, ctx):
    """Singular values of X_hat (Section 3, Eq. 3.4) from the Gram and the FP32 Jacobi solver:
    within ell * 2.4e-7 * sigma_1^2 / (2 sigma_j) + 1e-6 sigma_j of the LAPACK values (the
    eigenvalue error bound of the header, carried through the square root), and the decay rate
    fitted over the values above 1e-2 sigma_1 within 1e-3 relative of the oracle's."""
    pr = inputs.images(seed=5, n_samples=6000, r=30, ell=48)
    X = pr.X.astype(np.float64)
    QL, QR = O.sketch(X, pr.omega_L, pr.omega_R, pr.w)
    Xhat, _ = O.compress(X, QL, QR)
    s = np.array(lib.nmf_spectrum(ctx, cu(Xhat)))
    want = O.spectrum(Xhat)
    ell = Xhat.shape[0]
    tol = ell * 2.4e-7 * want[0] ** 2 / (2 * np.maximum(want, 1e-30)) + 1e-6 * want
    assert np.all(np.abs(s - want) <= tol), np.max(np.abs(s - want) / tol)
    p_gpu = lib.nmf_decay_rate(s, 1e-2)
    p_or = O.decay_rate(want, 1e-2)
    print(f"decay rate: gpu {p_gpu:.6g} oracle {p_or:.6g}")
    assert abs(p_gpu - p_or) <= 1e-3 * p_or
