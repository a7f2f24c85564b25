"""The context-free residual with static scratch against the workspace residual (nmf_residual).

Collected last so that it also runs after every other GPU test in the same process. Two calls in
a row check that the static partial-sum array carries nothing from one call to the next.
Tolerance: both entry points run the same kernels with the same grid, so the sums agree to FP64
rounding (1e-12 relative); the relative error formed from them agrees to 1e-12.
"""
import numpy as np
import pytest
import torch

from paper_1712_02248_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("seed,m,n,r", [(0, 300, 517, 7), (1, 2000, 1500, 20)])
def test_static_residual_matches_workspace_residual(lib, ctx, seed, m, n, r):
    pr = inputs.random_problem(seed, m, n, r, min(2 * r, 128))
    X = torch.from_numpy(np.ascontiguousarray(pr.X, np.float32)).cuda()
    W = torch.from_numpy(pr.W0.astype(np.float32)).cuda()
    H = torch.from_numpy(pr.H0.astype(np.float32)).cuda()
    rel_ws, e2_ws, x2_ws = lib.nmf_residual(ctx, lib.params(m, n, r, min(2 * r, 128)), X, W, H)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        lib.nmf_residual_static(X, W, H, out, stream=ctx.stream)
        ctx.stream.synchronize()
        e2, x2 = out.tolist()
        assert abs(e2 - e2_ws) <= 1e-12 * e2_ws
        assert abs(x2 - x2_ws) <= 1e-12 * x2_ws
        assert abs(np.sqrt(e2 / x2) - rel_ws) <= 1e-12 * rel_ws


def test_static_residual_rejects_bad_arguments(lib):
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    X = torch.ones(4, 4, device="cuda")
    # a rank above the supported maximum is refused before any launch
    with pytest.raises(lib.NmfError):
        lib.nmf_residual_static(X, torch.ones(4, 129, device="cuda"),
                                torch.ones(129, 4, device="cuda"), out)
    # so is an empty X (no rows)
    with pytest.raises(lib.NmfError):
        lib.nmf_residual_static(torch.ones(0, 4, device="cuda"), torch.ones(0, 2, device="cuda"),
                                torch.ones(2, 4, device="cuda"), out)
    # W and H whose shapes do not match X: refused by the binding before the call (the C entry
    # point sees only pointers)
    X = torch.ones(6, 5, device="cuda")
    with pytest.raises(ValueError):
        lib.nmf_residual_static(X, torch.ones(5, 2, device="cuda"), torch.ones(2, 5, device="cuda"),
                                out)
    with pytest.raises(ValueError):
        lib.nmf_residual_static(X, torch.ones(6, 2, device="cuda"), torch.ones(3, 5, device="cuda"),
                                out)
    with pytest.raises(ValueError):
        lib.nmf_residual_static(X, torch.ones(6, 2, device="cuda"), torch.ones(2, 4, device="cuda"),
                                out)
    with pytest.raises(ValueError):
        lib.nmf_residual_static(X, torch.ones(6, 2, device="cuda"), torch.ones(2, 5), out)
