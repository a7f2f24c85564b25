"""Seeded synthetic inputs for compressed NMF, shared by the tests, the bench and the smoke run.

This module holds none of the method's arithmetic: it only draws data matrices, Gaussian test
matrices and initial factors with numpy's PCG64 generator, in a fixed draw order, so that the
CUDA path and the CPU oracle can be fed bit-identical inputs.

Workloads (shapes of the paper's problem, Section 2, Eq. 2.1: X ~ W H, X non-negative m x n):

  planted_small   512 x 256, r = 8: W0, H0 entries |N(0,1)|, X = W0 H0 + U[0, 0.01)
  dense_20k_5k    20000 x 5000, r = 20: W0, H0 Exp(1), X = max(0, W0 H0 + 0.01 rms(W0 H0) N(0,1))
  images_4k_100k  4096 x 100000, r = 50: 64x64 Gaussian-blob parts, Exp(1) mixing weights with
                  70 % zeroed, 256-level Poisson-like noise (image-like data as in Section 5.1)
  planted_batch   independent planted problems with m, n, r drawn uniformly from ranges
  planted_warm    8192 x 2048, r = 16, Exp(1) factors + 2 % Gaussian noise

The Gaussian test matrices Omega_L (n x l) and Omega_R (m x l) of Section 3 and the U[0, 1)
initial factors are drawn here too (the paper: Omega ~ N(0,1); random initialisation).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Problem:
    X: np.ndarray          # m x n float32, row-major, non-negative
    r: int
    ell: int
    w: int
    omega_L: np.ndarray    # n x ell float32
    omega_R: np.ndarray    # m x ell float32
    W0: np.ndarray         # m x r float32 initial factor
    H0: np.ndarray         # r x n float32 initial factor
    seed: int
    name: str = ""


def _init_and_omega(rng, m, n, r, ell):
    omega_L = rng.standard_normal((n, ell), dtype=np.float32)
    omega_R = rng.standard_normal((m, ell), dtype=np.float32)
    W0 = rng.random((m, r), dtype=np.float32)
    H0 = rng.random((r, n), dtype=np.float32)
    return omega_L, omega_R, W0, H0


def planted_small(seed=0, m=512, n=256, r=8, oversample=10, w=2):
    """X = W0 H0 + E, W0 (m x r), H0 (r x n) entries |N(0,1)|, E uniform [0, 0.01)."""
    rng = np.random.default_rng(seed)
    Wt = np.abs(rng.standard_normal((m, r)))
    Ht = np.abs(rng.standard_normal((r, n)))
    E = rng.uniform(0.0, 0.01, size=(m, n))
    X = (Wt @ Ht + E).astype(np.float32)
    ell = r + oversample
    oL, oR, W0, H0 = _init_and_omega(rng, m, n, r, ell)
    return Problem(X, r, ell, w, oL, oR, W0, H0, seed, f"planted_small_{m}x{n}_r{r}")


def planted_exp(seed=0, m=20000, n=5000, r=20, ell=40, w=2, noise=0.01, name="dense"):
    """X = max(0, W0 H0 + noise * rms(W0 H0) * N(0,1)), W0, H0 entries Exp(1).

    Generated in row blocks so that the FP64 temporaries stay small at 20000 x 5000."""
    rng = np.random.default_rng(seed)
    Wt = rng.exponential(1.0, size=(m, r))
    Ht = rng.exponential(1.0, size=(r, n))
    # rms of W0 H0, accumulated exactly over row blocks
    X = np.empty((m, n), dtype=np.float32)
    blk = 2048
    ss = 0.0
    for i in range(0, m, blk):
        P = Wt[i:i + blk] @ Ht
        ss += float(np.sum(P * P))
    rms = np.sqrt(ss / (m * n))
    sigma = noise * rms
    for i in range(0, m, blk):
        P = Wt[i:i + blk] @ Ht
        Z = rng.standard_normal(P.shape)
        X[i:i + blk] = np.maximum(0.0, P + sigma * Z).astype(np.float32)
    oL, oR, W0, H0 = _init_and_omega(rng, m, n, r, ell)
    return Problem(X, r, ell, w, oL, oR, W0, H0, seed, f"{name}_{m}x{n}_r{r}")


def dense_20k_5k(seed=0, m=20000, n=5000):
    return planted_exp(seed, m=m, n=n, r=20, ell=40, w=2, noise=0.01, name="dense")


def planted_warm(seed=0, m=8192, n=2048):
    return planted_exp(seed, m=m, n=n, r=16, ell=32, w=2, noise=0.02, name="warm")


def images(seed=0, n_samples=100000, side=64, r=50, ell=70, w=3, parts=50):
    """Image-like X: features = side*side pixels (rows) x samples (columns), values in [0, 1].

    Each of `parts` parts is a Gaussian blob (centre U[0, side)^2, sigma U[2, 8] px) scaled to max
    1. Each sample mixes the parts with Exp(1) weights of which 70 % are zeroed, is scaled to max
    1, and is quantised with Poisson noise at 255 counts (256 grey levels)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64)
    B = np.empty((side * side, parts))
    for p in range(parts):
        cy, cx = rng.uniform(0, side, size=2)
        s = rng.uniform(2.0, 8.0)
        g = np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s))
        B[:, p] = (g / g.max()).ravel()
    m = side * side
    X = np.empty((m, n_samples), dtype=np.float32)
    blk = 8192
    for c in range(0, n_samples, blk):
        k = min(blk, n_samples - c)
        Wm = rng.exponential(1.0, size=(parts, k))
        Wm[rng.random((parts, k)) < 0.7] = 0.0
        clean = B @ Wm
        mx = clean.max(axis=0)
        mx[mx == 0] = 1.0
        clean /= mx[None, :]
        X[:, c:c + k] = np.minimum(1.0, rng.poisson(255.0 * clean) / 255.0).astype(np.float32)
    oL, oR, W0, H0 = _init_and_omega(rng, m, n_samples, r, ell)
    return Problem(X, r, ell, w, oL, oR, W0, H0, seed, f"images_{m}x{n_samples}_r{r}")


def batch_specs(count=256, seed=0, m_range=(500, 8000), n_range=(200, 3000), r_range=(5, 40),
                oversample=10):
    """Shapes of `count` independent problems with m, n, r uniform in the given ranges."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        r = int(rng.integers(r_range[0], r_range[1] + 1))
        out.append((m, n, r, min(r + oversample, m, n)))
    return out


def random_problem(seed, m, n, r, ell, w=2, noise=0.01):
    """Small planted problem of arbitrary shape (ragged sizes for parity tests)."""
    return planted_exp(seed, m=m, n=n, r=r, ell=ell, w=w, noise=noise, name="rand")
