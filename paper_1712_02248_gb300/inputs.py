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
  sparse_counts   topic-model term counts in CSR form (documents x words), for the sparse path

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


@dataclasses.dataclass
class SparseProblem:
    row_ptr: np.ndarray    # m + 1 int64
    col: np.ndarray        # nnz int32 (increasing within a row)
    val: np.ndarray        # nnz float32 counts
    shape: tuple
    r: int
    ell: int
    w: int
    omega_L: np.ndarray    # n x ell float32
    omega_R: np.ndarray    # m x ell float32
    W0: np.ndarray         # m x r float32
    H0: np.ndarray         # r x n float32
    seed: int

    def dense(self):
        """The m x n matrix as a dense float64 array (small problems only)."""
        m, n = self.shape
        X = np.zeros((m, n))
        rows = np.repeat(np.arange(m), np.diff(self.row_ptr))
        X[rows, self.col] = self.val
        return X


def sparse_counts(seed=0, m=5000, n=1000, r=60, ell=72, w=9, topics=20, mean_len=100,
                  alpha=0.1):
    """Term-count matrix of m documents over n words drawn from a topic model (stands in for the
    20 Newsgroups frequency matrix of Section 5.2, not available here): word popularity
    ~ 1 / (rank + 10), each of `topics` topics boosts a random 5 % of the words by Exp(1) x 20;
    a document draws its length from Poisson(mean_len), its topic mix from Dirichlet(alpha) and
    each word from its topic. Rows with no words and words never drawn stay empty."""
    rng = np.random.default_rng(seed)
    base = 1.0 / (np.arange(n) + 10.0)
    base = base[rng.permutation(n)]
    T = np.tile(base, (topics, 1))
    for t in range(topics):
        pick = rng.random(n) < 0.05
        T[t, pick] *= 20.0 * rng.exponential(1.0, pick.sum())
    T /= T.sum(axis=1, keepdims=True)
    cumT = np.cumsum(T, axis=1)
    theta = rng.dirichlet(np.full(topics, alpha), size=m)
    cumth = np.cumsum(theta, axis=1)
    lens = rng.poisson(mean_len, size=m)
    doc = np.repeat(np.arange(m), lens)
    u = rng.random(doc.size)
    topic = np.empty(doc.size, dtype=np.int64)
    for c in range(0, doc.size, 1 << 20):          # (tokens x topics) comparisons in chunks
        sl = slice(c, c + (1 << 20))
        topic[sl] = np.minimum((u[sl, None] > cumth[doc[sl]]).sum(axis=1), topics - 1)
    word = np.empty(doc.size, dtype=np.int64)
    u2 = rng.random(doc.size)
    for t in range(topics):
        sel = topic == t
        word[sel] = np.minimum(np.searchsorted(cumT[t], u2[sel]), n - 1)
    keys, counts = np.unique(doc * n + word, return_counts=True)
    rows = keys // n
    col = (keys % n).astype(np.int32)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    omega_L, omega_R, W0, H0 = _init_and_omega(rng, m, n, r, ell)
    return SparseProblem(row_ptr, col, counts.astype(np.float32), (m, n), r, ell, w, omega_L,
                         omega_R, W0, H0, seed)


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
