"""Training and evaluation of the learned warm start (include/nmf_rp.h: nmf_set_warmstart).

All device work, the library's and PyTorch's, is queued on the context's stream. Everything on the
device goes through the library's C ABI: the sketch, compression, warm-start
features, the iterations that produce the training targets, the network's forward and backward
passes and Adam. PyTorch only holds device memory and draws the synthetic training matrices.

Training set. Planted matrices X = max(0, W0 H0 + noise * rms(W0 H0) N(0,1)) with Exp(1) factors
(the distribution of the dense workloads); for each: two-sided sketch and compression, the
features (W_b, H_b, hscale, F_w, F_h) and a short compressed-NMF run started from (W_b, H_b)
(10 iterations by default); the targets map (W_b, H_b) onto where that run ends (D_w = sqrt(m)
(W* - W_b), D_h = sqrt(n) (H* - H_b) / hscale). A fixed number of random rows and columns of
each matrix enter the set. Targets from converged solves (hundreds of iterations) lower the
starting error as much but make the later iterations slower: the network then predicts an
average over the solutions a row can end in.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import nmf_rp as N


@dataclasses.dataclass
class WarmStartConfig:
    m: int = 2048
    n: int = 512
    r: int = 16
    ell: int = 32
    power_iters: int = 2
    noise: float = 0.02
    prec: str = "fp32"
    target_iters: int = 10       # iterations from the NNDSVD start that give the targets
    rows_per_matrix: int = 256   # sampled rows of W (and columns of H) per matrix
    hidden: int = 128
    steps: int = 1500
    batch: int = 4096
    lr: float = 2e-3


def planted(m, n, r, noise, gen, device):
    """X = max(0, W0 H0 + noise rms(W0 H0) N(0,1)), W0, H0 entries Exp(1)."""
    # 1 - U lies in (0, 1]: -log never sees the zero that torch.rand can return
    W0 = -torch.log1p(-torch.rand(m, r, device=device, generator=gen))
    H0 = -torch.log1p(-torch.rand(r, n, device=device, generator=gen))
    Y = W0 @ H0
    rms = Y.pow(2).mean().sqrt()
    return torch.clamp(Y + noise * rms * torch.randn(m, n, device=device, generator=gen), min=0)


def compressed(ctx, cfg, X, seed):
    p = N.params(cfg.m, cfg.n, cfg.r, cfg.ell, power_iters=cfg.power_iters, prec=cfg.prec,
                 seed=seed)
    Xp = N.nmf_quantize(ctx, X) if cfg.prec == "bf16" else X
    QL, QR = N.nmf_sketch(ctx, p, Xp)
    Xhat, Xchk = N.nmf_compress(ctx, p, Xp, QL, QR)
    return p, QL, QR, Xhat, Xchk


def make_training_set(ctx, cfg, count, seed):
    """(F_w, T_w, F_h, T_h) device tensors from `count` planted matrices."""
    with torch.cuda.stream(ctx.stream):   # torch work ordered with the library's on one stream
        return _make_training_set(ctx, cfg, count, seed)


def _make_training_set(ctx, cfg, count, seed):
    dev = ctx.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    k = cfg.rows_per_matrix
    Fws, Tws, Fhs, Ths = [], [], [], []
    for i in range(count):
        X = planted(cfg.m, cfg.n, cfg.r, cfg.noise, gen, dev)
        p, QL, QR, Xhat, Xchk = compressed(ctx, cfg, X, seed * 100003 + i)
        Wb, Hb, hs, Fw, Fh = N.nmf_warmstart_features(ctx, p, QL, Xhat)
        W, H = Wb.clone(), Hb.clone()
        N.nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, W, H, cfg.target_iters)
        N.nmf_sync(ctx)   # a latched device error surfaces with the matrix that raised it
        Tw, Th = N.nmf_warmstart_targets(ctx, Wb, Hb, hs, W, H)
        iw = torch.randint(0, cfg.m, (k,), device=dev, generator=gen)
        ih = torch.randint(0, cfg.n, (k,), device=dev, generator=gen)
        Fws.append(Fw[iw])
        Tws.append(Tw[iw])
        Fhs.append(Fh[ih])
        Ths.append(Th[ih])
    return (torch.cat(Fws).contiguous(), torch.cat(Tws).contiguous(),
            torch.cat(Fhs).contiguous(), torch.cat(Ths).contiguous())


def init_params(F, hidden, r, seed, device):
    """He-uniform hidden layers, zero output layer: the untrained network returns NNDSVD."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (F, hidden)) * np.sqrt(6.0 / F)
    W2 = rng.uniform(-1, 1, (hidden, hidden)) * np.sqrt(6.0 / hidden)
    v = np.concatenate([W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(hidden),
                        np.zeros(hidden * r), np.zeros(r)]).astype(np.float32)
    return torch.from_numpy(v).to(device)


def train_network(ctx, F, T, cfg, seed):
    """Adam on minibatches of the (features, targets) pairs; returns (params, loss history)."""
    with torch.cuda.stream(ctx.stream):
        return _train_network(ctx, F, T, cfg, seed)


def _train_network(ctx, F, T, cfg, seed):
    dev = ctx.device
    r = T.shape[1]
    params = init_params(F.shape[1], cfg.hidden, r, seed, dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    hist = []
    for step in range(1, cfg.steps + 1):
        idx = torch.randint(0, F.shape[0], (min(cfg.batch, F.shape[0]),), device=dev, generator=gen)
        want = step == 1 or step % 100 == 0 or step == cfg.steps
        loss = N.nmf_mlp_train_step(ctx, params, m, v, grad, step, cfg.lr, F[idx].contiguous(),
                                    T[idx].contiguous(), cfg.hidden, r, want_loss=want)
        if want:
            hist.append((step, loss))
    return params, hist


def train_warmstart(ctx, cfg, count, seed=0):
    """Train both networks; returns (params_w, params_h, info)."""
    Fw, Tw, Fh, Th = make_training_set(ctx, cfg, count, seed)
    pw, hw = train_network(ctx, Fw, Tw, cfg, seed + 1)
    ph, hh = train_network(ctx, Fh, Th, cfg, seed + 2)
    return pw, ph, {"samples": int(Fw.shape[0]), "loss_w": hw, "loss_h": hh,
                    "target_var_w": float(Tw.pow(2).mean()), "target_var_h": float(Th.pow(2).mean())}


def iterations_to_target(ctx, p, X, QL, QR, Xhat, Xchk, W, H, target, every=10, max_iters=1000):
    """Iterations (multiples of `every`) until the exact relative residual is <= target."""
    done = 0
    while done < max_iters:
        N.nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, W, H, every)
        done += every
        if N.nmf_residual(ctx, p, X, W, H)[0] <= target:
            return done
    return None
