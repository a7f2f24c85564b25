"""Python binding of libnmf_rp.so (include/nmf_rp.h): argument marshalling only.

Every function has the name of the C entry point it calls and takes torch CUDA tensors; outputs
the caller does not pass are allocated with torch on the tensors' device. Nothing here computes
any step of the method: each call goes straight to the library's CUDA kernels. Importing this
module loads the library and raises ImportError if it has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnmf_rp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1712_02248_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)

NMF_OK = 0
STATUS = {0: "NMF_OK", 1: "NMF_ERR_INVALID_ARG", 2: "NMF_ERR_CUDA", 3: "NMF_ERR_OOM",
          4: "NMF_ERR_QR_BREAKDOWN", 5: "NMF_ERR_NOT_FINITE", 6: "NMF_ERR_TIMEOUT",
          7: "NMF_ERR_UNSUPPORTED"}
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
RULE = {"fasthals": 0, "mu": 1}
INIT = {"given": 0, "nndsvd": 1, "mlp": 2}

EXPORTS = ["nmf_create", "nmf_destroy", "nmf_set_stream", "nmf_last_error", "nmf_sync",
           "nmf_launch_count", "nmf_workspace_size", "nmf_gaussian", "nmf_quantize",
           "nmf_dual_pass", "nmf_qr", "nmf_sketch", "nmf_compress", "nmf_iterate",
           "nmf_residual", "nmf_residual_static", "nmf_nndsvd", "nmf_solve", "nmf_set_profiling", "nmf_phase_times",
           "nmf_last_solve_info", "nmf_solve_batched", "nmf_last_batch_info",
           "nmf_mlp_param_count", "nmf_warmstart_features", "nmf_mlp_forward",
           "nmf_mlp_loss_grad", "nmf_mlp_adam", "nmf_mlp_train_step", "nmf_warmstart_apply",
           "nmf_set_warmstart", "nmf_quantized_bytes", "nmf_set_wait_limit",
           "nmf_monitor_terms", "nmf_gini", "nmf_iterate_full", "nmf_spectrum",
           "nmf_decay_rate", "nmf_sketch_csr", "nmf_compress_csr", "nmf_residual_csr",
           "nmf_solve_csr", "nmf_warmstart_targets"]
PHASES = ["quantize", "dual_pass", "qr", "iterate", "residual", "init"]


class nmf_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("r", ctypes.c_int32),
                ("ell", ctypes.c_int32), ("power_iters", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("rule", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("residual_every", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("target_rel_err", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("eps", ctypes.c_double)]


_vp, _i64, _i32, _u64, _u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32
_P = ctypes.POINTER(nmf_params)
_D = ctypes.POINTER(ctypes.c_double)


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_c = {
    "nmf_create": _sig("nmf_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "nmf_destroy": _sig("nmf_destroy", None, [_vp]),
    "nmf_set_stream": _sig("nmf_set_stream", ctypes.c_int, [_vp, _vp]),
    "nmf_last_error": _sig("nmf_last_error", ctypes.c_char_p, [_vp]),
    "nmf_sync": _sig("nmf_sync", ctypes.c_int, [_vp]),
    "nmf_launch_count": _sig("nmf_launch_count", _i64, [_vp]),
    "nmf_workspace_size": _sig("nmf_workspace_size", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "nmf_gaussian": _sig("nmf_gaussian", ctypes.c_int, [_vp, _i64, _i64, _u64, _u32, _vp]),
    "nmf_quantize": _sig("nmf_quantize", ctypes.c_int, [_vp, _i32, _vp, _i64, _i64, _i64, _vp]),
    "nmf_quantized_bytes": _sig("nmf_quantized_bytes", ctypes.c_size_t, [_i32, _i64, _i64]),
    "nmf_dual_pass": _sig("nmf_dual_pass", ctypes.c_int,
                          [_vp, _i32, _vp, _i64, _i64, _i64, _i32, _vp, _vp, _vp, _vp]),
    "nmf_qr": _sig("nmf_qr", ctypes.c_int, [_vp, _vp, _i64, _i32, _vp]),
    "nmf_sketch": _sig("nmf_sketch", ctypes.c_int, [_vp, _P, _vp, _i64, _vp, _vp, _vp, _vp]),
    "nmf_compress": _sig("nmf_compress", ctypes.c_int, [_vp, _P, _vp, _i64, _vp, _vp, _vp, _vp]),
    "nmf_iterate": _sig("nmf_iterate", ctypes.c_int, [_vp, _P, _vp, _vp, _vp, _vp, _vp, _vp, _i32]),
    "nmf_residual": _sig("nmf_residual", ctypes.c_int, [_vp, _P, _vp, _i64, _vp, _vp, _D, _D, _D]),
    "nmf_nndsvd": _sig("nmf_nndsvd", ctypes.c_int, [_vp, _P, _vp, _vp, _vp, _vp]),
    "nmf_residual_static": _sig("nmf_residual_static", ctypes.c_int,
                                [_i32, _vp, _vp, _i64, _i64, _i64, _i32, _vp, _vp, _vp]),
    "nmf_set_profiling": _sig("nmf_set_profiling", ctypes.c_int, [_vp, _i32]),
    "nmf_set_wait_limit": _sig("nmf_set_wait_limit", ctypes.c_int, [_vp, _i64]),
    "nmf_monitor_terms": _sig("nmf_monitor_terms", ctypes.c_int, [_vp, _D]),
    "nmf_gini": _sig("nmf_gini", ctypes.c_int, [_vp, _vp, _i64, _D]),
    "nmf_iterate_full": _sig("nmf_iterate_full", ctypes.c_int, [_vp, _P, _vp, _i64, _vp, _vp, _i32]),
    "nmf_spectrum": _sig("nmf_spectrum", ctypes.c_int, [_vp, _i64, _i32, _vp, _D]),
    "nmf_sketch_csr": _sig("nmf_sketch_csr", ctypes.c_int,
                           [_vp, _P, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "nmf_compress_csr": _sig("nmf_compress_csr", ctypes.c_int,
                             [_vp, _P, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "nmf_residual_csr": _sig("nmf_residual_csr", ctypes.c_int,
                             [_vp, _P, _vp, _vp, _vp, _i64, _vp, _vp, _D, _D, _D]),
    "nmf_solve_csr": _sig("nmf_solve_csr", ctypes.c_int,
                          [_vp, _P, _i32, _vp, _vp, _vp, _i64, _vp, _vp, _D, ctypes.POINTER(_i32)]),
    "nmf_decay_rate": _sig("nmf_decay_rate", ctypes.c_int, [_D, _i32, ctypes.c_double, _D]),
    "nmf_last_solve_info": _sig("nmf_last_solve_info", ctypes.c_int,
                                [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "nmf_phase_times": _sig("nmf_phase_times", ctypes.c_int,
                            [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]),
    "nmf_solve": _sig("nmf_solve", ctypes.c_int,
                      [_vp, _P, _i32, _vp, _i64, _vp, _vp, _D, ctypes.POINTER(_i32)]),
    "nmf_mlp_param_count": _sig("nmf_mlp_param_count", _i64, [_i32, _i32, _i32]),
    "nmf_warmstart_features": _sig("nmf_warmstart_features", ctypes.c_int,
                                   [_vp, _P, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nmf_mlp_forward": _sig("nmf_mlp_forward", ctypes.c_int,
                            [_vp, _i32, _i32, _i32, _vp, _vp, _i64, _vp]),
    "nmf_mlp_loss_grad": _sig("nmf_mlp_loss_grad", ctypes.c_int,
                              [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _i64, _vp, _D]),
    "nmf_mlp_adam": _sig("nmf_mlp_adam", ctypes.c_int,
                         [_vp, _i64, _vp, _vp, _vp, _vp, _i32, ctypes.c_float]),
    "nmf_mlp_train_step": _sig("nmf_mlp_train_step", ctypes.c_int,
                               [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _i32, ctypes.c_float,
                                _vp, _vp, _i64, _D]),
    "nmf_warmstart_apply": _sig("nmf_warmstart_apply", ctypes.c_int,
                                [_vp, _i64, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nmf_set_warmstart": _sig("nmf_set_warmstart", ctypes.c_int, [_vp, _i32, _i32, _vp, _vp]),
    "nmf_warmstart_targets": _sig("nmf_warmstart_targets", ctypes.c_int,
                                  [_vp, _i64, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nmf_last_batch_info": _sig("nmf_last_batch_info", ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "nmf_solve_batched": _sig("nmf_solve_batched", ctypes.c_int,
                              [_vp, _i32, _P, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                               ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _D]),
}


class NmfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


FLAG_STAGED_ITERATE = 1
FLAG_SIMT_DUAL_PASS = 2
FLAG_ROBUST_QR = 4
FLAG_TC_RESIDUAL = 8


def params(m, n, r, ell, power_iters=2, iters=0, rule="fasthals", prec="fp32", seed=0,
           residual_every=0, target_rel_err=0.0, alpha=0.0, beta=0.0, eps=0.0, flags=0):
    """Build an nmf_params struct (names as in include/nmf_rp.h)."""
    return nmf_params(int(m), int(n), int(r), int(ell), int(power_iters), int(iters),
                      RULE.get(rule, rule), PREC.get(prec, prec), int(seed), int(residual_every),
                      int(flags), float(target_rel_err), float(alpha), float(beta), float(eps))


class Context:
    """An nmf_ctx bound to a CUDA device and stream (torch's current stream by default)."""

    def __init__(self, device=None, stream=None):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        self.stream = s
        h = _vp()
        st = _c["nmf_create"](ctypes.byref(h), dev.index, _vp(s.cuda_stream))
        if st != NMF_OK:
            raise NmfError(st, "nmf_create failed")
        self.handle = h

    def set_stream(self, stream):
        self.stream = stream
        self._check(_c["nmf_set_stream"](self.handle, _vp(stream.cuda_stream)))

    def close(self):
        if getattr(self, "handle", None):
            _c["nmf_destroy"](self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != NMF_OK:
            msg = _c["nmf_last_error"](self.handle)
            raise NmfError(st, msg.decode() if msg else "")

    @property
    def launches(self):
        return int(_c["nmf_launch_count"](self.handle))


def _ptr(t):
    return _vp(t.data_ptr()) if t is not None else _vp(0)


def _dev_f32(t, name):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


class Fp8Copy:
    """The FP8 copy of an m x n matrix made by nmf_quantize: `buf` holds the library's byte layout
    (E4M3 codes with rows padded to 16 bytes, then one E8M0 scale byte a 32 x 32 tile)."""

    def __init__(self, buf, m, n):
        self.buf, self.shape = buf, (m, n)
        self.is_cuda, self.device = buf.is_cuda, buf.device

    def data_ptr(self):
        return self.buf.data_ptr()


def nmf_quantized_bytes(prec, m, n):
    return int(_c["nmf_quantized_bytes"](PREC.get(prec, prec), m, n))


def _x_arg(X, prec):
    if not X.is_cuda:
        raise ValueError("X must be a CUDA tensor")
    if prec == PREC["fp8"]:
        if not isinstance(X, Fp8Copy):
            raise ValueError("FP8 X must be the nmf_quantize copy (Fp8Copy)")
        return X, X.shape[1]
    if prec == PREC["bf16"]:
        if X.dtype != torch.bfloat16 or not X.is_contiguous():
            raise ValueError("BF16 X must be a contiguous bfloat16 tensor (see nmf_quantize)")
        return X, X.shape[1]
    if X.dtype != torch.float32 or X.stride(1) != 1:
        raise ValueError("X must be float32 with unit column stride")
    return X, X.stride(0)


def _empty(shape, like):
    return torch.empty(shape, dtype=torch.float32, device=like.device)


def workspace_size(p):
    out = ctypes.c_size_t(0)
    st = _c["nmf_workspace_size"](ctypes.byref(p), ctypes.byref(out))
    if st != NMF_OK:
        raise NmfError(st, "nmf_workspace_size")
    return int(out.value)


def nmf_sync(ctx):
    ctx._check(_c["nmf_sync"](ctx.handle))


def nmf_gaussian(ctx, rows, cols, seed, stream_id, out=None):
    out = out if out is not None else torch.empty((rows, cols), dtype=torch.float32, device=ctx.device)
    _dev_f32(out, "out")
    ctx._check(_c["nmf_gaussian"](ctx.handle, rows, cols, seed, stream_id, _ptr(out)))
    return out


def nmf_quantize(ctx, X, prec="bf16", out=None):
    """BF16 copy (a bfloat16 tensor) or FP8 copy (an Fp8Copy) of the FP32 matrix X."""
    m, n = X.shape
    pr = PREC.get(prec, prec)
    if X.dtype != torch.float32 or X.stride(1) != 1:
        raise ValueError("X must be float32 with unit column stride")
    if pr == PREC["fp8"]:
        nb = nmf_quantized_bytes(pr, m, n)
        buf = out.buf if isinstance(out, Fp8Copy) else torch.empty(nb, dtype=torch.uint8,
                                                                   device=X.device)
        if buf.numel() < nb:
            raise ValueError("FP8 buffer too small")
        ctx._check(_c["nmf_quantize"](ctx.handle, pr, _ptr(X), m, n, X.stride(0), _ptr(buf)))
        return Fp8Copy(buf, m, n)
    if out is None:
        out = torch.empty((m, n), dtype=torch.bfloat16, device=X.device)
    ctx._check(_c["nmf_quantize"](ctx.handle, pr, _ptr(X), m, n, X.stride(0), _ptr(out)))
    return out


def nmf_dual_pass(ctx, X, V=None, U=None, prec="fp32", Y=None, Z=None):
    """Y = X V and Z = X^T U in one pass over X (either pair may be omitted)."""
    pr = PREC.get(prec, prec)
    X, ldx = _x_arg(X, pr)
    m, n = X.shape
    ell = (V if V is not None else U).shape[1]
    if V is not None:
        _dev_f32(V, "V")
        Y = Y if Y is not None else _empty((m, ell), X)
    if U is not None:
        _dev_f32(U, "U")
        Z = Z if Z is not None else _empty((n, ell), X)
    ctx._check(_c["nmf_dual_pass"](ctx.handle, pr, _ptr(X), m, n, ldx, ell, _ptr(V), _ptr(U),
                                   _ptr(Y if V is not None else None),
                                   _ptr(Z if U is not None else None)))
    return Y, Z


def nmf_qr(ctx, Y, Q=None):
    _dev_f32(Y, "Y")
    Q = Q if Q is not None else _empty(Y.shape, Y)
    ctx._check(_c["nmf_qr"](ctx.handle, _ptr(Y), Y.shape[0], Y.shape[1], _ptr(Q)))
    return Q


def nmf_sketch(ctx, p, X, omega_L=None, omega_R=None, QL=None, QR=None):
    X, ldx = _x_arg(X, p.prec)
    QL = QL if QL is not None else _empty((p.m, p.ell), X)
    QR = QR if QR is not None else _empty((p.n, p.ell), X)
    _dev_f32(omega_L, "omega_L")
    _dev_f32(omega_R, "omega_R")
    ctx._check(_c["nmf_sketch"](ctx.handle, ctypes.byref(p), _ptr(X), ldx, _ptr(omega_L),
                                _ptr(omega_R), _ptr(QL), _ptr(QR)))
    return QL, QR


def nmf_compress(ctx, p, X, QL, QR, Xhat=None, Xchk=None):
    X, ldx = _x_arg(X, p.prec)
    Xhat = Xhat if Xhat is not None else _empty((p.ell, p.n), X)
    Xchk = Xchk if Xchk is not None else _empty((p.m, p.ell), X)
    ctx._check(_c["nmf_compress"](ctx.handle, ctypes.byref(p), _ptr(X), ldx, _ptr(_dev_f32(QL, "QL")),
                                  _ptr(_dev_f32(QR, "QR")), _ptr(Xhat), _ptr(Xchk)))
    return Xhat, Xchk


def nmf_iterate(ctx, p, QL, QR, Xhat, Xchk, W, H, iters):
    for t, nm in ((QL, "QL"), (QR, "QR"), (Xhat, "Xhat"), (Xchk, "Xchk"), (W, "W"), (H, "H")):
        _dev_f32(t, nm)
    ctx._check(_c["nmf_iterate"](ctx.handle, ctypes.byref(p), _ptr(QL), _ptr(QR), _ptr(Xhat),
                                 _ptr(Xchk), _ptr(W), _ptr(H), int(iters)))
    return W, H


def nmf_residual(ctx, p, X, W, H):
    """Returns (rel_err, ||X - W H||^2, ||X||^2); synchronises the stream."""
    X, ldx = _x_arg(X, 0)
    rel, e2, x2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ctx._check(_c["nmf_residual"](ctx.handle, ctypes.byref(p), _ptr(X), ldx, _ptr(_dev_f32(W, "W")),
                                  _ptr(_dev_f32(H, "H")), ctypes.byref(rel), ctypes.byref(e2),
                                  ctypes.byref(x2)))
    return rel.value, e2.value, x2.value


_STATIC_ERRORS = {
    1: "bad pointer, size or device",
    7: "the device needs more partial-sum slots than the static array holds",
    2: "set-up or launch failed",
}


def nmf_residual_static(X, W, H, out, stream=None):
    """||X - W H||^2 and ||X||^2 into `out` (2 float64 on X's device) with no context and no
    device allocation; queued on `stream` (torch's current stream), not synchronised."""
    X, ldx = _x_arg(X, 0)
    W, H = _dev_f32(W, "W"), _dev_f32(H, "H")
    if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 2 and out.is_contiguous()):
        raise ValueError("out must be a contiguous float64 CUDA tensor of 2 elements")
    # the C entry point receives bare pointers and cannot see these: a mismatch would make its
    # kernels read past the end of W or H
    if W.dim() != 2 or H.dim() != 2 or W.shape[0] != X.shape[0] or H.shape != (W.shape[1], X.shape[1]):
        raise ValueError(f"W must be ({X.shape[0]}, r) and H (r, {X.shape[1]}); got "
                         f"{tuple(W.shape)} and {tuple(H.shape)}")
    if not (W.device == X.device and H.device == X.device and out.device == X.device):
        raise ValueError("X, W, H and out must be on the same CUDA device")
    dev = X.device.index
    s = stream if stream is not None else torch.cuda.current_stream(X.device)
    st = _c["nmf_residual_static"](dev, _vp(s.cuda_stream), _ptr(X), X.shape[0], X.shape[1], ldx,
                                   W.shape[1], _ptr(W), _ptr(H), _ptr(out))
    if st != NMF_OK:
        raise NmfError(st, "nmf_residual_static: " + _STATIC_ERRORS.get(st, "error"))
    return out


def nmf_nndsvd(ctx, p, QL, Xhat, W=None, H=None):
    W = W if W is not None else _empty((p.m, p.r), QL)
    H = H if H is not None else _empty((p.r, p.n), QL)
    ctx._check(_c["nmf_nndsvd"](ctx.handle, ctypes.byref(p), _ptr(_dev_f32(QL, "QL")),
                                _ptr(_dev_f32(Xhat, "Xhat")), _ptr(W), _ptr(H)))
    return W, H


def nmf_solve(ctx, p, X, W, H, init="given"):
    """Whole pipeline on FP32 X; returns (rel_err, iterations run). W, H updated in place."""
    X, ldx = _x_arg(X, 0)
    rel, it = ctypes.c_double(), ctypes.c_int32()
    ctx._check(_c["nmf_solve"](ctx.handle, ctypes.byref(p), INIT.get(init, init), _ptr(X), ldx,
                               _ptr(_dev_f32(W, "W")), _ptr(_dev_f32(H, "H")), ctypes.byref(rel),
                               ctypes.byref(it)))
    return rel.value, it.value


def nmf_solve_batched(ctx, ps, Xs, Ws, Hs, init="given", rows_per_block=0):
    """Independent problems in one call: ps, Xs, Ws, Hs are equal-length lists (params structs,
    FP32 X, in/out W, H CUDA tensors). Returns the list of final relative residuals."""
    k = len(ps)
    if not (len(Xs) == len(Ws) == len(Hs) == k) or k == 0:
        raise ValueError("ps, Xs, Ws, Hs must be non-empty lists of equal length")
    arr = (nmf_params * k)(*ps)
    xp = (_vp * k)(*[_vp(_x_arg(x, 0)[0].data_ptr()) for x in Xs])
    ld = (_i64 * k)(*[x.stride(0) for x in Xs])
    wp = (_vp * k)(*[_vp(_dev_f32(w, "W").data_ptr()) for w in Ws])
    hp = (_vp * k)(*[_vp(_dev_f32(h, "H").data_ptr()) for h in Hs])
    out = (ctypes.c_double * k)()
    ctx._check(_c["nmf_solve_batched"](ctx.handle, k, arr, INIT.get(init, init), xp, ld, wp, hp,
                                       int(rows_per_block), out))
    return list(out)


def nmf_mlp_param_count(F, hidden, r):
    return int(_c["nmf_mlp_param_count"](F, hidden, r))


def nmf_warmstart_features(ctx, p, QL, Xhat):
    """(W_b, H_b, hscale, F_w, F_h) of include/nmf_rp.h's learned warm start."""
    dev = QL.device
    f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=dev)
    Wb, Hb, hs = f(p.m, p.r), f(p.r, p.n), f(p.r)
    Fw, Fh = f(p.m, 3 * p.r), f(p.n, 3 * p.r)
    ctx._check(_c["nmf_warmstart_features"](ctx.handle, ctypes.byref(p), _ptr(_dev_f32(QL, "QL")),
                                            _ptr(_dev_f32(Xhat, "Xhat")), _ptr(Wb), _ptr(Hb),
                                            _ptr(hs), _ptr(Fw), _ptr(Fh)))
    return Wb, Hb, hs, Fw, Fh


def nmf_mlp_forward(ctx, params, X, hidden, r, Y=None):
    _dev_f32(params, "params")
    _dev_f32(X, "X")
    Y = Y if Y is not None else torch.empty((X.shape[0], r), dtype=torch.float32, device=X.device)
    ctx._check(_c["nmf_mlp_forward"](ctx.handle, X.shape[1], hidden, r, _ptr(params), _ptr(X),
                                      X.shape[0], _ptr(Y)))
    return Y


def nmf_mlp_loss_grad(ctx, params, X, T, hidden, r, grad=None):
    """(loss, grad) of the mean squared error of network(X) against T."""
    _dev_f32(params, "params")
    grad = grad if grad is not None else torch.empty_like(params)
    loss = ctypes.c_double()
    ctx._check(_c["nmf_mlp_loss_grad"](ctx.handle, X.shape[1], hidden, r, _ptr(params),
                                        _ptr(_dev_f32(X, "X")), _ptr(_dev_f32(T, "T")), X.shape[0],
                                        _ptr(grad), ctypes.byref(loss)))
    return loss.value, grad


def nmf_mlp_adam(ctx, params, m, v, grad, step, lr):
    ctx._check(_c["nmf_mlp_adam"](ctx.handle, params.numel(), _ptr(params), _ptr(m), _ptr(v),
                                   _ptr(grad), int(step), float(lr)))


def nmf_mlp_train_step(ctx, params, m, v, grad, step, lr, X, T, hidden, r, want_loss=False):
    loss = ctypes.c_double()
    ctx._check(_c["nmf_mlp_train_step"](ctx.handle, X.shape[1], hidden, r, _ptr(params), _ptr(m),
                                         _ptr(v), _ptr(grad), int(step), float(lr),
                                         _ptr(_dev_f32(X, "X")), _ptr(_dev_f32(T, "T")),
                                         X.shape[0], ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def nmf_warmstart_targets(ctx, Wb, Hb, hscale, Wstar, Hstar):
    """Network targets (Tw m x r, Th n x r) that map (W_b, H_b) onto (W*, H*)."""
    m, r = Wb.shape
    n = Hb.shape[1]
    for t, nm in ((Wb, "Wb"), (Hb, "Hb"), (hscale, "hscale"), (Wstar, "Wstar"), (Hstar, "Hstar")):
        _dev_f32(t, nm)
    if Wstar.shape != (m, r) or Hb.shape != (r, n) or Hstar.shape != (r, n) or hscale.numel() != r:
        raise ValueError("shapes of W_b, H_b, hscale, W*, H* disagree")
    Tw = _empty((m, r), Wb)
    Th = _empty((n, r), Wb)
    ctx._check(_c["nmf_warmstart_targets"](ctx.handle, m, n, r, _ptr(Wb), _ptr(Hb), _ptr(hscale),
                                           _ptr(Wstar), _ptr(Hstar), _ptr(Tw), _ptr(Th)))
    return Tw, Th


def nmf_warmstart_apply(ctx, Wb, Dw, Hb, Dh, hscale, W=None, H=None):
    W = W if W is not None else torch.empty_like(Wb)
    H = H if H is not None else torch.empty_like(Hb)
    m, r = Wb.shape
    n = Hb.shape[1]
    ctx._check(_c["nmf_warmstart_apply"](ctx.handle, m, n, r, _ptr(Wb), _ptr(Dw), _ptr(Hb),
                                          _ptr(Dh), _ptr(hscale), _ptr(W), _ptr(H)))
    return W, H


def nmf_set_warmstart(ctx, hidden, r, params_w, params_h):
    ctx._check(_c["nmf_set_warmstart"](ctx.handle, hidden, r, _ptr(_dev_f32(params_w, "params_w")),
                                        _ptr(_dev_f32(params_h, "params_h"))))


def nmf_last_batch_info(ctx):
    """Rows of W per block the last batched solve used (autotuned when 0 was passed)."""
    v = _i32()
    ctx._check(_c["nmf_last_batch_info"](ctx.handle, ctypes.byref(v)))
    return v.value


def nmf_set_profiling(ctx, on=True):
    ctx._check(_c["nmf_set_profiling"](ctx.handle, 1 if on else 0))


def nmf_iterate_full(ctx, p, X, W, H, iters):
    """Full-data FastHALS (p.rule fasthals) or Lee-Seung MU (p.rule mu) on X (FP32, or the BF16 /
    FP8 nmf_quantize copy of p.prec); W, H updated in place."""
    X, ldx = _x_arg(X, p.prec)
    for t, nm in ((W, "W"), (H, "H")):
        _dev_f32(t, nm)
    if W.shape != (p.m, p.r) or H.shape != (p.r, p.n):
        raise ValueError(f"W must be ({p.m}, {p.r}) and H ({p.r}, {p.n})")
    ctx._check(_c["nmf_iterate_full"](ctx.handle, ctypes.byref(p), _ptr(X), ldx, _ptr(W),
                                      _ptr(H), int(iters)))
    return W, H


class Csr:
    """A sparse m x n matrix in CSR form on a CUDA device: row_ptr (int64, m + 1), col (int32,
    distinct within a row), val (float32)."""

    def __init__(self, row_ptr, col, val, shape):
        if not (row_ptr.is_cuda and row_ptr.dtype == torch.int64 and row_ptr.is_contiguous()):
            raise ValueError("row_ptr must be a contiguous int64 CUDA tensor")
        if not (col.is_cuda and col.dtype == torch.int32 and col.is_contiguous()):
            raise ValueError("col must be a contiguous int32 CUDA tensor")
        _dev_f32(val, "val")
        if row_ptr.numel() != shape[0] + 1 or col.numel() != val.numel():
            raise ValueError("row_ptr must hold m + 1 entries and col / val nnz each")
        self.row_ptr, self.col, self.val, self.shape = row_ptr, col, val, tuple(shape)
        self.nnz = val.numel()

    def _args(self):
        return _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val), self.nnz


def _csr_check(p, X):
    if not isinstance(X, Csr) or X.shape != (p.m, p.n):
        raise ValueError(f"X must be a Csr of shape ({p.m}, {p.n})")


def nmf_sketch_csr(ctx, p, X, omega_L=None, omega_R=None, QL=None, QR=None):
    _csr_check(p, X)
    QL = QL if QL is not None else _empty((p.m, p.ell), X.val)
    QR = QR if QR is not None else _empty((p.n, p.ell), X.val)
    ctx._check(_c["nmf_sketch_csr"](ctx.handle, ctypes.byref(p), *X._args(), _ptr(omega_L),
                                    _ptr(omega_R), _ptr(QL), _ptr(QR)))
    return QL, QR


def nmf_compress_csr(ctx, p, X, QL, QR, Xhat=None, Xchk=None):
    _csr_check(p, X)
    Xhat = Xhat if Xhat is not None else _empty((p.ell, p.n), X.val)
    Xchk = Xchk if Xchk is not None else _empty((p.m, p.ell), X.val)
    ctx._check(_c["nmf_compress_csr"](ctx.handle, ctypes.byref(p), *X._args(),
                                      _ptr(_dev_f32(QL, "QL")), _ptr(_dev_f32(QR, "QR")),
                                      _ptr(Xhat), _ptr(Xchk)))
    return Xhat, Xchk


def nmf_residual_csr(ctx, p, X, W, H):
    """(rel_err, ||X - W H||^2, ||X||^2) of sparse X; synchronises."""
    _csr_check(p, X)
    if W.shape != (p.m, p.r) or H.shape != (p.r, p.n):
        raise ValueError(f"W must be ({p.m}, {p.r}) and H ({p.r}, {p.n})")
    rel, e2, x2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ctx._check(_c["nmf_residual_csr"](ctx.handle, ctypes.byref(p), *X._args(),
                                      _ptr(_dev_f32(W, "W")), _ptr(_dev_f32(H, "H")),
                                      ctypes.byref(rel), ctypes.byref(e2), ctypes.byref(x2)))
    return rel.value, e2.value, x2.value


def nmf_solve_csr(ctx, p, X, W, H, init="given"):
    """Whole pipeline on sparse X; returns (rel_err, iterations run). W, H updated in place."""
    _csr_check(p, X)
    if W.shape != (p.m, p.r) or H.shape != (p.r, p.n):
        raise ValueError(f"W must be ({p.m}, {p.r}) and H ({p.r}, {p.n})")
    rel, it = ctypes.c_double(), ctypes.c_int32()
    ctx._check(_c["nmf_solve_csr"](ctx.handle, ctypes.byref(p), INIT.get(init, init), *X._args(),
                                   _ptr(_dev_f32(W, "W")), _ptr(_dev_f32(H, "H")),
                                   ctypes.byref(rel), ctypes.byref(it)))
    return rel.value, it.value


def nmf_spectrum(ctx, Xhat):
    """Singular values of X_hat (ell x n CUDA float32), descending, as a list of floats."""
    _dev_f32(Xhat, "Xhat")
    ell, n = Xhat.shape
    out = (ctypes.c_double * ell)()
    ctx._check(_c["nmf_spectrum"](ctx.handle, n, ell, _ptr(Xhat), out))
    return list(out)


def nmf_decay_rate(sigma, rel_floor=1e-3):
    """Exponential decay rate p of a descending spectrum (host computation in the library)."""
    arr = (ctypes.c_double * len(sigma))(*[float(v) for v in sigma])
    p = ctypes.c_double()
    st = _c["nmf_decay_rate"](arr, len(sigma), float(rel_floor), ctypes.byref(p))
    if st != NMF_OK:
        raise NmfError(st, "nmf_decay_rate: invalid spectrum or floor")
    return p.value


def nmf_gini(ctx, B):
    """Gini coefficient of the entries of the CUDA float32 tensor B (Section 5.1)."""
    _dev_f32(B, "B")
    g = ctypes.c_double()
    ctx._check(_c["nmf_gini"](ctx.handle, _ptr(B), B.numel(), ctypes.byref(g)))
    return g.value


def nmf_set_wait_limit(ctx, cycles=0):
    """Polling budget (SM clock cycles) of the persistent kernel's grid-barrier waits; 0 = default."""
    ctx._check(_c["nmf_set_wait_limit"](ctx.handle, int(cycles)))


def nmf_monitor_terms(ctx):
    """(cross, quad, ||X||^2, <X - X_q, X>) of the error monitor; synchronises the stream."""
    t = (ctypes.c_double * 4)()
    ctx._check(_c["nmf_monitor_terms"](ctx.handle, t))
    return tuple(t)


def nmf_phase_times(ctx, reset=True):
    """{phase: (milliseconds, spans)} since the last reset; synchronises the stream."""
    ms = (ctypes.c_double * len(PHASES))()
    cnt = (_i64 * len(PHASES))()
    ctx._check(_c["nmf_phase_times"](ctx.handle, ms, cnt, 1 if reset else 0))
    return {name: (ms[i], int(cnt[i])) for i, name in enumerate(PHASES)}


def nmf_last_solve_info(ctx):
    """(iterations, exact residual checks) of the last nmf_solve on this context."""
    it, ch = _i32(), _i32()
    ctx._check(_c["nmf_last_solve_info"](ctx.handle, ctypes.byref(it), ctypes.byref(ch)))
    return it.value, ch.value
