"""The C-ABI library loads and exports every entry point include/nmf_rp.h declares (no GPU).

Only host-side logic is exercised here: symbol resolution, the parameter checks of
nmf_workspace_size, the nmf_params layout, and the failure of nmf_create without a device.
"""
import ctypes
import os
import re

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nmf_rp.h")


@pytest.fixture(scope="module")
def N():
    import __graft_entry__ as g
    g.build()
    from paper_1712_02248_gb300 import nmf_rp
    return nmf_rp


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nmf_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(N):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(N.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(N.EXPORTS) == names


def test_params_struct_layout_matches_header(N):
    # int64 m, n; 6 x int32; uint64 seed; 2 x int32; 4 x double
    assert ctypes.sizeof(N.nmf_params) == 8 * 2 + 4 * 6 + 8 + 4 * 2 + 8 * 4
    assert N.nmf_params.seed.offset == 40
    assert N.nmf_params.target_rel_err.offset == 56


def test_workspace_size_checks_arguments(N):
    ok = N.params(20000, 5000, 20, 40, power_iters=2, prec="bf16")
    b = N.workspace_size(ok)
    # at least the BF16 copy of X plus the compressed data (Section 4.2 memory of the method)
    assert b >= 2 * 20000 * 5000 + 4 * 40 * (20000 + 5000) * 2
    for bad in (dict(r=0), dict(r=41), dict(ell=129, r=20), dict(m=30, n=30, ell=40),
                dict(power_iters=-1), dict(rule=7), dict(prec=9)):
        kw = dict(m=20000, n=5000, r=20, ell=40, power_iters=2)
        kw.update(bad)
        with pytest.raises(N.NmfError):
            N.workspace_size(N.params(**kw))


def test_create_without_gpu_fails_cleanly(N):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = N._c["nmf_create"](ctypes.byref(h), 0, None)
    assert st == 2 and not h.value    # NMF_ERR_CUDA, no context
    assert N._c["nmf_sync"](None) == 1


@pytest.mark.parametrize("m,n", [(1, 1), (31, 17), (32, 32), (33, 100), (20000, 5000),
                                 (4096, 100000), (7, 16)])
def test_quantized_bytes_match_the_copy_layouts(N, m, n):
    """Size query of the low-precision copies (host arithmetic, no GPU): BF16 2mn, FP32 4mn;
    FP8 codes with rows padded to 16 bytes, then the E8M0 bytes from a 256-byte boundary, one
    per 32 x 32 tile (the layout the oracle states in fp8_layout)."""
    import oracle as O
    assert N.nmf_quantized_bytes("bf16", m, n) == 2 * m * n
    assert N.nmf_quantized_bytes("fp32", m, n) == 4 * m * n
    assert N.nmf_quantized_bytes("fp8", m, n) == O.fp8_layout(m, n)[2]


def test_quantized_bytes_of_invalid_requests_is_zero(N):
    assert N.nmf_quantized_bytes("fp8", 0, 10) == 0
    assert N.nmf_quantized_bytes("bf16", 10, 0) == 0
    assert N.nmf_quantized_bytes(9, 10, 10) == 0


def test_decay_rate_host_function_matches_oracle(N):
    """nmf_decay_rate is host code of the library (no device): it fits the same exponential decay
    as the oracle's decay_rate, and refuses spectra it cannot fit."""
    import numpy as np
    rng = np.random.default_rng(5)
    for _ in range(5):
        p = rng.uniform(1e-3, 0.3)
        s = np.exp(-p * np.arange(60)) * (1 + 0.05 * rng.standard_normal(60)) * 3.0
        s = np.sort(np.abs(s))[::-1]
        assert abs(N.nmf_decay_rate(s, 1e-3) - O.decay_rate(s, 1e-3)) <= 1e-10
    with pytest.raises(N.NmfError):
        N.nmf_decay_rate([1.0], 0.0)
    with pytest.raises(N.NmfError):
        N.nmf_decay_rate([1.0, 1e-9, 1e-9], 1e-3)
