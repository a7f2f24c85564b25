"""Plain FP64 CPU oracle of random-projection compressed NMF (Torre & Graber, arXiv:1712.02248).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or execute anything in this
package: only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
use it. It shares no code with the CUDA library (no kernels, headers, helpers or constants), and it
never imports the library.

Every function is written for a reader to check against the paper by eye: numpy FP64, library
primitives (matmul, LAPACK QR/SVD) as single steps, no blocking or fusion beyond what the paper's
equations state. Functions whose result the paper does not fix are marked "parity unpinned".
"""
from .nmf_oracle import *  # noqa: F401,F403
from .fp8_oracle import *  # noqa: F401,F403
