"""Random-projection compressed NMF on GB300 (sm_103a).

`paper_1712_02248_gb300.nmf_rp` is the Python binding of the C-ABI library `libnmf_rp.so`
(argument marshalling only; every step runs in the library's CUDA kernels). Importing it loads the
library and raises if it has not been built. `paper_1712_02248_gb300.inputs` draws seeded
synthetic inputs and needs no GPU.
"""
