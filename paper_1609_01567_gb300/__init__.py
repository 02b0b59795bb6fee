"""GB300 (sm_103a) sum-product LDPC decoder for any irregular code.

The compute path lives in the C-ABI library ``libldpc_gb300.so`` (CUDA
kernels under ``csrc/``); :mod:`.ldpc` is the thin Python binding over it.
Importing this package loads nothing; the library is opened on first use.
"""
