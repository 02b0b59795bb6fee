"""FP64 CPU oracle of the sum-product LDPC decoder (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It shares no code with the CUDA library.
"""
