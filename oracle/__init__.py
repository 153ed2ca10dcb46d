"""CPU oracle of the DG-MHD hot path: plain FP64 numpy, written from the paper.

This package is test infrastructure. Only the tests, `__graft_entry__.smoke()`
and the benchmark's CPU-baseline / reference arm may import it. It shares no
code with the CUDA library and the product path never calls it.
"""
