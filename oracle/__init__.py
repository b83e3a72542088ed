"""CPU oracle: plain, slow, obviously correct restatements of what the GEMM
landscape-smoothing method computes ("From Roofline to Ruggedness", arXiv
2605.29752).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  The
product (the C-ABI library under ``paper_2605_29752_gb300``) never imports,
links or executes anything here, and this package never imports the product.
The two share nothing but the seeded operand streams of ``synthetic.py``.

Modules
  gemm       C = A B in float64 on the BF16 operands, and the error bound (Sec. 2.2, Sec. 7.1)
  dp         best-of-tiles selection and the T0 -> T1 -> T2 padding/splitting DP (Sec. 6.4, Sec. 7.1)
  roughness  throughput surface, roughness per axis, slice and 3D conventions (Sec. 2 definitions, Sec. 8.6)
  landscape  first-principles ideal and optimal landscapes, KOL grading (Sec. 9, Sec. 10)
  fp8        e4m3 block quantisation and the block-scaled GEMM reference

Parity status: gemm, dp, roughness, fp8 quantisation and the ideal landscape are
pinned by tests/test_oracle_*.py.  The first-principles *optimal* landscape
(landscape.optimal_surface) is pinned by its parts and by hand-worked cells on
GB300 constants, but stays "parity unpinned" against the paper's own numbers:
the values the paper prints for it cannot be reproduced from its stated constants.  The FP8 GEMM error has no
bound in the paper beyond float32 accumulation ("parity unpinned" for its
observed error; its exact-product special cases are pinned).
"""
