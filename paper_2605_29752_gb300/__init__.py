"""GB300-native BF16 GEMM landscape smoothing ("From Roofline to Ruggedness",
arXiv 2605.29752): sm_103a tcgen05 GEMM kernels in six tile variants, the
sweep that measures the (M, N, K) throughput landscape, roughness statistics,
and the best-of / padding-and-splitting plan table with O(1) lookup.

The compute lives in the C-ABI library ``librg.so`` (headers in
``include/rg.h``); ``paper_2605_29752_gb300.rg`` is its ctypes binding and
``paper_2605_29752_gb300.build`` compiles it.  Importing the binding without a
built library raises ImportError: there is no CPU fallback.
"""
__all__ = ["rg", "build"]
