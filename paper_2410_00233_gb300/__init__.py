"""GB300-native Kronecker-product-sum split Bregman deblurring (arXiv 2410.00233).

The compute path lives in the C-ABI library ``libkpsb.so`` (CUDA, sm_103a) built from
``csrc/``; ``kpsb`` is its thin ctypes binding.  Importing this package does not load the
library; ``paper_2410_00233_gb300.kpsb.lib()`` does, and raises if it is missing.
"""
__all__ = ["inputs", "kpsb"]
