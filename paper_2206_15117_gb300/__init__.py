"""GB300-native full-polarisation AW-projection gridding (arXiv:2206.15117).

The compute path is the C-ABI library ``libaw.so`` (CUDA, sm_103a), declared in
``include/aw.h``; ``paper_2206_15117_gb300.aw`` is its thin ctypes binding.
Importing this package loads nothing; ``aw`` loads the library on first use
and raises if it is missing.
"""
__all__ = ["aw", "synthetic"]
