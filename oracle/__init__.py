"""FP64 CPU oracle for full-polarisation AW-projection gridding (arXiv:2206.15117).

TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU-baseline
leg of the benchmark may import anything from this package.  The CUDA library
never does, and this package never imports the CUDA library or its Python
binding: the two share no code.  Inputs come from the seeded generators in
``paper_2206_15117_gb300.synthetic`` (geometry and random numbers only).

Modules
-------
core  : the method in plain NumPy/FP64 (prolate-spheroidal taper, Jones and
        Mueller matrices, Eq. 4-6, kernel synthesis, grid correction and
        normalisation, the mosaic weighting of Eq. 1) plus ctypes wrappers of
        the C loops in ``aw_oracle.c`` (coordinates, gridding, degridding,
        direct DFT).
mlp   : FP64 SIREN surrogate forward, analytic backward and Adam step.
clean : Cotton-Schwab major cycles around an FP32 Hogbom minor cycle.
mosaic: image-plane reprojection between SIN frames and the Eq. 1 combination.

Parity status: every function is pinned by tests under ``tests/`` against
values the paper prints, closed forms, library special functions or brute
force; see the per-function docstrings.
"""
