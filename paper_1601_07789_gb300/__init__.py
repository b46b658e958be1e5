"""flyte multibyte floating point on GB300: k-byte pack/unpack fused into BLAS.

Importing the package is cheap: the CUDA library is loaded on first use by
``paper_1601_07789_gb300.flyte`` (the ctypes binding over ``libflyte.so``),
which raises if the library has not been built.
"""
