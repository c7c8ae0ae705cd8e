"""GB300-native SP2 density-matrix purification on thresholded ELLPACK matrices.

The CUDA library (libsp2ell.so, C ABI declared in include/sp2ell.h) does every step of
the computation; `paper_2102_08505_gb300.sp2ell` is its thin ctypes binding and
`paper_2102_08505_gb300.inputs` draws seeded synthetic inputs.  Importing this package
loads nothing; the binding loads the library on first use and raises if it is missing.
"""
__all__ = ["inputs", "sp2ell"]
