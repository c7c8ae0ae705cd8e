"""CPU FP64 oracle for SP2 purification on thresholded ELLPACK matrices.

Test infrastructure only: tests, the smoke check and the CPU-baseline leg of the
benchmark use it to check the CUDA library.  The product path never imports it.
"""
