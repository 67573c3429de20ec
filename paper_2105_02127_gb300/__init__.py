"""GB300-native TENO finite-volume residual and SSP-RK3 on unstructured triangles.

The compute path lives in the CUDA library built from csrc/ (C ABI declared in
include/teno.h); `paper_2105_02127_gb300.teno` is its thin ctypes binding and is
imported on demand so that the input generators can be used without it.
"""
__all__ = ["inputs", "teno"]
