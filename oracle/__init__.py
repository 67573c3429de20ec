"""Plain FP64 CPU oracle of the TENO finite-volume residual.

Test infrastructure: only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  The product path never
does, and this package shares no code with it.
"""
