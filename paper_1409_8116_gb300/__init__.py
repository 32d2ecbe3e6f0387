"""GB300-native (sm_103a) direct FFT Poisson solver after PoisFFT (arXiv 1409.8116).

The solver is the C-ABI library libpoisfft.so (include/poisfft.h) built from
csrc/; `binding` is its thin ctypes wrapper.  Importing this package does not
load the library; `from paper_1409_8116_gb300 import binding` does, and fails
if the library has not been built.
"""

__all__ = ["binding", "build"]
