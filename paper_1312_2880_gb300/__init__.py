"""GB300-native shifted-Laplacian multigrid solver for the 2-D Helmholtz equation (arXiv 1312.2880).

The solver itself is the CUDA library ``libhz.so`` (C ABI in ``include/hz.h``); :mod:`.hz` is its
Python binding and :mod:`.inputs` draws the seeded synthetic media and sources. The library is
loaded lazily so that ``inputs`` can be imported without a GPU.
"""

__all__ = ["hz", "inputs", "build"]
