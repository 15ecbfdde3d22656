"""FP64 CPU oracle for the shifted-Laplacian multigrid Helmholtz solver (test infrastructure).

This package is test infrastructure, not part of the library. Only the test
suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg and
``--impl reference`` arm may import it; the CUDA library never does, and this
package imports nothing from the library.

It restates the method of Livshits, "Shifted Laplacian based multigrid
preconditioners for solving indefinite Helmholtz equations" (arXiv 1312.2880),
in plain numpy/scipy in complex FP64: the discretisation (Sec. 1, Eqs. 1-3),
Gauss-Seidel and its local Fourier analysis (Sec. 4), Kaczmarz relaxation of
the normal equations (Sec. 4-5), the V-cycle with its operator roles and the
HLM/SL/HYB variants (Sec. 5), right-preconditioned Bi-CGSTAB (Sec. 6), and the ray
correction with the stand-alone cycle solver of Table 7 (Sec. 6).
"""
from .helmholtz import *  # noqa: F401,F403
from .lfa import *  # noqa: F401,F403
from .ray import *  # noqa: F401,F403
