"""FP64 CPU oracle for the ghost-fill operator ``g = A x + b``.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA library
(no kernels, headers, helpers, tables or constant generators); the two meet
only at the seeded workload descriptions of ``paper_2605_14780_gb300.synth``.

What it computes, and where the paper defines it (Sec. III):

* ``regions``   the data / ghost / full region numbering (Sec. III-A),
* ``rows``      the sparse rows of zero padding, pure-function (constant)
  rows, halo copies, circular and symmetric maps and user CSR rows
  (Sec. III-B; Alg. 1; Table III's F_LIST and F_NNZ/F_COL/F_DATA),
* ``sphere``    the user-defined interpolation rows of a cubed sphere
  (Sec. III-B, the ``Itp`` matrix) as 1-D Lagrange interpolation along the
  neighbour panel row, with the 2x2 basis change of vector components
  (Sec. V-A),
* ``operator``  explicit assembly of ``A`` as CSR and of ``b``, the in-place
  apply ``y_G = A x_D + b`` and the adjoint ``x_D += A^T y_G, y_G = 0``.

Every floating-point step is FP64.  Parity pins live in ``tests/``; the one
function without an external pin is named in its own docstring.
"""
from .operator import (OracleError, build_operator, apply, apply_adjoint,
                       row_scale)

__all__ = ["OracleError", "build_operator", "apply", "apply_adjoint",
           "row_scale"]
