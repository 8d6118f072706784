"""GB300-native ghost-cell filling on block-structured grids.

Boundary conditions are applied as one affine sparse operator
``g = A x + b`` (arxiv 2605.14780, Sec. III) that overwrites every block's
ghost layers: zero and constant padding, halo copies, circular and symmetric
maps, cubed-sphere panel-edge interpolation with vector rotation, and user
CSR rows, plus the adjoint ``A^T``.  All arithmetic runs in the sm_103a
kernels of the ``libbcgb300`` shared library; :mod:`.bc` is a thin ctypes
binding over its C ABI (``include/bc.h``).

Importing the package loads nothing; :func:`bc.load_library` (called by the
binding on first use) raises if the compiled library is missing.
"""
__all__ = ["bc", "specs", "synth"]
