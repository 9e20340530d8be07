"""tnrc: tensor-network robust control (arXiv 2603.03639) on one GB300.

The ensemble-averaged TEBD/MPS fidelity of a qubit chain under random
parasitic ZZ crosstalk and its costate gradient, computed by hand-written
sm_103a CUDA kernels behind the C ABI of ``include/tnrc.h``.

  * ``tnrc``      -- ctypes binding of the C ABI (``Context``)
  * ``build``     -- in-tree build of ``lib/libtnrc.so``
"""
from .tnrc import Context, TNRCError, footprint, lib  # noqa: F401
