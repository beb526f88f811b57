"""GB300 (sm_103a) Mobius domain-wall MSPCG solver (arXiv:2104.05615).

The compute path is the CUDA library behind include/dwf.h; `binding` is the
ctypes layer with the C names, `lattice` a convenience wrapper holding torch
device tensors.  `inputs` draws the seeded synthetic gauge fields and sources.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "binding", "lattice"]
