"""GB300-native plane-wave block eigensolver (LOBPCG step of Kohn-Sham DFT).

The compute path is the CUDA library built from csrc/ (see build.py); this
package is its thin Python binding.  Importing it without the built library
raises ImportError.
"""
from .binding import *  # noqa: F401,F403
from .binding import Cell, PwError, LIB_PATH  # noqa: F401


def new_block(npw: int, nb: int, device="cuda"):
    """A column-major complex128 (npw, nb) CUDA tensor (band = column)."""
    import torch
    return torch.empty((nb, npw), dtype=torch.complex128, device=device).T
