"""GB300 (sm_103a) library for the FFT-based method-of-lines solution of thin-film (2D) and
bulk (3D) magnetization problems of type-II superconductors (Prigozhin & Sokolovsky,
arXiv:1801.04869).

The compute path is the CUDA library built from csrc/ (C interface in include/mf.h); the
`native` module is its ctypes binding.  Nothing here falls back to a CPU implementation.
"""
from .native import (MF_ERR_NOCONV, MF_OK, MF_READ_HZ, MF_READ_J, MF_READ_MOMENT, MFError,  # noqa: F401
                     Problem, from_workload, load)

__all__ = ["Problem", "from_workload", "load", "MFError", "MF_OK", "MF_ERR_NOCONV",
           "MF_READ_HZ", "MF_READ_MOMENT", "MF_READ_J"]
