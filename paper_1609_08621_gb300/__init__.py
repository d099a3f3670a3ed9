"""GB300-native FMM force solve (PKDGRAV3, arXiv:1609.08621, Sec. 3).

``binding``  ctypes binding of the C ABI (include/fmm.h) of the CUDA library.
``build``    nvcc build of the library for sm_103a.
``synth``    seeded synthetic particle sets.
"""
from . import synth  # noqa: F401

__all__ = ["binding", "build", "synth"]
