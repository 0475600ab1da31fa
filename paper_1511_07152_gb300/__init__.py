"""Separable W-projection gridding and degridding for NVIDIA GB300 (sm_103a).

A CUDA library (``csrc/``, C ABI in ``include/sepw.h``) implements the hot
path of Merry (2015), "Approximating W projection as a separable kernel":
1-D GCF tables (Eq. gt), location of visibilities on the grid and the plane
stack, binning, gridding with the separable update of Sec. 5, its adjoint
(degridding), and the image step with grid correction.  ``sepw`` is a thin
ctypes binding with the C names; it loads the built library on first use and
raises if it is missing (there is no CPU fallback).  ``build`` compiles it.
"""
import importlib


_SUBMODULES = ("build", "sepw", "autotune", "autograd", "major_cycle")


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    if name in _SUBMODULES:
        return importlib.import_module(f"{__name__}.{name}")
    mod = importlib.import_module(__name__ + ".sepw")
    return getattr(mod, name)
