"""GB300-native periodic thermal-microstructure homogenization and OC design
(after Quan, Zhai & Fu, OpenTM, arXiv 2405.19991).

The computation lives in libotm.so (C ABI in include/otm.h, CUDA kernels for
sm_103a under csrc/).  ``paper_2405_19991_gb300.otm`` is its thin ctypes
binding (argument marshalling only) and ``paper_2405_19991_gb300.warmstart``
the host-side driver of the learned warm start's training loop.  There is no
CPU fallback: importing the binding fails when the library is missing.
"""
import os as _os

PKG_DIR = _os.path.dirname(_os.path.abspath(__file__))
LIB_PATH = _os.path.join(PKG_DIR, "libotm.so")


def build(verbose: bool = False, force: bool = False) -> str:
    from .build import build as _b
    return _b(verbose=verbose, force=force)
