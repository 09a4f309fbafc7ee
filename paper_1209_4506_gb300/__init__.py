"""GB300 (sm_103a) grid-side Hartree step of arXiv:1209.4506.

Submodules:
  capi     ctypes declarations of the C ABI (include/hartree.h)
  hartree  PyTorch-facing plan wrapper (device memory and streams only)
  synth    seeded synthetic inputs (diamond supercells, random cells)
  build    in-tree nvcc build of libhartree_gb300.so

Importing the package loads nothing; the CUDA library is loaded on first use.
"""

__all__ = ["capi", "hartree", "synth", "build"]


def __getattr__(name):
    import importlib

    if name in ("capi", "hartree", "synth", "build", "autograd"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in ("HartreePlan", "atoms_reorder"):
        return getattr(importlib.import_module(f"{__name__}.hartree"), name)
    raise AttributeError(name)
