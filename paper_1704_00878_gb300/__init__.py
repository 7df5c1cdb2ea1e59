"""GB300 (sm_103a) center-star multiple sequence alignment.

The hot path of HAlign-II's protein MSA (arXiv 1704.00878): choose a center
sequence, align every sequence to it with affine-gap Smith-Waterman (Eq. 1-2)
plus traceback, merge the inserted spaces into one alignment.  All of it runs
as hand-written CUDA kernels in libmsa.so behind the C ABI of include/msa.h;
`binding` is the thin ctypes layer with the same function names.
"""
from . import _build  # noqa: F401

__all__ = ["binding", "build"]


def build(force=False):
    """Compile libmsa.so in-tree for sm_103a."""
    return _build.build(force=force)


def __getattr__(name):
    if name == "binding":
        import importlib
        return importlib.import_module(__name__ + ".binding")
    raise AttributeError(name)
