"""GB300-native MDLG hot path: 2D Lennard-Jones MD fused with MDLG coarse-graining.

The compute path lives in the CUDA library ``libmdlg.so`` (sources under
``csrc/``, C-ABI declared in ``include/mdlg.h``).  ``mdlg`` is a thin ctypes
binding to it; ``inputs`` holds the seeded synthetic-input generators.

Submodules are imported lazily so that ``inputs`` can be used without the
CUDA library being built.
"""

__all__ = ["mdlg", "inputs", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
