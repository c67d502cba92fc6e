"""FM-index search on one GB300: eight-Occ steps, exact and inexact backward search.

The CUDA library (libfmocc.so, C ABI in include/fmocc.h) is loaded lazily by ``fmocc``;
``synth`` holds the seeded input generators.
"""
__all__ = ["fmocc", "synth"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
