"""GB300-native Barnes-Hut octree gravity (Ferrari, Lavagna, Blazquez 2019).

The compute path is the C-ABI library ``libgravity.so`` built from ``csrc/``
(hand-written sm_103a CUDA).  ``gravity`` is its thin ctypes binding; ``inputs``
draws seeded synthetic bodies.  Submodules are imported lazily so that the input
generators can be used on machines without the CUDA library.
"""
__all__ = ["gravity", "inputs"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
