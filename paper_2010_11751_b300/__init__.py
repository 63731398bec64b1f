"""B300-native lattice Boltzmann stream-and-collide library (D3Q19 / D3Q27).

The compute path is the CUDA shared library ``liblbm.so`` built from ``csrc/``
for sm_103a; ``lbm`` is its thin ctypes binding.  Importing the package does not
load the library: the first call through ``lbm`` does, and raises if the
library is missing.  ``inputs`` holds seeded synthetic workloads only.
"""
import importlib

__all__ = ["lbm", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
