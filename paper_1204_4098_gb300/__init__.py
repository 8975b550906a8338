"""GB300-native pseudopotential D2Q9 lattice Boltzmann (Li, Luo & Li).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through the thin ctypes binding in ``lbm.py``.  Importing the package
does not load the library; the first call into ``lbm`` does, and fails loudly
when it is missing.
"""
from . import inputs  # noqa: F401
