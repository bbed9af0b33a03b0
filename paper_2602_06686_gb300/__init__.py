"""GB300-native (sm_103a) Purified-TRT lattice Boltzmann hot path.

The product is the C-ABI library ``_lib/liblbm.so`` (``include/lbm.h``) built
from ``csrc/`` by :func:`build.build`; :mod:`.lbm` is its ctypes binding.
"""
from .lbm import (COLLISIONS, Batch, LATTICES, LAYOUTS, STORAGES, Lattice, LBMError,  # noqa: F401
                  buffer_sizes, copy_ceiling, load_library, make_params)
