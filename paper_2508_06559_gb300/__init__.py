"""GB300-native (sm_103a) exact round-by-round CFR solver for open-hand, fixed-deck Pasur.

The solver lives in a CUDA library behind the C ABI of include/pasur.h; ``pasur`` is its thin
ctypes binding and ``build`` compiles it in-tree.
"""
from . import pasur  # noqa: F401
from .pasur import Ctx, PasurError, Tree, load, pasur_config_default, pasur_deal  # noqa: F401
