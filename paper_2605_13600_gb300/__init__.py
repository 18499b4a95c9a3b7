"""GB300-native (sm_103a) SCOUP sparse code uplift.

The compute lives in ``libscoup.so`` (hand-written CUDA behind the C ABI of
``include/scoup.h``); this package is its ctypes binding.  Importing it loads
the library and fails loudly if it has not been built.
"""
from ._lib import ScoupError, load as _load
from .scoup import *  # noqa: F401,F403

_load()

__version__ = "0.1.0"
