"""GB300-native (sm_103a) SCOUP sparse code uplift.

The compute lives in ``libscoup.so`` (hand-written CUDA behind the C ABI of
``include/scoup.h``); this package is its ctypes binding.  The library is
loaded on first use and any entry point raises ImportError if it has not been
built (``paper_2605_13600_gb300.build.build()``): there is no fallback.
"""
from ._lib import ScoupError  # noqa: F401
from .scoup import *  # noqa: F401,F403

__version__ = "0.1.0"
