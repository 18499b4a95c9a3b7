"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package draws random scenes, cameras, region maps and sparse codes. It
holds none of the uplift arithmetic (no projection, compositing, scatter or
Top-K): both the oracle and the CUDA library consume the arrays it returns.
"""
from .scenes import *  # noqa: F401,F403
