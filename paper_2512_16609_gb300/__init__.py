"""GB300 (sm_103a) implementation of the Hazedefy per-frame dehazing path.

The compute path is libhazedefy.so (hand-written CUDA kernels behind the C
interface in include/hazedefy.h); `binding` exposes that interface to Python
with the same names."""
from . import binding  # noqa: F401
from .binding import *  # noqa: F401,F403

__all__ = [n for n in dir(binding) if n.startswith(("hz_", "HZ_"))] + ["binding", "params", "HzError"]
