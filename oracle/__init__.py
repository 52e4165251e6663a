"""FP64 CPU oracle of the Hazedefy dehazing path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package; the product path never does."""
from .hazedefy_oracle import *  # noqa: F401,F403
from .hazedefy_oracle import OracleParams, FrameResult  # noqa: F401
