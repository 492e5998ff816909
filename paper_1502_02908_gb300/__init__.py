"""GB300-native event-based SISe / SISe3 epidemic simulation (arXiv:1502.02908 hot path).

The simulation runs in libepisim.so (hand-written CUDA for sm_103a behind the C ABI of
include/episim.h); ``binding.Sim`` wraps it.  ``workloads`` draws the seeded synthetic
inputs.  Importing the package loads nothing; the library is loaded on first use.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "binding", "build"]
