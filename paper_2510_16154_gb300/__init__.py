"""GB300-native agent-based optimal-control image solver (arXiv 2510.16154).

The compute path is ``libagents.so`` (CUDA for sm_103a behind the C ABI of
``include/agents.h``); ``paper_2510_16154_gb300.lib`` is its ctypes binding.  Importing
this package loads nothing; ``lib.load()`` (called by every binding function) loads the
library and raises if it has not been built.
"""
from . import _lib as lib

__all__ = ["lib"]
