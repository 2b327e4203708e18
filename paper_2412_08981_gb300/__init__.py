"""GB300-native non-nested multilevel smoothed Schwarz solver (arXiv 2412.08981).

The product is libmsp.so (CUDA for sm_103a, C ABI in include/msp.h); this
package holds its sources (csrc/), its in-tree build (build.py) and a thin
ctypes binding with the C names (msp.py).
"""
from . import msp  # noqa: F401
from .msp import Hierarchy, Instance, MspError, Server, load  # noqa: F401

__all__ = ["msp", "Hierarchy", "Instance", "MspError", "Server", "load"]
