"""GB300-native Gamma-point periodic J/K build with Ewald-split ERIs.

The compute path is libjk.so (hand-written sm_103a CUDA behind the C ABI of
include/jk.h); ``paper_2410_22278_gb300.jk`` is its ctypes binding and
``paper_2410_22278_gb300.build`` compiles it in-tree.
"""
from . import jk  # noqa: F401
from .jk import (JK_FP64, JK_MIXED, JkError, Plan, Server, ewald_point_charges,  # noqa: F401
                 plan_from_cell)
