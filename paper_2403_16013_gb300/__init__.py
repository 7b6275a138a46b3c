"""GB300-native complex multi-component (DD/TD/QD) LU with partial pivoting.

The compute path is libmclu.so (hand-written CUDA for sm_103a, C ABI in
include/mclu.h).  ``binding`` mirrors the C entry points, ``api`` offers torch
plane-tensor wrappers and the differentiable ``solve``; ``inputs`` holds the
seeded synthetic workloads.  Importing the package does not load the CUDA
library; the first call into ``binding``/``api`` does, and fails loudly if it
is missing.
"""

__all__ = ["api", "binding", "inputs", "build"]
