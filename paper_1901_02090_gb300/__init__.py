"""GB300-native adaptive BDDC for mixed RT0/P0 Darcy flow (arXiv:1901.02090).

The solver lives in ``libbddc.so`` (C ABI in ``include/bddc.h``): host setup
in C++, and per solve one persistent CUDA kernel for sm_103a running
Algorithm 1 (coarse solve, subdomain solves, and CG on the interface with the
BDDC preconditioner of Algorithm 2).  ``bddc`` is the Python binding.
"""

from .build import build, LIB as LIB_PATH  # noqa: F401
