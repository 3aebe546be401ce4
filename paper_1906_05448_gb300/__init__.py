"""GB300 (sm_103a) lattice Boltzmann library with IBB and IBM no-slip walls.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbm.h``); ``lbm`` is its thin ctypes binding.
"""
from . import build  # noqa: F401
from .lbm import (BC_IBB, BC_IBM_B, BC_IBM_U, BC_NONE, BF16S, F16S, F32, F64, RATES_DHUMIERES,  # noqa: F401
                  RATES_SRT, STATS_BINS, STATS_UNMASK, Lattice, LbmError, load, make_grid, workspace_bytes)
