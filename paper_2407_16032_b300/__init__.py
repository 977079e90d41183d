"""B300-native (sm_103a) BDIM incompressible-flow time step (WaterLily, arXiv 2407.16032).

The solver is the CUDA library ``libwl.so`` behind the C ABI of ``include/wl.h``;
``wl`` is its ctypes binding. Build with ``python -m paper_2407_16032_b300.build``.
"""
from .wl import Sim, WLError, lib, sim_from_case, EXPORTS, LIB_PATH  # noqa: F401
