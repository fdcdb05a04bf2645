"""GB300-native (sm_103a) checkerboard local-update Monte Carlo of Demchik &
Strelchenko, "Monte Carlo simulations on Graphics Processing Units"
(arXiv:0903.3053): 2D Ising Metropolis and 4D SU(2) heat-bath sweeps in
hand-written CUDA behind the C ABI of include/mc.h (libmc.so)."""
from .mc import (  # noqa: F401
    MC_COLD, MC_HOT, MC_KIND_ISING, MC_KIND_SU2, MC_LAYOUT_INT8, MC_LAYOUT_MSC32, MC_FMT_INT8, MC_FMT_BITS,
    MC_FMT_F32, MC_FMT_NATIVE, MC_MODE_AUTO, MC_MODE_GRID, MC_MODE_RESIDENT, VAN, Batch, Chain, Group, MCError, ising, su2, load,
    mc_workspace_bytes,
)

__version__ = "1.0"
