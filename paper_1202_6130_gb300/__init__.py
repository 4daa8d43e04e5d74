"""GB300-native engine for the pseudo-potential lattice-Boltzmann wetting model
of Colosqui, Kavousanakis, Papathanasiou & Kevrekidis (arXiv:1202.6130).

The fused per-timestep update (streaming, moments, pseudo-potential, fluid-fluid
and fluid-solid forces, wall momentum exchange, EDM-BGK collision) is one
hand-written sm_103a CUDA kernel behind the C ABI of ``include/lbm.h``;
``Simulation`` is a thin binding of that ABI.
"""
from . import analysis
from ._lib import (LBM_BF16S, LBM_D2Q9, LBM_D2Q21, LBM_FP16S, LBM_FP32, LBM_FP64, LBM_PSI_EOS,
                   LBM_PSI_EXP, LBM_ROUND_NEAREST, LBM_ROUND_STOCHASTIC, LbmError, load)
from .sim import Batch, Simulation, wall_core_tail, wall_gaussian_filter

__all__ = ["Simulation", "Batch", "LbmError", "load", "wall_gaussian_filter", "wall_core_tail",
           "LBM_D2Q9", "LBM_D2Q21", "LBM_FP64", "LBM_FP32", "LBM_FP16S", "LBM_BF16S",
           "LBM_PSI_EXP", "LBM_PSI_EOS", "LBM_ROUND_STOCHASTIC", "LBM_ROUND_NEAREST", "analysis"]
