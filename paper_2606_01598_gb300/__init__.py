"""GB300-native differentiable particle-mesh Ewald for point charges and point dipoles
(and, forward and first derivatives only, point quadrupoles), with the learned charge/dipole
network trained through it.

The compute path is ``libgbpme.so`` (CUDA for sm_103a, built in-tree by ``build.build()``)
behind the C ABI of ``include/gbpme.h``; this package is its thin Python binding.
"""
from .pme import (BatchPlan, Plan, PMEEnergy, PMEQuadEnergy, autotune_brick, launch_count,  # noqa: F401
                  mesh_dims, pme_energy, pme_quad_energy)
from ._abi import PMEError, header_functions, load as load_library  # noqa: F401
from .net import Net, pack_params, unpack_params  # noqa: F401

__all__ = ["Plan", "BatchPlan", "PMEEnergy", "pme_energy", "PMEQuadEnergy", "pme_quad_energy",
           "mesh_dims", "launch_count", "PMEError", "autotune_brick",
           "header_functions", "load_library", "Net", "pack_params", "unpack_params"]
