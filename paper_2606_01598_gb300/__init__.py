"""GB300-native differentiable particle-mesh Ewald for point charges and point dipoles.

The compute path is ``libgbpme.so`` (CUDA for sm_103a, built in-tree by ``build.build()``)
behind the C ABI of ``include/gbpme.h``; this package is its thin Python binding.
"""
from .pme import BatchPlan, Plan, PMEEnergy, launch_count, mesh_dims, pme_energy  # noqa: F401
from ._abi import PMEError, header_functions, load as load_library  # noqa: F401

__all__ = ["Plan", "BatchPlan", "PMEEnergy", "pme_energy", "mesh_dims", "launch_count", "PMEError",
           "header_functions", "load_library"]
