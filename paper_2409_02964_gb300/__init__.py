"""GB300 (sm_103a) implementation of the fused D2Q9 stream + collide step of the
consistent MRT lattice Boltzmann method for the volume-averaged Navier-Stokes
equations (MRTLB-VANSE, arXiv:2409.02964).

``capi`` binds the C ABI of ``include/lbm_vanse.h``; ``Lattice`` (one lattice) and
``Batch`` (many independent lattices) are thin handles over it; ``Lattice3D`` is the
handle of the D3Q19 form of the scheme (``include/lbm_vanse3d.h``). The computation runs only in the CUDA library (``liblbm_vanse.so``).
"""
from . import build, capi  # noqa: F401
from .adjoint import Channel, OutletMomentum, outlet_momentum  # noqa: F401
from .batch import Batch, BatchLattice  # noqa: F401
from .lattice import Lattice, LbmError  # noqa: F401
from .lattice3d import Lattice3D  # noqa: F401

__all__ = ["Batch", "BatchLattice", "Channel", "Lattice", "Lattice3D", "LbmError", "OutletMomentum", "build",
           "capi", "outlet_momentum"]
