"""GB300-native elastic-wall D3Q19 lattice Boltzmann hot path.

The product is the C-ABI shared library ``liblbm.so`` (``include/lbm.h``)
built from ``csrc/`` for sm_103a; :class:`Lattice` (and :class:`Ensemble`,
:class:`MLP` for the learned warm start) is its Python binding.
Importing :class:`Lattice` needs the built library and a CUDA device; there
is no CPU fallback.
"""
from ._capi import (LBM_BF16S, LBM_F16S, LBM_F32, LBM_F64, LbmError,  # noqa: F401
                    EXPORTS, LIB_PATH)


def __getattr__(name):
    if name in ("Lattice", "Ensemble"):
        from . import lattice
        return getattr(lattice, name)
    if name in ("MLP", "warm_frame"):
        from . import mlp
        return getattr(mlp, name)
    raise AttributeError(name)
