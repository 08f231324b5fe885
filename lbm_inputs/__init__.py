"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This package only produces inputs: voxel label grids (0 solid, 1 fluid, 2+k
ghost node of iolet k), iolet descriptions, per-voxel parameter fields,
seeded initial fields and the warm-start network's initial parameters.  It contains none of the lattice Boltzmann method's
arithmetic, so both the oracle and the product may import it.
"""
from .geometry import (Geometry, Iolet, tube, duct, closed_box, random_labels, murray_tree,  # noqa: F401
                       tube_ensemble, rest_radius, wall_normals)
from .fields import random_fields, gather  # noqa: F401
from .mlp import mlp_shapes, mlp_init, mlp_batch  # noqa: F401
