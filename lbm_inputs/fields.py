"""Seeded initial fields on the voxel grid, and gathering them at site coordinates.

Fields are defined per voxel so that each side (oracle or library) gathers
them at the coordinates of its own fluid sites; no site numbering is assumed.
"""
import numpy as np


def random_fields(seed, shape, drho=1e-3, umax=0.02, smooth=2):
    """Smooth random density and velocity fields on a ``shape`` voxel grid.

    Returns ``rho`` [nx,ny,nz] with ``|rho - 1| <= drho`` and ``u``
    [nx,ny,nz,3] with components bounded by ``umax``; white noise is
    box-filtered ``smooth`` times along each axis so that the initial state is
    not dominated by grid-scale noise.
    """
    rng = np.random.default_rng(seed)

    def field():
        a = rng.uniform(-1.0, 1.0, shape)
        for _ in range(smooth):
            for ax in range(3):
                a = (np.roll(a, 1, ax) + a + np.roll(a, -1, ax)) / 3.0
        m = np.abs(a).max()
        return a / m if m > 0 else a

    rho = 1.0 + drho * field()
    u = np.stack([umax * field() for _ in range(3)], -1)
    return rho, u


def gather(grid, coords):
    """Values of a per-voxel grid (scalar [nx,ny,nz] or vector [nx,ny,nz,k]) at integer coords [n,3]."""
    coords = np.asarray(coords)
    return np.ascontiguousarray(grid[coords[:, 0], coords[:, 1], coords[:, 2]])
