"""Test helpers: build the CUDA path and the oracle on the same seeded inputs.

The two sides share only ``lbm_inputs`` (labels, iolets, per-voxel fields).
Each side gathers per-voxel fields at the coordinates of its own sites.
"""
import numpy as np

import lbm_inputs as I
from oracle import Oracle


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def wall_params_from_grid(grid, coords, wall_sites):
    """Per-wall-site values of a per-voxel parameter grid."""
    return I.gather(grid, coords[wall_sites])


def make_pair(geo, storage="f64", tau=0.8, wall_model=1, F=0.85, kappa=0.0, rho0=1.0,
              fields=None, F_grid=None, kappa_grid=None, bulk_sites=None):
    """(Lattice, Oracle) on the same geometry, parameters and initial state.

    ``fields`` = (rho_grid, u_grid) per-voxel initial fields or None (rest);
    ``F_grid`` / ``kappa_grid`` per-voxel wall parameters (else scalars);
    ``bulk_sites`` sites per lane of the bulk kernel (None: the library default).
    """
    from paper_2108_08783_gb300 import Lattice
    lat = Lattice(geo.labels, geo.iolets, storage=storage, tau=tau)
    if bulk_sites is not None:
        lat.tune(bulk_sites=bulk_sites)
    orc = Oracle(geo.labels, geo.iolets, tau=tau, wall_model=wall_model, F=F, kappa=kappa,
                 rho0=rho0)
    lex = lat.export()
    oex = orc.export()
    lF, oF = F, F
    lK, oK = kappa, kappa
    if F_grid is not None:
        lF = wall_params_from_grid(F_grid, lex["coords"], lex["wall_sites"])
        oF = wall_params_from_grid(F_grid, oex["coords"], oex["wall_sites"])
    if kappa_grid is not None:
        lK = wall_params_from_grid(kappa_grid, lex["coords"], lex["wall_sites"])
        oK = wall_params_from_grid(kappa_grid, oex["coords"], oex["wall_sites"])
    lat.set_wall("elastic" if wall_model else "bounceback", rho0=rho0, F=lF, kappa=lK)
    orc.configure(tau, wall_model, rho0, oF, oK)
    if fields is not None:
        rho, u = fields
        lat.init_fields(I.gather(rho, lex["coords"]), I.gather(u, lex["coords"]))
        orc.init_equilibrium(I.gather(rho, oex["coords"]), I.gather(u, oex["coords"]))
    return lat, orc
