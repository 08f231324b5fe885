"""Fused diagnostics (lbm_step_diag) on the GPU.

The last of the requested steps reduces the mass and the iolet fluxes of the
state it reads, from the moments its kernels form anyway (per tile in the
compute type, across tiles in FP64).  They must equal lbm_reduce of that
same state (a separate pass over the populations) and, in FP64 storage, the
oracle's reduction after the same number of steps.

Tolerances.  FP64 compute: the two reductions differ only in summation order
(1e-12 relative).  FP32 compute: each site's rho - 1 is a sum of 19 FP32
values (|g_i| < 0.1 here), rounded at most 19 times by 2^-24 of a partial sum
below 0.3, and each tile adds 32 of them in 5 rounds; the bound below takes
the worst case of both per tile (far below the ~1.6 that one tile's
rho - 1 contributes with the density offset these tests start from, so a
tile counted twice or missed fails).  Fluxes: the momentum rho u of a site in
FP32 (converted to FP64) against j in FP64, 2^-22 relative per site.
"""
import numpy as np
import pytest

import lbm_inputs as I
from lbm_pair import make_pair

pytestmark = pytest.mark.gpu


def _fields(seed, shape, offset=0.05):
    rho, u = I.random_fields(seed, shape, drho=1e-3, umax=0.02)
    return rho + offset, u


def _mass_bound(lat, storage):
    if storage == "f64":
        return 1e-12 * lat.n
    n_tiles = int(lat.info()[3])
    per_site = 19 * 2.0 ** -24 * 0.3
    per_tile = 5 * 2.0 ** -24 * 32 * 0.3
    return lat.n * per_site + n_tiles * per_tile


def _check(lat, storage, out, ref):
    assert abs(out[0] - ref[0]) <= _mass_bound(lat, storage), (out[0], ref[0])
    rt = 1e-12 if storage == "f64" else 2.0 ** -22
    np.testing.assert_allclose(out[1:], ref[1:], rtol=rt, atol=rt * 1e-3 * lat.n)


@pytest.mark.parametrize("storage,bulk_sites", [("f64", None), ("f32", 1), ("f32", 2),
                                                ("f16s", 2), ("bf16s", 3), ("f16s", 4)])
def test_step_diag_equals_reduce_of_the_state_it_reads(storage, bulk_sites):
    geo = I.tube(12, 159, u_mean=0.025)
    lat, _ = make_pair(geo, storage, tau=0.8, wall_model=1, F=0.85, kappa=0.75 * 12 / 0.5,
                       fields=_fields(3, geo.shape), bulk_sites=bulk_sites)
    assert int(lat.info()[4]) > 0  # bulk tiles are part of the sum
    for steps in (37, 1, 2):  # odd and even layouts, repeated calls
        lat.step(steps - 1)
        lat.sync()
        ref = lat.reduce()
        out = lat.step_diag(1)
        lat.sync()
        _check(lat, storage, out, ref)
    # several steps in one call: the last one reduces (the state after 3),
    # against the same state reached again from a checkpoint
    f0, s0 = lat.populations(), int(lat.info()[7])
    out = lat.step_diag(4, np.zeros(1 + lat.n_iolets))
    lat.sync()
    lat.set_populations(f0, s0)
    lat.step(3)
    lat.sync()
    _check(lat, storage, out, lat.reduce())


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_step_diag_with_sites_linked_to_two_iolets(storage):
    geo = I.random_labels(4, (14, 11, 3))
    lat, _ = make_pair(geo, storage, tau=0.7, wall_model=1, F=0.8, kappa=2.0,
                       fields=_fields(5, geo.shape))
    for steps in (5, 6):
        lat.step(steps)
        lat.sync()
        ref = lat.reduce()
        out = lat.step_diag(1)
        lat.sync()
        _check(lat, storage, out, ref)


def test_step_diag_matches_the_oracle_reduction():
    geo = I.tube(12, 159, u_mean=0.025)
    lat, orc = make_pair(geo, "f64", tau=0.8, wall_model=1, F=0.85, kappa=0.75 * 12 / 0.5,
                         fields=_fields(7, geo.shape))
    out = lat.step_diag(301)  # reduces the state after 300 steps
    lat.sync()
    orc.run(300)
    np.testing.assert_allclose(out, orc.reduce(), rtol=1e-10, atol=1e-12 * lat.n)


def test_step_diag_rejects_bad_arguments():
    from paper_2108_08783_gb300 import LbmError
    geo = I.tube(6, 40, u_mean=0.02)
    lat, _ = make_pair(geo, "f32")
    with pytest.raises(LbmError):
        lat.step_diag(0)
