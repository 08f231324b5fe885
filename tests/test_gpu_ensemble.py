"""Batched ensembles (one launch per step kernel for all members) on the GPU.

Members are uneven tubes from the seeded ensemble family (radius, length,
Eh/r0, inlet period, tau per member).  An ensemble must reproduce the same
lattices advanced one by one, with direct launches and with captured-graph
replays, to rounding: the ensemble kernels inline the same update as the
single-lattice kernels, but the compiler may contract multiply-adds
differently in each, so the two may differ in the last bits of a stored
population (FP32: < 1e-6 absolute; FP16 storage: a few units of its last
place).  Every member must also match its own FP64 oracle.
"""

# |f_ensemble - f_alone| bound per storage: rounding-level, far below the
# effect of any wrong member parameter.
ATOL = {"f32": 1e-6, "f16s": 1e-4}
import numpy as np
import pytest

import lbm_inputs as I
from lbm_pair import rel_l2

pytestmark = pytest.mark.gpu


def _members(n=5, seed=1, scale=0.25):
    out = []
    for prm in I.tube_ensemble(seed=seed, count=n):
        R = max(3.0, prm["radius"] * scale)
        L = max(8, int(prm["length"] * scale))
        geo = I.tube(R, L, u_mean=0.02, u_amp=0.01, period=prm["period"],
                     phase=0.1 * len(out))
        kappa = 0.75 * R / prm["eh_r0"]
        out.append((geo, prm["tau"], kappa, 0.5 + 0.1 * len(out)))
    return out


def _lattices(members, storage):
    from paper_2108_08783_gb300 import Lattice
    lats = []
    for geo, tau, kappa, F in members:
        lat = Lattice(geo.labels, geo.iolets, storage=storage, tau=tau)
        lat.set_wall("elastic", rho0=1.0, F=F, kappa=kappa)
        lats.append(lat)
    return lats


@pytest.mark.parametrize("graph_steps,persistent", [(0, 0), (4, 0), (0, 1)])
@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_ensemble_equals_members_alone(storage, graph_steps, persistent):
    from paper_2108_08783_gb300 import Ensemble
    members = _members()
    alone = _lattices(members, storage)
    batch = _lattices(members, storage)
    ens = Ensemble(batch)
    ens.tune(graph_steps=graph_steps, schedule=1, prefetch=64, persistent=persistent)
    for chunk in (5, 10, 9):  # odd and even counts, graph replays plus direct steps
        ens.step(chunk)
        for lat in alone:
            lat.step(chunk)
        ens.sync()
        for a, b in zip(alone, batch):
            a.sync()
            np.testing.assert_allclose(b.populations(), a.populations(), rtol=0,
                                       atol=ATOL[storage])
    ens.close()


@pytest.mark.parametrize("bulk_sites", [2, 3, 4])
@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_ensemble_bulk_pairing_equals_members_alone(storage, bulk_sites):
    """The two-sites-per-lane bulk kernels in an ensemble (a warp's two tiles may
    belong to two members) against the same members stepped alone with the same
    kernels, on tubes large enough to have bulk tiles."""
    from paper_2108_08783_gb300 import Ensemble
    members = _members(n=6, seed=3, scale=0.5)
    alone = _lattices(members, storage)
    batch = _lattices(members, storage)
    assert sum(int(l.info()[4]) for l in batch) > 50  # bulk tiles
    for lat in alone:
        lat.tune(bulk_sites=bulk_sites)
    ens = Ensemble(batch)
    ens.tune(bulk_sites=bulk_sites, schedule=1)
    for chunk in (5, 10, 9):
        ens.step(chunk)
        for lat in alone:
            lat.step(chunk)
        ens.sync()
        for a, b in zip(alone, batch):
            a.sync()
            np.testing.assert_allclose(b.populations(), a.populations(), rtol=0,
                                       atol=ATOL[storage])
    ens.close()


def test_ensemble_members_match_oracle():
    from oracle import Oracle
    from paper_2108_08783_gb300 import Ensemble
    members = _members(n=4, seed=2)
    lats = _lattices(members, "f64")
    ens = Ensemble(lats)
    ens.tune(graph_steps=10)
    ens.step(131)
    ens.sync()
    for (geo, tau, kappa, F), lat in zip(members, lats):
        orc = Oracle(geo.labels, geo.iolets, tau=tau, wall_model=1, F=F, kappa=kappa)
        orc.run(131)
        rl, ul = lat.moments()
        ro, uo = orc.moments()
        assert rel_l2(rl, ro) < 1e-10 and rel_l2(ul, uo) < 1e-10
    ens.close()


def test_ensemble_rejects_mixed_members():
    from paper_2108_08783_gb300 import Ensemble, LbmError
    members = _members(n=2)
    a = _lattices(members[:1], "f32")
    b = _lattices(members[1:], "f16s")
    with pytest.raises(LbmError):
        Ensemble(a + b)
    c = _lattices(members, "f32")
    c[0].step(1)
    with pytest.raises(LbmError):
        Ensemble(c)


def test_persistent_grid_barrier_times_out_and_the_context_survives():
    """Fault injection on the host side: the grid barrier is told to wait for
    one arrival that never comes; every CTA gives up after its bounded spin,
    lbm_ensemble_sync reports LBM_ETIMEOUT, and the same lattices step on
    normally afterwards."""
    from paper_2108_08783_gb300 import Ensemble, LbmError
    members = _members(n=3)
    lats = _lattices(members, "f32")
    ens = Ensemble(lats)
    ens.tune(persistent=1, barrier_extra=1)
    ens.step(3)
    with pytest.raises(LbmError) as e:
        ens.sync()
    assert e.value.status == -5  # LBM_ETIMEOUT
    ens.tune(barrier_extra=0)
    for lat in lats:
        lat.init_fields()
    ens.step(4)
    ens.sync()
    alone = _lattices(members, "f32")
    for a, b in zip(alone, lats):
        a.step(4)
        a.sync()
        np.testing.assert_allclose(b.populations(), a.populations(), rtol=0, atol=ATOL["f32"])
    ens.close()
