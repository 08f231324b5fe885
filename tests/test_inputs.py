"""The seeded synthetic inputs follow their stated recipes: tube site counts,
the Murray tree's branching law, angles, lengths and taper, the ensemble and
warm-start families' ranges, and reproducibility from the seed."""
import numpy as np
import pytest

import lbm_inputs as I
from lbm_inputs.geometry import _tree_segments


def test_tube_site_counts():
    assert int((I.tube(8, 64).labels == 1).sum()) == 13_312
    assert int((I.tube(40, 1024).labels == 1).sum()) == 5_144_576
    g = I.tube(8, 64)
    # ghost planes one node beyond the caps, radially inside
    assert int((g.labels[:, :, 0] == 2).sum()) == int((g.labels[:, :, 1] == 1).sum())
    assert int((g.labels[:, :, -1] == 3).sum()) == int((g.labels[:, :, -2] == 1).sum())


def test_murray_tree_recipe():
    segs = _tree_segments(0, 6, 48.0)
    assert len(segs) == 2 ** 7 - 1
    by_level = {}
    for p, d, L, r0, r1, lev in segs:
        assert abs(np.linalg.norm(d) - 1) < 1e-12
        assert 8.0 * r0 - 1e-9 <= L <= 12.0 * r0 + 1e-9
        assert r1 == pytest.approx(0.9 * r0)
        by_level.setdefault(lev, []).append((p, d, L, r0, r1))
    assert by_level[0][0][3] == 48.0
    # children: Murray's law r_p^3 = r_c1^3 + r_c2^3, split in [0.4, 0.6], angles 30-60 degrees,
    # starting at the parent's end
    for lev in range(6):
        parents, children = by_level[lev], by_level[lev + 1]
        for i, (p, d, L, r0, r1) in enumerate(parents):
            c1, c2 = children[2 * i], children[2 * i + 1]
            assert c1[3] ** 3 + c2[3] ** 3 == pytest.approx(r1 ** 3)
            assert 0.4 - 1e-12 <= c1[3] ** 3 / r1 ** 3 <= 0.6 + 1e-12
            for c in (c1, c2):
                np.testing.assert_allclose(c[0], p + L * d, atol=1e-9)
                ang = np.degrees(np.arccos(np.clip(np.dot(c[1], d), -1, 1)))
                assert 30.0 - 1e-9 <= ang <= 60.0 + 1e-9


def test_murray_tree_voxelisation_is_seeded_and_sparse():
    a = I.murray_tree(seed=3, depth=3, root_radius=8.0)
    b = I.murray_tree(seed=3, depth=3, root_radius=8.0)
    np.testing.assert_array_equal(a.labels, b.labels)
    fill = (a.labels == 1).mean()
    assert 0.0 < fill < 0.2
    assert len(a.iolets) == 1 + 2 ** 3  # root inlet, one outlet per leaf


def test_ensemble_family_ranges():
    fam = I.tube_ensemble(seed=0, count=256)
    R = np.array([m["radius"] for m in fam])
    L = np.array([m["length"] for m in fam])
    E = np.array([m["eh_r0"] for m in fam])
    T = np.array([m["period"] for m in fam])
    tau = np.array([m["tau"] for m in fam])
    assert R.min() >= 6 and R.max() <= 24 and L.min() >= 64 and L.max() <= 512
    assert E.min() >= 0.05 and E.max() <= 5 and T.min() >= 1000 and T.max() <= 5000
    assert tau.min() >= 0.55 and tau.max() <= 1.0
    # Eh/r0 log-uniform: about half the members below the geometric mean sqrt(0.05 * 5) = 0.5
    assert 0.35 < np.mean(E < 0.5) < 0.65
    for m in fam:
        assert m["kappa"] == pytest.approx(0.75 * m["radius"] / m["eh_r0"])


def test_warm_start_family_and_features():
    from paper_2108_08783_gb300 import warmstart as W
    fam = W.family(0, 64)
    held = W.family(100003, 64)
    assert all(0.01 <= p["u_in"] <= 0.04 for p in fam)
    assert not any(p == q for p in fam for q in held)
    f = W.features(fam[0])
    assert len(f) == W.N_GLOBAL
    rs, us = W.scales(fam[0])
    assert us == fam[0]["u_in"] and rs > 0


def test_mlp_init_is_glorot_and_seeded():
    th = I.mlp_init(5, 7, 256, 4, 3)
    np.testing.assert_array_equal(th, I.mlp_init(5, 7, 256, 4, 3))
    W0 = th[:256 * 7].reshape(256, 7)
    assert np.abs(W0).max() <= np.sqrt(6.0 / (256 + 7))
    assert th[256 * 7:256 * 7 + 256].max() == 0.0  # biases start at zero
