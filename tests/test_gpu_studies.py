"""Rigid vs elastic wall shear stress on a seeded bifurcating tree (the
analogue of the paper's Sec. 3 limits-of-agreement comparison), on the GPU
path."""
import numpy as np
import pytest

import lbm_inputs as I

pytestmark = pytest.mark.gpu


def test_elastic_wall_lowers_wall_shear_stress_on_a_tree():
    from paper_2108_08783_gb300 import studies
    geo = I.murray_tree(seed=1, depth=3, root_radius=12.0)
    geo.iolets[0].u_mean = 0.03
    e, r, s = studies.wss_agreement(geo, tau=0.8, F=0.85, kappa=0.75 * 12.0 / 0.5, steps=3000)
    assert e.shape == r.shape and e.size > 1000
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(r))
    # lower shear stress with the elastic wall, as the paper reports (Sec. 3)
    assert s["bias"] < 0 and s["mean_a"] < s["mean_b"]
    assert s["frac_a_below_b"] > 0.5
    assert s["lower"] < s["bias"] < s["upper"]
