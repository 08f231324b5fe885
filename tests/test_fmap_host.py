"""The host F-map precompute (lbm_fmap, Sec. 2.3 Eq. F) against the oracle's
closed form (oracle/analytic.py, Bessel power series), and its limits.
lbm_fmap runs on the host only, so these checks need no GPU."""
import numpy as np
import pytest

from oracle import analytic as OA


@pytest.fixture(scope="module")
def studies():
    from paper_2108_08783_gb300 import build
    build.build()
    from paper_2108_08783_gb300 import studies
    return studies


def test_fmap_matches_oracle_closed_form(studies):
    alpha = np.array([0.0, 1e-3, 0.5, 1.0, 3.0, 4.0, 8.68, 12.0, 20.0])
    dr = np.array([0.0, 0.01, 0.05, 0.1, 0.3])
    for M in (0.7, 0.9 + 0.05j, 0.3 - 0.2j):
        F = studies.fmap(alpha, dr, M)
        ref = np.array([[OA.f_ratio(a, d, M) for d in dr] for a in alpha])
        np.testing.assert_allclose(F, ref, rtol=1e-10, atol=1e-12)


def test_fmap_limits(studies):
    alpha = np.linspace(0.0, 20.0, 11)
    F = studies.fmap(alpha, [0.0], 0.6)
    np.testing.assert_allclose(F, 1.0, atol=1e-12)        # dr = 0: same point
    F0 = studies.fmap(alpha, [0.05, 0.1], 0.0)
    np.testing.assert_allclose(F0, 1.0, atol=1e-15)       # M = 0: no radial variation
    assert np.isnan(studies.fmap([2.0], [0.0], 1.0)).all()  # 0/0


def test_fmap_rejects_out_of_range(studies):
    from paper_2108_08783_gb300 import LbmError
    for a, d in (([-1.0], [0.1]), ([30.0], [0.1]), ([1.0], [1.0]), ([1.0], [-0.1])):
        with pytest.raises(LbmError):
            studies.fmap(a, d, 0.5)


def test_limits_of_agreement_statistics(studies):
    rng = np.random.default_rng(0)
    b = rng.uniform(1, 2, 500)
    a = 0.8 * b + rng.normal(0, 0.01, 500)
    s = studies.limits_of_agreement(a, b)
    d = a - b
    assert s["bias"] == pytest.approx(d.mean())
    assert s["upper"] - s["lower"] == pytest.approx(2 * 1.96 * d.std(ddof=1))
    assert s["frac_a_below_b"] == 1.0
