"""The learned warm start against the zero-velocity start on held-out tubes.

A small member of the tube family (radius 4-8, length 24-64, tau 0.7-1) keeps
the test short: 48 tubes are solved to steady state by the method, the
network is trained on their fields by the library's kernels, and 8 held-out
tubes are run from rest and from the network's proposal.  The learned start
must need fewer steps to reach a relative change of u below 1e-6 per step,
and both starts must end at the same solution."""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_start_converges_in_fewer_steps_than_rest():
    from paper_2108_08783_gb300 import warmstart as W
    fk = dict(radius=(4.0, 8.0), length=(24, 64), tau=(0.7, 1.0))
    r = W.study(n_train=48, n_eval=8, seed=1, samples_per_tube=512, iters=1200, max_steps=30000,
                family_kw=fk, log=lambda *a: None)
    assert r["unconverged_zero"] == 0 and r["unconverged_warm"] == 0
    assert r["loss_last"] < 0.1 * r["loss_first"]
    assert r["init_err_warm_median"] < 0.3          # zero start: 1 by definition
    assert r["steps_warm_mean"] < 0.85 * r["steps_zero_mean"]
    assert r["final_err_max"] < 5e-3
