"""The error model behind the 16-bit storage bounds, checked on the CPU.

The FP64 oracle is run with its stored populations rounded after every step
to binary16 or bfloat16 (as shifted storage g = f - w, the format the GPU
stores), against the same oracle unrounded.  The rel-L2 errors of rho - 1
and u after 1000 steps from rest must stay within BOUND_FACTOR times the
random-walk estimate (storage_bounds.rounding_walk_estimate), the bound the
GPU parity tests use; and bfloat16's error must be the larger one.
"""
import numpy as np
import pytest

import lbm_inputs as I
from oracle import Oracle, velocity_set
from storage_bounds import BOUND_FACTOR, UNIT_ROUNDOFF, round_storage, rounding_walk_estimate

from analytic_ref import rel_l2


def _run(storage, steps, geo):
    o = Oracle(geo.labels, geo.iolets, tau=0.8, wall_model=1, F=0.85, kappa=12.0)
    if storage is None:
        o.run(steps)
        return o
    _, w, _ = velocity_set()
    f = o.populations()
    o.set_populations(round_storage(f - w, storage) + w, step=0)
    for _ in range(steps):
        o.run(1)
        f = o.populations()
        o.set_populations(round_storage(f - w, storage) + w, step=o.step)
    return o


def test_rounded_oracle_stays_within_the_storage_bounds():
    geo = I.tube(6, 127, u_mean=0.025)
    steps = 1000
    ref = _run(None, steps, geo)
    e_rho, e_u = rounding_walk_estimate(ref, steps)
    r0, u0 = ref.moments()
    errs = {}
    for st in ("f16s", "bf16s"):
        r, u = _run(st, steps, geo).moments()
        er, eu = rel_l2(r - 1, r0 - 1), rel_l2(u, u0)
        us = UNIT_ROUNDOFF[st]
        assert er < BOUND_FACTOR * us * e_rho and eu < BOUND_FACTOR * us * e_u, (st, er, eu)
        errs[st] = (er, eu)
    assert errs["bf16s"][0] > errs["f16s"][0] and errs["bf16s"][1] > errs["f16s"][1]
