"""Host logic of the launch-knob autotuner (``coordinate_search``), on fake timers.

The search starts from the library's defaults, changes a knob only for a gain
above the noise margin, and sweeps again until nothing changes, so knobs whose
best values depend on each other are still found together."""
import itertools

from paper_2108_08783_gb300.lattice import coordinate_search, default_knobs


def run(cost, knobs, start, **kw):
    state = {}
    applied = []

    def apply(cfg):
        state.clear()
        state.update(cfg)
        applied.append(dict(cfg))

    best, results = coordinate_search(apply, lambda: cost(state), knobs, start, **kw)
    return best, results, applied


def test_defaults_match_the_library():
    assert default_knobs("f32") == dict(bulk_sites=1, bulk_warps=4, prefetch=4096)
    assert default_knobs("f16s") == dict(bulk_sites=2, bulk_warps=4, prefetch=0)
    assert default_knobs("bf16s") == dict(bulk_sites=2, bulk_warps=4, prefetch=0)
    assert default_knobs("f64") == dict(bulk_sites=1, bulk_warps=4, prefetch=0)


def test_keeps_a_better_start_that_one_sweep_from_the_first_candidates_misses():
    # one site per lane is best only with a prefetch distance; two sites per
    # lane are best without one (the FP32 tube's landscape)
    table = {(1, 0): 1.10, (1, 4096): 1.00, (2, 0): 1.05, (2, 4096): 1.04}
    cost = lambda s: table[(s["bulk_sites"], s["prefetch"])]
    knobs = (("bulk_sites", (1, 2)), ("prefetch", (0, 4096)))
    best, _, applied = run(cost, knobs, dict(bulk_sites=1, prefetch=4096))
    assert best == dict(bulk_sites=1, prefetch=4096)
    assert applied[-1] == best


def test_second_sweep_finds_coupled_optimum():
    # from (1, 0) the first sweep moves prefetch to 2048 only after sites has
    # been tried at prefetch 0; sites = 3 is best only with prefetch 2048
    table = {}
    for a, b in itertools.product((1, 2, 3), (0, 2048)):
        table[(a, b)] = 1.0
    table[(1, 0)] = 1.00
    table[(2, 0)] = 1.20
    table[(3, 0)] = 1.10
    table[(1, 2048)] = 0.90
    table[(2, 2048)] = 0.95
    table[(3, 2048)] = 0.80
    cost = lambda s: table[(s["bulk_sites"], s["prefetch"])]
    knobs = (("bulk_sites", (1, 2, 3)), ("prefetch", (0, 2048)))
    best, _, _ = run(cost, knobs, dict(bulk_sites=1, prefetch=0))
    assert best == dict(bulk_sites=3, prefetch=2048)


def test_gain_below_margin_keeps_the_current_value():
    cost = lambda s: {4: 1.000, 8: 0.997}[s["bulk_warps"]]
    best, _, _ = run(cost, (("bulk_warps", (4, 8)),), dict(bulk_warps=4))
    assert best["bulk_warps"] == 4
    cost = lambda s: {4: 1.000, 8: 0.990}[s["bulk_warps"]]
    best, _, _ = run(cost, (("bulk_warps", (4, 8)),), dict(bulk_warps=4))
    assert best["bulk_warps"] == 8


def test_each_measurement_warms_up_then_keeps_the_best_trial():
    calls = []

    def timer():
        calls.append(1)
        return [5.0, 2.0, 3.0][(len(calls) - 1) % 3]  # warm-up, then two trials

    best, results = coordinate_search(lambda cfg: None, timer, (("graph_steps", (20,)),),
                                      dict(graph_steps=20))
    assert best == dict(graph_steps=20)
    assert [ms for _, ms in results] == [2.0]
    assert len(calls) == 3


def test_start_value_outside_candidates_is_kept_unless_beaten():
    cost = lambda s: {4096: 1.0, 0: 1.2, 1024: 1.1}[s["prefetch"]]
    best, results, _ = run(cost, (("prefetch", (0, 1024)),), dict(prefetch=4096))
    assert best["prefetch"] == 4096
    assert {cfg["prefetch"] for cfg, _ in results} == {4096, 0, 1024}


def test_joint_knobs_leave_a_local_optimum_one_knob_at_a_time_cannot():
    # the batched FP32 ensemble's landscape: the defaults (1, 4096) beat every
    # single-knob move, but (2, 0) is 4 % faster still
    table = {(1, 0): 1.10, (1, 4096): 1.00, (2, 0): 0.96, (2, 4096): 1.05}
    cost = lambda s: table[(s["bulk_sites"], s["prefetch"])]
    start = dict(bulk_sites=1, prefetch=4096)
    best, _, _ = run(cost, (("bulk_sites", (1, 2)), ("prefetch", (0, 4096))), start)
    assert best == start  # one knob at a time stops at the local optimum
    joint = ((("bulk_sites", "prefetch"), list(itertools.product((1, 2), (0, 4096)))),)
    best, results, applied = run(cost, joint, start)
    assert best == dict(bulk_sites=2, prefetch=0)
    assert applied[-1] == best
    # each grid point measured once per sweep; the second sweep changes nothing
    assert len(results) == 4 + 4
