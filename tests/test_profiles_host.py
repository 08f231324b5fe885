"""The committed ncu step traffic (profiles/traffic.json) that bench.py reports as
``roofline.traffic``: each entry names the kernel source it was taken on, the
summary it comes from carries the same source hash, and the bytes are those of
one step of that workload (between 0.8x and 1.3x its algorithmic bytes: L2
reuse and deferred write-back below, re-reads above)."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SITES = {"tube40": 5_144_576, "tree": 10_250_521}  # fluid sites of the two workloads
BYTES = {"f32": 4, "f16s": 2, "bf16s": 2, "f64": 8}


def entries():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("key", sorted(entries()))
def test_traffic_entry_is_one_step_of_its_workload(key):
    rec = entries()[key]
    config, storage = key.split("/")
    algo = SITES[config] * 2 * 19 * BYTES[storage]
    assert 0.8 * algo < rec["bytes_per_launch"] < 1.3 * algo
    assert len(rec["kernels_sha1"]) == 40


@pytest.mark.parametrize("key", sorted(entries()))
def test_traffic_entry_matches_its_summary(key):
    rec = entries()[key]
    words = [w.strip("(),;") for w in rec["detail"].split()]
    names = [w for w in words if w.startswith("profiles/")]
    assert names, "the entry names the summary it comes from"
    for name in names:
        with open(os.path.join(ROOT, name)) as f:
            text = f.read()
        assert rec["kernels_sha1"] in text.replace("\n", "")
