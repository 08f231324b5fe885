"""The checked build (-DLBM_CHECKED) on the GPU: every population slot is
stored exactly once per step (the in-place AA streaming relies on it) and every
neighbour index stays in range, on tubes, ducts, random sparse geometries (one
of them with sites linked to two iolets), a bifurcating tree and a tube with
bulk tiles, in both storages and wall models, with every bulk-kernel pairing
of FP32, for odd and even steps.

The checked build counts each store of the step kernels per slot and checks
the counts after every step; a violation is reported by lbm_sync as
LBM_ECHECK instead of trapping.  It runs in a subprocess because a process
loads one build of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, sys.argv[1])
import lbm_inputs as I
from paper_2108_08783_gb300 import Lattice
geos = [I.tube(6, 40, u_mean=0.02, u_amp=0.01, period=50.0), I.duct(7, 5, 33),
        I.murray_tree(seed=2, depth=2, root_radius=6.0)]
for seed in range(3):
    geos.append(I.random_labels(seed, (12, 11, 37), fill=0.7, n_iolets=2))
geos.append(I.random_labels(4, (14, 11, 3), fill=0.8))  # sites linked to two iolets
modes = {"f32": (1, 2, 3, 4), "f64": (1,)}
count = 0
geos.append(I.tube(8, 255, u_mean=0.02))  # bulk tiles for the paired bulk kernels
for geo in geos:
    for storage in ("f32", "f64"):
        for wall in ("elastic", "bounceback"):
            for mode in modes[storage]:
                lat = Lattice(geo.labels, geo.iolets, storage=storage, tau=0.8)
                lat.set_wall(wall, rho0=1.0, F=0.85, kappa=5.0)
                lat.tune(bulk_sites=mode)
                for step in range(5):
                    lat.step(1)
                    lat.sync()  # raises LbmError(LBM_ECHECK) on a violation
                count += 1
                lat.close()
print("CHECKED-OK", count)
"""


def test_every_slot_is_written_once_per_step(tmp_path):
    from paper_2108_08783_gb300 import build
    lib = build.build(out=str(tmp_path / "liblbm_checked.so"), extra=["-DLBM_CHECKED"])
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "CHECKED-OK 80" in r.stdout
