"""lbm_reduce_noalloc against lbm_reduce, through the C ABI.

lbm_reduce_noalloc serves callers that must not allocate device memory during
the call (a hook running while another memory pool owns the device, or a loop
that cannot take cudaMalloc's synchronisation); its scratch is a fixed device
array inside the library.  Both calls run the same reduction kernels with the
same grid on the same state, so their results must be equal bit for bit: a
partial or an output slot left over from an earlier call would show.  This
file is collected last so that a failure here leaves every other test already
run; it also passes on its own in a fresh process, where its first call
performs the per-device set-up.
"""
import ctypes as C

import numpy as np
import pytest

import lbm_inputs as I

pytestmark = pytest.mark.gpu


def _p(a):
    return C.c_void_p(a.ctypes.data)


def _lattice(geo, storage="f64"):
    from paper_2108_08783_gb300 import Lattice
    lat = Lattice(geo.labels, geo.iolets, storage=storage, tau=0.8)
    lat.set_wall("elastic", rho0=1.0, F=0.85, kappa=12.0)
    return lat


def _noalloc_host(lib, lat, n_out):
    out = np.full(n_out, np.nan)
    rc = lib.lbm_reduce_noalloc(lat.h, _p(out), 0)
    assert rc == 0, lib.lbm_last_error(lat.h)
    return out


def test_reduce_noalloc_matches_reduce_on_consecutive_calls():
    import torch
    from paper_2108_08783_gb300 import _capi
    geo = I.tube(8, 64, u_mean=0.025)
    lat = _lattice(geo)
    lib = _capi.lib()
    n_out = 1 + len(geo.iolets)
    for chunk in (37, 40):  # odd, then even storage layout
        lat.step(chunk)
        ref = lat.reduce()
        for _ in range(2):  # two calls in a row
            np.testing.assert_array_equal(_noalloc_host(lib, lat, n_out), ref)
        dev = torch.full((n_out,), float("nan"), dtype=torch.float64, device="cuda")
        for _ in range(2):
            dev.fill_(float("nan"))
            rc = lib.lbm_reduce_noalloc(lat.h, C.c_void_p(dev.data_ptr()), 1)
            assert rc == 0, lib.lbm_last_error(lat.h)
            lat.sync()
            np.testing.assert_array_equal(dev.cpu().numpy(), ref)
    lat.close()


def test_reduce_noalloc_after_a_lattice_with_another_iolet_count():
    """Calls alternate between a tree (one inlet, eight leaf outlets) and a tube
    (two iolets) in FP32: the shared array holds the other lattice's partials
    and outputs each time, and every result still equals lbm_reduce's."""
    from paper_2108_08783_gb300 import _capi
    lib = _capi.lib()
    tree = I.murray_tree(seed=1, depth=3, root_radius=10.0)
    tree.iolets[0].u_mean = 0.02
    tube = I.tube(6, 48, u_mean=0.02)
    lats = [(_lattice(tree, "f32"), 1 + len(tree.iolets)), (_lattice(tube, "f32"), 1 + len(tube.iolets))]
    assert lats[0][1] != lats[1][1]
    for rnd in range(3):
        for lat, n_out in (lats if rnd % 2 == 0 else lats[::-1]):
            lat.step(7 + rnd)
            ref = lat.reduce()
            assert np.all(np.isfinite(ref)) and np.any(ref[1:] != 0.0)
            np.testing.assert_array_equal(_noalloc_host(lib, lat, n_out), ref)
    for lat, _ in lats:
        lat.close()
