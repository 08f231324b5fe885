"""lbm_reduce_noalloc against lbm_reduce, through the C ABI.

lbm_reduce_noalloc serves callers that must not allocate device memory during
the call (a hook running while another memory pool owns the device, or a loop
that cannot take cudaMalloc's synchronisation); its scratch is a fixed device
array inside the library.  This file is collected last so that a failure here
leaves every other test already run; it also passes on its own in a fresh
process, where its first call performs the per-device set-up.
"""
import ctypes as C

import numpy as np
import pytest

import lbm_inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance used by the other GPU tests


def _p(a):
    return C.c_void_p(a.ctypes.data)


def test_reduce_noalloc_matches_reduce_on_consecutive_calls():
    import torch
    from paper_2108_08783_gb300 import Lattice, _capi
    geo = I.tube(8, 64, u_mean=0.025)
    lat = Lattice(geo.labels, geo.iolets, storage="f64", tau=0.8)
    lat.set_wall("elastic", rho0=1.0, F=0.85, kappa=12.0)
    lib = _capi.lib()
    n_out = 1 + len(geo.iolets)
    for chunk in (37, 40):  # odd, then even storage layout
        lat.step(chunk)
        ref = lat.reduce()
        for _ in range(2):  # two calls in a row
            out = np.zeros(n_out)
            rc = lib.lbm_reduce_noalloc(lat.h, _p(out), 0)
            assert rc == 0, lib.lbm_last_error(lat.h)
            np.testing.assert_allclose(out, ref, rtol=TOL, atol=0)
        dev = torch.zeros(n_out, dtype=torch.float64, device="cuda")
        for _ in range(2):
            dev.zero_()
            rc = lib.lbm_reduce_noalloc(lat.h, C.c_void_p(dev.data_ptr()), 1)
            assert rc == 0, lib.lbm_last_error(lat.h)
            lat.sync()
            np.testing.assert_allclose(dev.cpu().numpy(), ref, rtol=TOL, atol=0)
    lat.close()
