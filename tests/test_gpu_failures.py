"""Failure paths on the GPU that fault nothing: a device allocator that runs
out of memory part-way through lbm_build_lattice must give LBM_ENOMEM with a
message and hand back every block it was given; a build that succeeds hands
them all back at lbm_destroy."""
import ctypes as C

import numpy as np
import pytest

import lbm_inputs as I

pytestmark = pytest.mark.gpu


def _build_with_failing_allocator(fail_at):
    import torch
    from paper_2108_08783_gb300 import _capi as A
    from paper_2108_08783_gb300.lattice import iolet_struct
    L = A.lib()
    live, given = set(), []

    def alloc(nbytes, user):
        if len(given) >= fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes))
        given.append(p)
        live.add(p)
        return p

    def free(p, user):
        live.discard(p)
        torch.cuda.caching_allocator_delete(p)

    fa, ff = A.ALLOC_FN(alloc), A.FREE_FN(free)
    al = A.LbmAllocator(fa, ff, None)
    geo = I.tube(5, 20, u_mean=0.02)
    labels = np.ascontiguousarray(geo.labels, np.uint8)
    arr = (A.LbmIolet * len(geo.iolets))(*[iolet_struct(io) for io in geo.iolets])
    h = C.c_void_p()
    rc = L.lbm_build_lattice(C.c_void_p(labels.ctypes.data), *labels.shape, C.cast(arr, C.c_void_p),
                             len(geo.iolets), A.LBM_F32, 0.8, C.byref(al),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(h))
    msg = L.lbm_last_error(None).decode()
    if rc == A.LBM_OK:
        L.lbm_destroy(h)
    torch.cuda.synchronize()
    return rc, msg, len(given), live


def test_allocation_failure_is_reported_and_nothing_leaks():
    from paper_2108_08783_gb300 import _capi as A
    ok_at = None
    for fail_at in range(0, 64):
        rc, msg, n_given, live = _build_with_failing_allocator(fail_at)
        assert not live, "blocks not returned after fail_at=%d" % fail_at
        if rc == A.LBM_OK:
            ok_at = fail_at
            break
        assert rc == A.LBM_ENOMEM, (fail_at, rc, msg)
        assert "allocation" in msg
        assert n_given == fail_at
    assert ok_at is not None and ok_at > 5  # the build needs several blocks
