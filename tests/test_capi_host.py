"""Host-side checks of the C-ABI library that need no GPU.

The library is built here (nvcc cross-compiles sm_103a) and loaded; every
symbol include/lbm.h declares must be exported.  Input validation of
lbm_build_lattice happens before any CUDA call, so its error paths are tested
on the CPU too.  No compute call is made.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import lbm_inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2108_08783_gb300 import build
    build.build()
    from paper_2108_08783_gb300 import _capi
    return _capi


def _declared():
    names = set()
    for h in ("lbm.h", "lbm_mlp.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_core_calls():
    names = _declared()
    for n in ("lbm_build_lattice", "lbm_set_wall_params", "lbm_step", "lbm_moments"):
        assert n in names


def test_library_exports_every_declared_symbol(capi):
    lib = C.CDLL(capi.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(capi.EXPORTS) == _declared()


def _build(capi, labels, iolets=(), storage=0, tau=0.8):
    from paper_2108_08783_gb300.lattice import iolet_struct
    L = capi.lib()
    labels = np.ascontiguousarray(labels, np.uint8)
    arr = (capi.LbmIolet * max(1, len(iolets)))(*[iolet_struct(io) for io in iolets])
    h = C.c_void_p()
    rc = L.lbm_build_lattice(C.c_void_p(labels.ctypes.data), *labels.shape,
                             C.cast(arr, C.c_void_p), len(iolets), storage, tau, None, None,
                             C.byref(h))
    return rc, L.lbm_last_error(None).decode(), h


def test_build_rejects_bad_inputs_before_touching_the_gpu(capi):
    g = I.tube(4, 8)
    rc, msg, h = _build(capi, g.labels, g.iolets, tau=0.5)
    assert rc == capi.LBM_EINVAL and "tau" in msg and not h.value
    rc, msg, _ = _build(capi, g.labels, g.iolets, storage=7)
    assert rc == capi.LBM_EINVAL and "storage" in msg
    rc, msg, _ = _build(capi, g.labels, g.iolets[:1])  # label 3 without iolet 1
    assert rc == capi.LBM_EINVAL and "label" in msg
    bad = I.Iolet(kind=0, centre=(0, 0, 0), axis=(0.0, 0.0, 0.0), radius=4.0)
    rc, msg, _ = _build(capi, g.labels, [bad, g.iolets[1]])
    assert rc == capi.LBM_EINVAL and "iolet 0" in msg
    # one fluid site touching two different velocity inlets
    lab = np.zeros((3, 3, 3), np.uint8)
    lab[1, 1, 1] = 1
    lab[1, 1, 0] = 2
    lab[1, 1, 2] = 3
    vel = I.Iolet(kind=0, centre=(1, 1, 0), axis=(0.0, 0.0, 1.0), radius=2.0)
    rc, msg, _ = _build(capi, lab, [vel, vel])
    assert rc == capi.LBM_EINVAL and "two velocity inlets" in msg
    rc, msg, _ = _build(capi, np.zeros((0, 3, 3), np.uint8))
    assert rc == capi.LBM_EINVAL


def test_status_strings(capi):
    assert capi.status_name(capi.LBM_EUNSTABLE) == "LBM_EUNSTABLE"
    assert capi.status_name(capi.LBM_OK) == "LBM_OK"


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2108_08783_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            text = open(os.path.join(dirpath, f), errors="ignore").read() if f.endswith(
                (".py", ".cu", ".cpp", ".h")) else ""
            assert not re.search(r"^\s*(from|import)\s+oracle", text, re.M), f
            assert "liboracle" not in text and "lbm_oracle" not in text, f
