"""Host logic of the lattice build on the CPU (no GPU): lbm_plan_lattice runs
the library's compaction and tile classification alone; its counts must match
the oracle's own builder (sites, wall sites, wall links) and a numpy
restatement of the tile classes (bulk: no link leaves the fluid and every
direction has one offset for the whole tile; coherent boundary: some links
leave the fluid but each direction's fluid links share one offset;
irregular: otherwise)."""
import ctypes as C

import numpy as np
import pytest

import lbm_inputs as I

D = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
     (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1),
     (0, 1, -1), (0, -1, 1)]


@pytest.fixture(scope="module")
def capi():
    from paper_2108_08783_gb300 import build
    build.build()
    from paper_2108_08783_gb300 import _capi
    return _capi


def _plan(capi, geo, tau=0.8):
    from paper_2108_08783_gb300.lattice import iolet_struct
    labels = np.ascontiguousarray(geo.labels, np.uint8)
    arr = (capi.LbmIolet * max(1, len(geo.iolets)))(*[iolet_struct(io) for io in geo.iolets])
    out = np.zeros(8, np.int64)
    rc = capi.lib().lbm_plan_lattice(C.c_void_p(labels.ctypes.data), *labels.shape,
                                     C.cast(arr, C.c_void_p), len(geo.iolets), tau,
                                     C.c_void_p(out.ctypes.data))
    assert rc == 0, capi.lib().lbm_last_error(None).decode()
    return out


def _classes(labels):
    """(bulk tiles, coherent tiles, irregular tiles, bulk sites) by brute force."""
    nx, ny, nz = labels.shape
    idx = np.flatnonzero((labels == 1).ravel())
    n = idx.size
    site = -np.ones(labels.size, np.int64)
    site[idx] = np.arange(n)
    x, y, z = np.unravel_index(idx, labels.shape)
    off = np.empty((18, n), np.int64)
    for k, (a, b, c) in enumerate(D):
        xx, yy, zz = x + a, y + b, z + c
        ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        j = np.ravel_multi_index((np.clip(xx, 0, nx - 1), np.clip(yy, 0, ny - 1),
                                  np.clip(zz, 0, nz - 1)), labels.shape)
        v = np.where(ok, site[j], -1)
        off[k] = np.where(v >= 0, v - np.arange(n), np.iinfo(np.int64).min)
    bulk = coh = irr = bulk_sites = 0
    for t in range((n + 31) // 32):
        o = off[:, t * 32:(t + 1) * 32]
        fluid = o != np.iinfo(np.int64).min
        uniform = all(np.unique(o[k][fluid[k]]).size <= 1 for k in range(18))
        if not uniform:
            irr += 1
        elif fluid.all():
            bulk += 1
            bulk_sites += o.shape[1]
        else:
            coh += 1
    return bulk, coh, irr, bulk_sites


GEOMETRIES = [
    I.tube(6, 40, u_mean=0.02), I.tube(5.5, 33, u_mean=0.02), I.duct(7, 5, 33),
    I.closed_box(9, 11, 13), I.murray_tree(seed=2, depth=2, root_radius=6.0),
] + [I.random_labels(s, (10, 12, 37), fill=0.7) for s in range(3)]


@pytest.mark.parametrize("geo", GEOMETRIES, ids=lambda g: g.name)
def test_plan_matches_oracle_builder_and_tile_classes(capi, geo):
    from oracle import Oracle
    p = _plan(capi, geo)
    orc = Oracle(geo.labels, geo.iolets, tau=0.8)
    ex = orc.export()
    assert p[0] == orc.n
    assert p[1] == len(ex["wall_sites"])
    assert p[2] == len(ex["wall_links"])
    assert p[3] == (orc.n + 31) // 32
    assert tuple(p[[4, 5, 6, 7]]) == _classes(np.asarray(geo.labels))


def test_plan_rejects_what_the_build_rejects(capi):
    geo = I.tube(4, 8)
    bad = np.array(geo.labels)
    bad[0, 0, 0] = 9  # label beyond 2 + n_iolets
    from paper_2108_08783_gb300.lattice import iolet_struct
    arr = (capi.LbmIolet * 2)(*[iolet_struct(io) for io in geo.iolets])
    out = np.zeros(8, np.int64)
    rc = capi.lib().lbm_plan_lattice(C.c_void_p(np.ascontiguousarray(bad).ctypes.data),
                                     *bad.shape, C.cast(arr, C.c_void_p), 2, 0.8,
                                     C.c_void_p(out.ctypes.data))
    assert rc == -1
    assert capi.lib().lbm_last_error(None).decode()
