"""The paper's workflow around the hot path (Sec. 2.3 F map; Sec. 3 rigid vs
elastic wall-shear-stress agreement), on the library's own calls.

``fmap`` wraps the host precompute ``lbm_fmap``; ``wss_agreement`` runs one
geometry twice on the GPU (rigid bounce-back wall and elastic wall, same
inflow) and compares the instantaneous wall shear stress at every wall site
with Bland-Altman limits of agreement (bias +- 1.96 standard deviations of
the differences), the statistic of the paper's Sec. 3 comparison.
"""
import ctypes as C

import numpy as np

from . import _capi as A


def fmap(alpha, dr_over_R, M):
    """Complex F on the grid alpha x dr_over_R (``lbm_fmap``), shape
    [len(alpha)][len(dr_over_R)]."""
    a = np.ascontiguousarray(np.atleast_1d(alpha), np.float64)
    d = np.ascontiguousarray(np.atleast_1d(dr_over_R), np.float64)
    out = np.zeros((a.size, d.size, 2))
    M = complex(M)
    rc = A.lib().lbm_fmap(C.c_void_p(a.ctypes.data), a.size, C.c_void_p(d.ctypes.data), d.size,
                          M.real, M.imag, C.c_void_p(out.ctypes.data))
    if rc != A.LBM_OK:
        raise A.LbmError(rc, "lbm_fmap: arguments out of range")
    return out[..., 0] + 1j * out[..., 1]


def limits_of_agreement(a, b):
    """Bland-Altman statistics of paired samples (a, b): bias = mean(a - b),
    limits bias +- 1.96 sd(a - b), and the fraction of pairs with a < b."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = a - b
    bias = float(d.mean())
    sd = float(d.std(ddof=1)) if d.size > 1 else 0.0
    return dict(n=int(d.size), bias=bias, lower=bias - 1.96 * sd, upper=bias + 1.96 * sd,
                sd=sd, mean_a=float(a.mean()), mean_b=float(b.mean()),
                frac_a_below_b=float(np.mean(d < 0)))


def wss_agreement(geo, tau, F, kappa, steps, storage="f32", rho0=1.0):
    """Instantaneous WSS at every wall site after ``steps`` steps from rest,
    elastic wall (F, kappa) against rigid bounce-back; returns
    (wss_elastic, wss_rigid, limits_of_agreement(elastic, rigid))."""
    import lbm_inputs as I
    from . import Lattice
    out = {}
    for model in ("elastic", "bounceback"):
        lat = Lattice(geo.labels, geo.iolets, storage=storage, tau=tau)
        if model == "elastic":
            lat.set_wall("elastic", rho0=rho0, F=F, kappa=kappa)
        else:
            lat.set_wall("bounceback")
        lat.step(steps)
        lat.sync()
        ex = lat.export()
        s = ex["wall_sites"]
        out[model] = lat.wss(s, I.wall_normals(geo, ex["coords"][s]))
        lat.close()
    return out["elastic"], out["bounceback"], limits_of_agreement(out["elastic"],
                                                                  out["bounceback"])
