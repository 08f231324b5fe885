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


if __name__ == "__main__":
    import argparse
    import json
    import lbm_inputs as I
    ap = argparse.ArgumentParser(description="F map and rigid vs elastic WSS agreement")
    ap.add_argument("--M", type=complex, default=complex(0.9, 0.0),
                    help="elastic-tube coefficient M of Eq. F (not fixed by the paper)")
    ap.add_argument("--steps", type=int, default=2400, help="steps from rest before the WSS snapshot")
    ap.add_argument("--depth", type=int, default=6)
    ap.add_argument("--storage", default="f32")
    a = ap.parse_args()
    alpha = [0.5, 1.0, 2.0, 3.0, 4.0, 6.0, 8.0, 10.0]
    drs = [0.01, 0.02, 0.05, 0.1]
    F = np.abs(fmap(alpha, drs, a.M))
    print("|F| for M = %s (rows alpha %s, columns dr/R %s)" % (a.M, alpha, drs))
    for al, row in zip(alpha, F):
        print("  alpha %5.1f: %s" % (al, " ".join("%.4f" % v for v in row)))
    geo = I.murray_tree(seed=0, depth=a.depth, root_radius=48.0)
    geo.iolets[0].u_mean = 0.03
    geo.iolets[0].u_amp = 0.02
    geo.iolets[0].period = 4000.0
    e, r, s = wss_agreement(geo, tau=0.6, F=0.85, kappa=0.75 * 48.0 / 0.5, steps=a.steps,
                            storage=a.storage)
    s["tree"] = "Murray tree depth %d, root R 48 (%d sites), %d steps from rest, pulsatile " \
                "inflow 0.03 + 0.02 sin(2 pi n / 4000)" % (a.depth, geo.n_fluid(), a.steps)
    print(json.dumps(s))
