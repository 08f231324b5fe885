"""Error model of shifted 16-bit population storage (test helper, CPU).

Each step rounds every stored g_i = f_i - w_i once, to the storage's
significand: an error uniform within +-u_s |g_i| (rms u_s |g_i| / sqrt 3),
with u_s = 2^-11 for binary16 (11-bit significand) and 2^-8 for bfloat16
(8 bits).  The collision conserves mass and momentum, so it does not damp the
errors of those moments: they add like a random walk over the steps
(sqrt(steps)).  Per site the rounding of the 19 values adds sqrt(sum g_i^2)
to the error of rho - 1 = sum g_i, and sqrt(sum g_i^2 |c_i|^2) to that of
rho u.  The parity tests bound the GPU's error by BOUND_FACTOR times this
estimate; the CPU test of this module checks the estimate against the FP64
oracle with its stored populations rounded the same way.
"""
import numpy as np

UNIT_ROUNDOFF = {"f16s": 2.0 ** -11, "bf16s": 2.0 ** -8}
BOUND_FACTOR = 4.0


def rounding_walk_estimate(orc, steps):
    """(e_rho, e_u): the expected rel-L2 errors of (rho - 1) and of u after
    `steps` steps are u_s e_rho and u_s e_u, from the oracle's current fields."""
    from oracle import velocity_set
    c, w, _ = velocity_set()
    c = c.astype(np.float64)
    g = orc.populations() - w
    rho, u = orc.moments()
    walk = np.sqrt(steps) / np.sqrt(3.0)
    s_rho = np.sqrt(np.mean(np.sum(g * g, 1)))
    s_j = np.sqrt(np.mean(np.sum(g * g * np.sum(c * c, 1)[None], 1)))
    e_rho = walk * s_rho / np.sqrt(np.mean((rho - 1.0) ** 2))
    e_u = walk * s_j / np.sqrt(np.mean(np.sum((rho[:, None] * u) ** 2, 1)))
    return e_rho, e_u


def round_storage(g, storage):
    """g (float64) rounded to the storage format (to nearest, ties to even), as float64."""
    if storage == "f16s":
        return g.astype(np.float16).astype(np.float64)
    if storage == "bf16s":
        b = np.ascontiguousarray(g, np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(storage)
