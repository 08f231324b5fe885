"""ctypes front end of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the product package.  It shares no
code with the CUDA path; the only module both sides import is ``lbm_inputs``
(seeded geometries and fields, which hold none of the method's arithmetic).

Every function is a thin marshalling layer over the C oracle; the arithmetic
(equilibrium, collision, streaming, boundary rules, Bessel series) is in C.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

Q = 19


class OrcIolet(C.Structure):
    _fields_ = [("kind", C.c_int32), ("profile", C.c_int32), ("rho", C.c_double),
                ("u_mean", C.c_double), ("u_amp", C.c_double), ("period", C.c_double),
                ("phase", C.c_double), ("centre", C.c_double * 3), ("axis", C.c_double * 3),
                ("radius", C.c_double)]


_lib = None


def lib():
    """Load (building first if needed) the oracle shared object."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.orc_build.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]
    L.orc_build.restype = C.c_int
    for name in ("orc_n_sites", "orc_n_wall_sites", "orc_n_wall_links", "orc_step_count"):
        getattr(L, name).argtypes = [P]
        getattr(L, name).restype = C.c_int64
    L.orc_export.argtypes = [P, P, P, P, P]
    L.orc_configure.argtypes = [P, C.c_double, C.c_int32, C.c_double, P, P, C.c_int64, P, C.c_int32]
    L.orc_configure.restype = C.c_int
    L.orc_run.argtypes = [P, C.c_int64, C.c_int32]
    L.orc_run.restype = C.c_int
    L.orc_init_equilibrium.argtypes = [P, P, P]
    L.orc_set_populations.argtypes = [P, P, C.c_int64]
    L.orc_get_populations.argtypes = [P, P]
    L.orc_moments.argtypes = [P, P, P]
    L.orc_wall_state.argtypes = [P, P, P]
    L.orc_reduce.argtypes = [P, P]
    L.orc_wss.argtypes = [P, P, P, C.c_int64, P]
    L.orc_free.argtypes = [P]
    L.orc_velocity_set.argtypes = [P, P, P]
    L.orc_equilibrium.argtypes = [C.c_double, P, P]
    L.orc_collide.argtypes = [P, C.c_double, P]
    L.orc_bessel_j01.argtypes = [C.c_double, C.c_double, dp, dp]
    L.orc_womersley_shape.argtypes = [C.c_double, C.c_double, dp]
    _lib = L
    return L


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def default_threads():
    return max(1, len(os.sched_getaffinity(0)))


# ---------------------------------------------------------------- pure helpers

def velocity_set():
    """(c [19,3] int32, w [19] float64, opp [19] int32) of the oracle."""
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    lib().orc_velocity_set(_ptr(c), _ptr(w), _ptr(opp))
    return c, w, opp


def equilibrium(rho, u):
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(Q)
    lib().orc_equilibrium(float(rho), _ptr(u), _ptr(out))
    return out


def collide(f, tau):
    f = np.ascontiguousarray(f, np.float64)
    out = np.zeros(Q)
    lib().orc_collide(_ptr(f), float(tau), _ptr(out))
    return out


def bessel_j01(z):
    j0 = (C.c_double * 2)()
    j1 = (C.c_double * 2)()
    lib().orc_bessel_j01(float(np.real(z)), float(np.imag(z)), j0, j1)
    return complex(j0[0], j0[1]), complex(j1[0], j1[1])


def womersley_shape(alpha, xi):
    s = (C.c_double * 2)()
    lib().orc_womersley_shape(float(alpha), float(xi), s)
    return complex(s[0], s[1])


def iolet_struct(io):
    """Marshal an ``lbm_inputs.Iolet`` into the oracle's own struct."""
    s = OrcIolet()
    s.kind = int(io.kind)
    s.profile = int(io.profile)
    s.rho = float(io.rho)
    s.u_mean = float(io.u_mean)
    s.u_amp = float(io.u_amp)
    s.period = float(io.period)
    s.phase = float(io.phase)
    for d in range(3):
        s.centre[d] = float(io.centre[d])
        s.axis[d] = float(io.axis[d])
    s.radius = float(io.radius)
    return s


# ---------------------------------------------------------------- the lattice

class Oracle:
    """One oracle lattice built from voxel labels (0 solid, 1 fluid, 2+k ghost of iolet k)."""

    def __init__(self, labels, iolets=(), tau=0.8, wall_model=1, rho0=1.0, F=0.85, kappa=0.0,
                 threads=None):
        labels = np.ascontiguousarray(labels, np.uint8)
        assert labels.ndim == 3
        self.shape = labels.shape
        self.iolets = list(iolets)
        self.threads = default_threads() if threads is None else int(threads)
        h = C.c_void_p()
        rc = lib().orc_build(_ptr(labels), *[int(v) for v in labels.shape], len(self.iolets),
                             C.byref(h))
        if rc != 0:
            raise ValueError("oracle lattice build failed (%d)" % rc)
        self.h = h
        self.n = lib().orc_n_sites(h)
        self.n_wall = lib().orc_n_wall_sites(h)
        self.n_wall_links = lib().orc_n_wall_links(h)
        self.configure(tau, wall_model, rho0, F, kappa)
        self.init_equilibrium()

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.orc_free(h)
            self.h = None

    def configure(self, tau, wall_model=1, rho0=1.0, F=0.85, kappa=0.0):
        F = np.ascontiguousarray(np.atleast_1d(F), np.float64)
        kappa = np.ascontiguousarray(np.atleast_1d(kappa), np.float64)
        nparam = max(F.size, kappa.size)
        if F.size == 1 and nparam > 1:
            F = np.full(nparam, F[0])
        if kappa.size == 1 and nparam > 1:
            kappa = np.full(nparam, kappa[0])
        arr = (OrcIolet * max(1, len(self.iolets)))(*[iolet_struct(io) for io in self.iolets])
        rc = lib().orc_configure(self.h, float(tau), int(wall_model), float(rho0), _ptr(F),
                                 _ptr(kappa), nparam, C.cast(arr, C.c_void_p), len(self.iolets))
        if rc != 0:
            raise ValueError("oracle configure failed (%d)" % rc)
        self.tau = tau

    def export(self):
        """dict of coords [n,3] int32, nbr [n,18] int64, wall_sites [w], wall_links [l,2]."""
        coords = np.zeros((self.n, 3), np.int32)
        nbr = np.zeros((self.n, 18), np.int64)
        ws = np.zeros(self.n_wall, np.int64)
        wl = np.zeros((self.n_wall_links, 2), np.int64)
        lib().orc_export(self.h, _ptr(coords), _ptr(nbr), _ptr(ws), _ptr(wl))
        return {"coords": coords, "nbr": nbr, "wall_sites": ws, "wall_links": wl}

    def coords(self):
        return self.export()["coords"]

    def init_equilibrium(self, rho=None, u=None):
        rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
        u = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1, 3)
        lib().orc_init_equilibrium(self.h, _ptr(rho), _ptr(u))

    def set_populations(self, f, step=0):
        f = np.ascontiguousarray(f, np.float64).reshape(self.n, Q)
        lib().orc_set_populations(self.h, _ptr(f), int(step))

    def populations(self):
        f = np.zeros((self.n, Q))
        lib().orc_get_populations(self.h, _ptr(f))
        return f

    def run(self, steps, threads=None):
        rc = lib().orc_run(self.h, int(steps), self.threads if threads is None else int(threads))
        if rc != 0:
            raise ValueError("oracle run failed (%d)" % rc)

    @property
    def step(self):
        return lib().orc_step_count(self.h)

    def moments(self):
        rho = np.zeros(self.n)
        u = np.zeros((self.n, 3))
        lib().orc_moments(self.h, _ptr(rho), _ptr(u))
        return rho, u

    def wall_state(self):
        dE = np.zeros(self.n_wall)
        Uw = np.zeros((self.n_wall, 3))
        lib().orc_wall_state(self.h, _ptr(dE), _ptr(Uw))
        return dE, Uw

    def reduce(self):
        out = np.zeros(1 + len(self.iolets))
        lib().orc_reduce(self.h, _ptr(out))
        return out

    def wss(self, sites, normals):
        sites = np.ascontiguousarray(sites, np.int64)
        normals = np.ascontiguousarray(normals, np.float64).reshape(-1, 3)
        out = np.zeros(sites.size)
        lib().orc_wss(self.h, _ptr(sites), _ptr(normals), sites.size, _ptr(out))
        return out
