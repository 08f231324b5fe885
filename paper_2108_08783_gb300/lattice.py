"""Python binding of the C ABI: one ``Lattice`` per ``lbm_ctx``.

Only argument marshalling lives here; every step of the method runs in the
library's CUDA kernels.  PyTorch provides device memory (through the caching
allocator, passed to the library as an allocator callback) and the CUDA
stream.
"""
import ctypes as C
import itertools

import numpy as np

from . import _capi as A

STORAGE = {"f64": A.LBM_F64, "f32": A.LBM_F32, "f16s": A.LBM_F16S, "bf16s": A.LBM_BF16S}
WALL = {"bounceback": A.LBM_WALL_BOUNCEBACK, "elastic": A.LBM_WALL_ELASTIC_GZS}


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def default_knobs(storage):
    """The launch knobs a new lattice or ensemble starts with (``lbm_tune``): two
    sites per lane for 16-bit storage, one otherwise; an L2 prefetch distance of
    4096 tiles for FP32 storage, none otherwise; CTAs of 4 warps."""
    sixteen = storage in ("f16s", "bf16s")
    return dict(bulk_sites=2 if sixteen else 1, bulk_warps=4,
                prefetch=4096 if storage == "f32" else 0)


def coordinate_search(apply, timer, knobs, start, trials=2, sweeps=3, margin=0.005):
    """Tune launch knobs by coordinate search from ``start``.

    ``knobs`` lists (name, candidates); a name may be a tuple of knob names
    whose candidates are tuples of values, searched jointly (knobs whose best
    values depend on each other, such as the bulk kernel's sites per lane and
    its prefetch distance, where a search one knob at a time can stop at
    either of two local optima).  Each entry in turn takes every candidate with
    the others held; ``apply(cfg)`` sets a configuration and ``timer()``
    returns the ms of a trial (the first call after ``apply`` only warms up,
    e.g. captures a graph; the best of ``trials`` more is kept).  A candidate
    replaces the current value only when it is faster by more than ``margin``
    (relative), so timing noise does not walk away from the start.  The sweeps
    repeat until one changes nothing, at most ``sweeps`` times.  Returns
    (best, [(cfg, ms)])."""
    best = dict(start)
    results = []

    def measure(cfg):
        apply(cfg)
        timer()
        ms = min(timer() for _ in range(trials))
        results.append((dict(cfg), ms))
        return ms

    for _ in range(sweeps):
        changed = False
        for name, cands in knobs:
            names = name if isinstance(name, tuple) else (name,)
            values = (lambda v: v) if isinstance(name, tuple) else (lambda v: (v,))
            cur = tuple(best[n] for n in names)
            times = {cur: measure(best)}
            for v in cands:
                v = values(v)
                if v not in times:
                    times[v] = measure(dict(best, **dict(zip(names, v))))
            v = min(times, key=times.get)
            if v != cur and times[v] < times[cur] * (1.0 - margin):
                best.update(zip(names, v))
                changed = True
        if not changed:
            break
    apply(best)
    return best, results


def iolet_struct(io):
    """Marshal an iolet description (any object with the ``lbm_iolet`` fields)."""
    s = A.LbmIolet()
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


class _TorchAllocator:
    """lbm_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self._alloc = A.ALLOC_FN(self._do_alloc)
        self._free = A.FREE_FN(self._do_free)
        self.struct = A.LbmAllocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:
            return None

    def _do_free(self, ptr, user):
        try:
            self.torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


class Lattice:
    """A compacted D3Q19 lattice on one GPU (wraps ``lbm_build_lattice``).

    ``labels`` is a uint8 voxel grid [nx, ny, nz] (0 solid, 1 fluid, 2+k ghost
    of iolet k); ``iolets`` the iolet descriptions; ``storage`` one of
    ``f64 f32 f16s bf16s``.
    """

    def __init__(self, labels, iolets=(), storage="f64", tau=0.8, device=0, stream=None,
                 torch_allocator=True):
        import torch
        self._lib = A.lib()
        labels = np.ascontiguousarray(labels, np.uint8)
        assert labels.ndim == 3
        self.shape = labels.shape
        self.storage = storage
        self.tau = float(tau)
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.n_iolets = len(iolets)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self._alloc = _TorchAllocator(self.device, stream) if torch_allocator else None
        arr = (A.LbmIolet * max(1, len(iolets)))(*[iolet_struct(io) for io in iolets])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.lbm_build_lattice(
                _ptr(labels), *[int(v) for v in labels.shape], C.cast(arr, C.c_void_p),
                len(iolets), STORAGE[storage], self.tau,
                C.byref(self._alloc.struct) if self._alloc else None,
                C.c_void_p(stream.cuda_stream), C.byref(h))
        A.check(rc, None)
        self.h = h
        info = self.info()
        self.n = int(info[0])
        self.n_wall = int(info[1])
        self.n_wall_links = int(info[2])

    # ------------------------------------------------------------ lifetime
    def close(self):
        h = getattr(self, "h", None)
        if h is not None:
            self._lib.lbm_destroy(h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        return A.check(rc, self.h)

    # ------------------------------------------------------------ calls
    def info(self):
        out = np.zeros(12, np.int64)
        self._check(self._lib.lbm_info(self.h, _ptr(out)))
        return out

    @property
    def step_count(self):
        return int(self.info()[7])

    def set_wall(self, model="elastic", rho0=1.0, F=0.85, kappa=0.0):
        F = np.ascontiguousarray(np.atleast_1d(F), np.float64)
        kappa = np.ascontiguousarray(np.atleast_1d(kappa), np.float64)
        n = max(F.size, kappa.size)
        if F.size == 1 and n > 1:
            F = np.full(n, F[0])
        if kappa.size == 1 and n > 1:
            kappa = np.full(n, kappa[0])
        self._check(self._lib.lbm_set_wall_params(self.h, WALL[model], float(rho0), _ptr(F),
                                                  _ptr(kappa), n))

    def init_fields(self, rho=None, u=None):
        rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
        u = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1, 3)
        self._check(self._lib.lbm_init_fields(self.h, _ptr(rho), _ptr(u)))

    def step(self, n=1):
        self._check(self._lib.lbm_step(self.h, int(n)))

    def step_diag(self, n=1, out=None):
        """``lbm_step_diag``: n steps, the last of which also reduces the mass and
        iolet fluxes of the state it reads into ``out`` (float64 [1 + n_iolets],
        complete after the next sync)."""
        if out is None:
            out = np.zeros(1 + self.n_iolets)
        self._check(self._lib.lbm_step_diag(self.h, int(n), _ptr(out)))
        return out

    def sync(self):
        self._check(self._lib.lbm_sync(self.h))

    def moments(self):
        rho = np.zeros(self.n)
        u = np.zeros((self.n, 3))
        self._check(self._lib.lbm_moments(self.h, _ptr(rho), _ptr(u), 0))
        return rho, u

    def moments_into(self, rho, u):
        """Write moments into device tensors (float64 [n], [n,3]) asynchronously."""
        self._check(self._lib.lbm_moments(self.h, C.c_void_p(rho.data_ptr()),
                                          C.c_void_p(u.data_ptr()), 1))

    def warm_features(self, frame, targets=True):
        """Per-site features x [n][n_global + 2] and (optionally) targets t [n][3]
        from the current fields, as device tensors (``lbm_warm_features``)."""
        import torch
        x = torch.empty((self.n, frame.n_global + 2), dtype=torch.float32, device=self.device)
        t = torch.empty((self.n, 3), dtype=torch.float32, device=self.device) if targets else None
        self._check(self._lib.lbm_warm_features(self.h, C.byref(frame), C.c_void_p(x.data_ptr()),
                                                C.c_void_p(t.data_ptr()) if targets else None))
        return x, t

    def warm_start(self, net, frame):
        """Initial fields proposed by the network ``net`` (an MLP) for this
        lattice, f = f^eq(rho, u) (``lbm_warm_start``)."""
        self._check(self._lib.lbm_warm_start(self.h, net.h, C.byref(frame)))

    def export(self):
        coords = np.zeros((self.n, 3), np.int32)
        nbr = np.zeros((self.n, 18), np.int32)
        ws = np.zeros(self.n_wall, np.int64)
        wl = np.zeros((self.n_wall_links, 2), np.int64)
        self._check(self._lib.lbm_export_lattice(self.h, _ptr(coords), _ptr(nbr), _ptr(ws),
                                                 _ptr(wl)))
        return {"coords": coords, "nbr": nbr, "wall_sites": ws, "wall_links": wl}

    def coords(self):
        coords = np.zeros((self.n, 3), np.int32)
        self._check(self._lib.lbm_export_lattice(self.h, _ptr(coords), None, None, None))
        return coords

    def wall_state(self):
        dE = np.zeros(self.n_wall)
        Uw = np.zeros((self.n_wall, 3))
        self._check(self._lib.lbm_wall_state(self.h, _ptr(dE), _ptr(Uw)))
        return dE, Uw

    def reduce(self):
        out = np.zeros(1 + self.n_iolets)
        self._check(self._lib.lbm_reduce(self.h, _ptr(out)))
        return out

    def populations(self):
        f = np.zeros((self.n, 19))
        self._check(self._lib.lbm_get_populations(self.h, _ptr(f), 0))
        return f

    def set_populations(self, f, step=0):
        f = np.ascontiguousarray(f, np.float64).reshape(self.n, 19)
        self._check(self._lib.lbm_set_populations(self.h, _ptr(f), int(step), 0))

    def checkpoint(self):
        nb = self._lib.lbm_checkpoint_bytes(self.h)
        buf = np.zeros(nb, np.uint8)
        self._check(self._lib.lbm_checkpoint_save(self.h, _ptr(buf), nb))
        return buf

    def restore(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        self._check(self._lib.lbm_checkpoint_load(self.h, _ptr(buf), buf.size))

    def profile(self, enable=True):
        self._check(self._lib.lbm_profile(self.h, 1 if enable else 0))

    def tune(self, prefetch=None, bulk_sites=None, bulk_warps=None, graph_steps=None):
        """Launch knobs (``lbm_tune``): L2 prefetch distance of the bulk kernel in
        tiles, the bulk kernel's sites per lane and their pairing (1 to 4), and
        its warps per CTA (4 or 8)."""
        if prefetch is not None:
            self._check(self._lib.lbm_tune(self.h, A.LBM_TUNE_PREFETCH, int(prefetch)))
        if bulk_sites is not None:
            self._check(self._lib.lbm_tune(self.h, A.LBM_TUNE_BULK_SITES, int(bulk_sites)))
        if bulk_warps is not None:
            self._check(self._lib.lbm_tune(self.h, A.LBM_TUNE_BULK_WARPS, int(bulk_warps)))
        if graph_steps is not None:
            self._check(self._lib.lbm_tune(self.h, A.LBM_TUNE_GRAPH_STEPS, int(graph_steps)))

    def time_steps(self, n):
        """Device ms of n steps (CUDA events on the lattice's stream)."""
        import torch
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        self.sync()
        e0.record(self.stream)
        self.step(n)
        e1.record(self.stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def autotune(self, bulk_sites=(1, 2, 3, 4), bulk_warps=(4, 8), prefetch=(0, 2048, 4096),
                 graph_steps=(20, 0), trial_steps=40, trials=2, sweeps=3):
        """Choose the bulk kernel's site tile (one site per lane, a 32-site tile per
        warp; or two per lane, 64 sites per warp, paired as adjacent sites or as
        two tiles), its CTA size, its L2 prefetch distance and graph replay by
        timing each candidate on this lattice (``coordinate_search`` from the
        library's defaults, sites per lane and prefetch distance jointly;
        ``trials`` and ``sweeps`` as there).  Every trial, and the warm-up run
        before each candidate's trials, advances the lattice by ``trial_steps``
        steps (an even number keeps both parities equal)."""
        if self.storage == "f64":
            bulk_sites = (1,)
        elif self.storage in ("f16s", "bf16s") and 5 not in bulk_sites:
            bulk_sites = tuple(bulk_sites) + (5,)  # TMA-staged even steps
        start = dict(default_knobs(self.storage), graph_steps=20)
        knobs = ((("bulk_sites", "prefetch"), list(itertools.product(bulk_sites, prefetch))),
                 ("bulk_warps", bulk_warps), ("graph_steps", graph_steps))
        return coordinate_search(lambda cfg: self.tune(**cfg),
                                 lambda: self.time_steps(trial_steps), knobs, start,
                                 trials=trials, sweeps=sweeps)

    def profile_read(self):
        """Since profile(True): ((step ms, bulk-kernel ms), (bulk launches, boundary launches))."""
        ms = np.zeros(2)
        n = np.zeros(2, np.int64)
        self._check(self._lib.lbm_profile_read(self.h, _ptr(ms), _ptr(n)))
        return (float(ms[0]), float(ms[1])), (int(n[0]), int(n[1]))

    def wss(self, sites, normals):
        sites = np.ascontiguousarray(sites, np.int64)
        normals = np.ascontiguousarray(normals, np.float64).reshape(-1, 3)
        out = np.zeros(sites.size)
        self._check(self._lib.lbm_wss(self.h, _ptr(sites), _ptr(normals), sites.size, _ptr(out)))
        return out


class Ensemble:
    """Many independent lattices advanced by one launch of each step kernel per
    timestep (wraps ``lbm_ensemble_create``).  The member Lattices stay owned
    by the caller and must outlive the ensemble; call :meth:`sync` before
    using a member's own methods."""

    def __init__(self, lattices):
        self._lib = A.lib()
        self.members = list(lattices)
        arr = (C.c_void_p * len(self.members))(*[m.h.value for m in self.members])
        h = C.c_void_p()
        rc = self._lib.lbm_ensemble_create(arr, len(self.members), C.byref(h))
        if rc != A.LBM_OK:
            raise A.LbmError(rc, "lbm_ensemble_create failed")
        self.h = h
        self.stream = self.members[0].stream  # the ensemble's work is ordered with it
        self.n = sum(m.n for m in self.members)
        self.settings = {"prefetch": None, "schedule": 0, "graph_steps": 0, "persistent": 0,
                         "bulk_sites": None, "bulk_warps": 4}

    def _check(self, rc):
        if rc != A.LBM_OK:
            raise A.LbmError(rc, self._lib.lbm_ensemble_last_error(self.h).decode())

    def step(self, n=1):
        self._check(self._lib.lbm_ensemble_step(self.h, int(n)))

    def sync(self):
        self._check(self._lib.lbm_ensemble_sync(self.h))

    def tune(self, prefetch=None, schedule=None, graph_steps=None, persistent=None,
             barrier_extra=None, bulk_sites=None, bulk_warps=None):
        if prefetch is not None:
            self._check(self._lib.lbm_ensemble_tune(self.h, A.LBM_TUNE_PREFETCH, int(prefetch)))
            self.settings["prefetch"] = int(prefetch)
        if schedule is not None:
            self._check(self._lib.lbm_ensemble_tune(self.h, A.LBM_TUNE_SCHEDULE, int(schedule)))
            self.settings["schedule"] = int(schedule)
        if graph_steps is not None:
            self._check(self._lib.lbm_ensemble_tune(self.h, A.LBM_TUNE_GRAPH_STEPS,
                                                    int(graph_steps)))
            self.settings["graph_steps"] = int(graph_steps)
        if persistent is not None:
            self._check(self._lib.lbm_ensemble_tune(self.h, A.LBM_TUNE_PERSISTENT,
                                                    int(persistent)))
            self.settings["persistent"] = int(persistent)
        if barrier_extra is not None:
            self._check(self._lib.lbm_ensemble_tune(self.h, A.LBM_TUNE_BARRIER_EXTRA,
                                                    int(barrier_extra)))
        if bulk_sites is not None:
            self._check(self._lib.lbm_ensemble_tune(self.h, A.LBM_TUNE_BULK_SITES,
                                                    int(bulk_sites)))
            self.settings["bulk_sites"] = int(bulk_sites)
        if bulk_warps is not None:
            self._check(self._lib.lbm_ensemble_tune(self.h, A.LBM_TUNE_BULK_WARPS,
                                                    int(bulk_warps)))
            self.settings["bulk_warps"] = int(bulk_warps)

    def time_steps(self, n):
        """Device ms of n steps (CUDA events on the ensemble's stream)."""
        import torch
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        self.sync()
        e0.record(self.stream)
        self.step(n)
        e1.record(self.stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def autotune(self, prefetch=(0, 1024, 2048, 4096, 8192), schedule=(0, 1),
                 graph_steps=(0, 20), persistent=(0, 1), bulk_sites=(1, 2, 3, 4),
                 bulk_warps=(4, 8), trial_steps=40, trials=2, sweeps=3):
        """Choose the schedule knobs by timing each candidate on this ensemble
        (``coordinate_search`` from the library's defaults, sites per lane and
        prefetch distance jointly): member order, the bulk kernel's site tile
        (one site per lane, 32 sites per warp; or two per lane, 64 per warp,
        paired as adjacent sites or as two tiles), its CTA size and L2 prefetch
        distance, graph replay and the persistent kernel (``trials`` and
        ``sweeps`` as there).  Every trial, and the warm-up run before each
        candidate's trials, advances the members by ``trial_steps`` steps."""
        storage = self.members[0].storage
        if storage == "f64":
            bulk_sites = (1,)
        start = dict(default_knobs(storage), schedule=0, graph_steps=0, persistent=0)
        knobs = (("schedule", schedule),
                 (("bulk_sites", "prefetch"), list(itertools.product(bulk_sites, prefetch))),
                 ("bulk_warps", bulk_warps), ("graph_steps", graph_steps),
                 ("persistent", persistent))
        return coordinate_search(lambda cfg: self.tune(**cfg),
                                 lambda: self.time_steps(trial_steps), knobs, start,
                                 trials=trials, sweeps=sweeps)

    def close(self):
        h = getattr(self, "h", None)
        if h is not None:
            self._lib.lbm_ensemble_destroy(h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
