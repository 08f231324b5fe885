"""Benchmark of the elastic-wall D3Q19 LBGK step on GB300 (one JSON line).

Workload (default): the long pulsatile tube - radius 40, length 1024,
~5.15 M fluid sites, tau 0.6, inlet 0.03 + 0.02 sin(2 pi n / 4000) (parabolic),
density outlet rho = 1, elastic wall F = 0.85 with Eh/r0 = 0.5
(kappa = 0.75 * 40 / 0.5 = 60), populations in FP32 (``--storage``).
A "step" is one full timestep of the lattice (both kernels).  The populations
(19 * 4 B * 5.15 M = 391 MB per copy) exceed the 129 MB L2, so no flush is
needed between steps.

  value      site updates per second (MLUPS) over the timed device region,
             CUDA events on the lattice's stream, max over ranks;
  e2e        the same metric through the public C ABI with host buffers:
             initial fields copied in from pinned memory, every step followed
             by lbm_reduce (FP64 mass and iolet fluxes read back to the host),
             final moments copied out - all inside the timed region;
  roofline   one step (k_bulk on the lattice's stream with k_boundary beside it
             on a side stream): algorithmic bytes (2 * 19 * sizeof(storage) per
             site update) / the step's CUDA-event duration (fork to join),
             against the measured HBM copy bandwidth; traffic = ncu DRAM bytes of
             the same step when the recorded kernel source matches;
  cpu_baseline  the FP64 CPU oracle on the same workload, a bounded number of
             steps on all host cores;
  wall_cost  ms per step with the elastic wall and with rigid bounce-back on the
             same workload (the paper reports the elastic step no dearer);
  mixed_precision  every storage (FP64/FP32/FP16S/BF16S) run from rest on the
             same workload: MLUPS, speed-up over FP32 and the rel-L2 error of
             the wall shear stress and of u against the FP64 path (which
             matches the FP64 oracle to 1e-10), a table with no chosen error
             budget;
  tree       the seeded depth-6 Murray tree (10.25 M sites, 43 % of its tiles
             irregular): MLUPS, step roofline fraction and WSS error against
             the FP64 path for FP32, FP16S and BF16S storage;
  ensemble   256 seeded elastic tubes (63.5 M sites) batched into one launch
             per step kernel, autotuned: FP16S and FP32 MLUPS, FP32 stepped
             one lattice at a time, and the WSS error of every storage
             against the FP64 path on a 32-member subset.

``--impl reference`` times the oracle alone (the reference arm of this tier).
Under torchrun every rank runs its own copy of the workload (independent
vessels, no data-path collective): weak scaling.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

BYTES = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}
# lbm_step's default graph block (LBM_TUNE_GRAPH_STEPS): whole blocks of 20 steps
# replay a captured graph that also launches one k_advance (the device step
# counter) after its steps
GRAPH_STEPS = 20
DTYPE = {"f64": "f64", "f32": "f32", "f16s": "f32", "bf16s": "f32"}
METRIC = "elastic-wall D3Q19 MLUPS & % HBM roofline; mixed-prec vs FP32 at fixed error"


def workload(args):
    import lbm_inputs as I
    if args.config == "tube40":
        geo = I.tube(40, 1024, u_mean=0.03, u_amp=0.02, period=4000.0)
        params = dict(tau=0.6, F=0.85, kappa=0.75 * 40 / 0.5, rho0=1.0)
        name = "long pulsatile tube R=40 L=1024 (~5.15M sites), tau=0.6, Eh/r0=0.5"
    elif args.config == "tree":
        geo, params = tree_workload()
        name = ("seeded Murray tree depth 6, root R=48, 10%% taper (%d sites), tau=0.6, Eh/r0=0.5"
                % geo.n_fluid())
    elif args.config == "tube8":
        geo = I.tube(8, 64, u_mean=0.025)
        params = dict(tau=0.8, F=0.85, kappa=12.0, rho0=1.0)
        name = "straight cylinder R=8 L=64 (~13k sites), tau=0.8, Eh/r0=0.5"
    else:
        raise SystemExit("unknown config " + args.config)
    return geo, params, name


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_traffic(storage, config):
    """DRAM bytes of one step (its bulk and boundary launches, mean of an odd and
    an even step) from the committed ncu summary, or None if the kernel source
    changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        src = open(os.path.join(ROOT, "paper_2108_08783_gb300", "csrc", "kernels.cu"), "rb").read()
        key = "%s/%s" % (config, storage)
        if key in rec and rec[key]["kernels_sha1"] == hashlib.sha1(src).hexdigest():
            return float(rec[key]["bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle(geo, params, seconds=12.0, max_steps=200, min_steps=2, threads=None):
    """MLUPS of the FP64 oracle over a time-bounded sample (all host cores by
    default)."""
    from oracle import Oracle
    from oracle.oracle import default_threads
    threads = threads or default_threads()
    orc = Oracle(geo.labels, geo.iolets, tau=params["tau"], wall_model=1, F=params["F"],
                 kappa=params["kappa"], rho0=params["rho0"], threads=threads)
    orc.run(1)  # page in
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps and (steps < min_steps or time.perf_counter() - t0 < seconds):
        orc.run(1)
        steps += 1
    dt = time.perf_counter() - t0
    return orc.n * steps / dt / 1e6, threads, steps, dt


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "CPU part", "Model"):
                    return v.strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_short_tube_full_run():
    """Wall seconds of the oracle's full run of the short tube (R = 8, L = 64, 2000
    steps from rest, all host cores)."""
    from oracle import Oracle
    import lbm_inputs as I
    geo = I.tube(8, 64, u_mean=0.025)
    orc = Oracle(geo.labels, geo.iolets, tau=0.8, wall_model=1, F=0.85, kappa=12.0, rho0=1.0)
    t0 = time.perf_counter()
    orc.run(2000)
    return time.perf_counter() - t0, orc.n


def wall_cost(args, geo, params, steps=2000):
    """ms per step of the elastic wall and of rigid bounce-back on the same
    workload and storage (the paper finds the elastic step no dearer)."""
    import torch
    from paper_2108_08783_gb300 import Lattice
    out = {}
    for model in ("elastic", "bounceback"):
        lat = Lattice(geo.labels, geo.iolets, storage=args.storage, tau=params["tau"])
        if model == "elastic":
            lat.set_wall("elastic", rho0=params["rho0"], F=params["F"], kappa=params["kappa"])
        else:
            lat.set_wall("bounceback")
        lat.step(20)
        lat.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        lat.step(steps)
        e1.record(lat.stream)
        e1.synchronize()
        lat.sync()
        out[model + "_ms_per_step"] = e0.elapsed_time(e1) / steps
        lat.close()
    out["elastic_over_rigid"] = out["elastic_ms_per_step"] / out["bounceback_ms_per_step"]
    return out


def _timed_run(lat, steps):
    """Device ms of `steps` steps of one lattice: CUDA events on its stream at
    the two ends of the run only, and the mean step time from the same run."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    lat.sync()
    ms = e0.elapsed_time(e1)
    return ms, ms / steps


def storage_table(geo, params, steps, storages=("f64", "f32", "f16s", "bf16s"), tune=None):
    """Each storage run from rest on the same geometry for `steps` steps: MLUPS,
    step roofline fraction, and the rel-L2 error of the wall shear stress at the
    wall sites and of u against the FP64 path (first entry).  No error budget is
    chosen: the table is read at whatever budget a user has."""
    import lbm_inputs as I
    from paper_2108_08783_gb300 import Lattice
    peak, _ = measured_peaks()
    res, ref = {}, None
    for st in storages:
        lat = Lattice(geo.labels, geo.iolets, storage=st, tau=params["tau"])
        lat.set_wall("elastic", rho0=params["rho0"], F=params["F"], kappa=params["kappa"])
        if tune and st != "f64":
            lat.tune(**tune)
        ms, step_ms = _timed_run(lat, steps)
        ex = lat.export()
        s = ex["wall_sites"]
        wss = lat.wss(s, I.wall_normals(geo, ex["coords"][s]))
        u = lat.moments()[1]
        info = lat.info()
        n = lat.n
        lat.close()
        if ref is None:
            ref = (wss, u)
        res[st] = {"mlups": n * steps / ms / 1e3,
                   "roofline_frac": n * 2 * 19 * BYTES[st] / (step_ms * 1e-3) / 1e9 / peak,
                   "wss_rel_l2": float(np.linalg.norm(wss - ref[0]) / np.linalg.norm(ref[0])),
                   "u_rel_l2": float(np.linalg.norm(u - ref[1]) / np.linalg.norm(ref[1]))}
        res["irregular_tile_share"] = float(info[6]) / max(1, int(info[3]))
        res["sites"] = int(n)
    if "f32" in res:
        for st in storages:
            res[st]["speedup_vs_f32"] = res[st]["mlups"] / res["f32"]["mlups"]
    return res


def precision_study(args, geo, params, steps):
    """Every storage on the main workload (see storage_table)."""
    res = storage_table(geo, params, steps)
    return {"steps": steps, "reference": "f64 storage (matches the FP64 oracle to 1e-10)", **res}


def tree_workload():
    import lbm_inputs as I
    geo = I.murray_tree(seed=0, depth=6, root_radius=48.0)
    geo.iolets[0].u_mean = 0.03
    geo.iolets[0].u_amp = 0.02
    geo.iolets[0].period = 4000.0
    params = dict(tau=0.6, F=0.85, kappa=0.75 * 48.0 / 0.5, rho0=1.0)
    return geo, params


def tree_study(args, steps):
    """The depth-6 tree in FP64 (reference), FP32, FP16S and BF16S storage."""
    geo, params = tree_workload()
    res = storage_table(geo, params, steps)
    return {"workload": "seeded Murray tree depth 6, root R=48, tau=0.6, Eh/r0=0.5", "steps": steps,
            "reference": "f64 storage", **res}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    """Largest value over the ranks (timing only; the data path has no collective)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


ENSEMBLE_STEPS = 2000  # timed steps of the ensemble workload (at most)


def ensemble_members(seed=0, count=256):
    """The 256-tube ensemble family: radius U(6,24), length U(64,512), Eh/r0 log-U(0.05,5),
    inlet period U(1000,5000), tau U(0.55,1.0); F = 0.85, parabolic pulsatile
    inlet of mean 0.01 + 0.005 sin(2 pi n / T).

    Some soft, low-tau members of this family are unstable under the elastic
    wall: member 97 (tau 0.56, R 23.5) diverges after ~3,750 steps, in the
    FP64 oracle as on the GPU; at twice this inflow member 252 (tau 0.554,
    R 23.9) diverges after ~2,700 steps.  ENSEMBLE_STEPS keeps the whole
    ensemble run (autotuning included) below that."""
    import lbm_inputs as I
    out = []
    for prm in I.tube_ensemble(seed=seed, count=count):
        geo = I.tube(prm["radius"], prm["length"], u_mean=0.01, u_amp=0.005, period=prm["period"])
        out.append((geo, prm["tau"], prm["kappa"]))
    return out


def _ensemble_lattices(members, storage):
    from paper_2108_08783_gb300 import Lattice
    lats = []
    for geo, tau, kappa in members:
        lat = Lattice(geo.labels, geo.iolets, storage=storage, tau=tau)
        lat.set_wall("elastic", rho0=1.0, F=0.85, kappa=kappa)
        lats.append(lat)
    return lats


def _timed(fn, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def ensemble_error_table(members, steps=1000, every=8):
    """WSS and u error of each storage against the FP64 path on every `every`-th
    member of the ensemble, batched, `steps` steps from rest."""
    import lbm_inputs as I
    from paper_2108_08783_gb300 import Ensemble
    sub = members[::every]
    res, ref = {}, None
    for st in ("f64", "f32", "f16s", "bf16s"):
        lats = _ensemble_lattices(sub, st)
        ens = Ensemble(lats)
        ens.step(steps)
        ens.sync()
        wss, u = [], []
        for (geo, _, _), lat in zip(sub, lats):
            ex = lat.export()
            s = ex["wall_sites"]
            wss.append(lat.wss(s, I.wall_normals(geo, ex["coords"][s])))
            u.append(lat.moments()[1].ravel())
        ens.close()
        for lat in lats:
            lat.close()
        wss, u = np.concatenate(wss), np.concatenate(u)
        if ref is None:
            ref = (wss, u)
        res[st] = {"wss_rel_l2": float(np.linalg.norm(wss - ref[0]) / np.linalg.norm(ref[0])),
                   "u_rel_l2": float(np.linalg.norm(u - ref[1]) / np.linalg.norm(ref[1]))}
    return {"members": len(sub), "steps": steps, "reference": "f64 storage", **res}


def ensemble_study(args, steps, warmup):
    """Batched ensemble (256 uneven tubes): one launch per step kernel for all
    members, autotuned schedule; FP16S and FP32 storage batched, FP32 stepped one
    lattice at a time, and the storages' errors on a subset."""
    from paper_2108_08783_gb300 import Ensemble
    from paper_2108_08783_gb300._capi import LBM_EUNSTABLE, LbmError
    members = ensemble_members()
    out = {}
    peak, _ = measured_peaks()
    for storage in ("f16s", "f32"):
        lats = _ensemble_lattices(members, storage)
        n = sum(l.n for l in lats)
        ens = Ensemble(lats)
        # one timed trial per candidate and at most two sweeps: 28 candidates of
        # 2 x 20 steps each, at most 2,240 steps; then every member starts again
        # from rest, so the timed run is the same 2,000-odd steps from rest
        # whatever the search took (the family's least stable member diverges
        # after ~3,750 steps)
        best, trials = ens.autotune(trial_steps=20, trials=1, sweeps=2)
        trial_unstable = 0
        for l in lats:
            l.init_fields()
            try:
                l.sync()  # reads (and clears) a density flag raised during the search
            except LbmError as err:
                if err.status != LBM_EUNSTABLE:
                    raise
                trial_unstable += 1
        ens.step(warmup)
        ms = _timed(lambda: ens.step(steps), ens.stream)
        ens.sync()
        out[storage] = {"batched_mlups": n * steps / ms / 1e3, "autotuned": best,
                        "autotune_trials": len(trials),
                        "members_unstable_during_autotune": trial_unstable,
                        "ms_per_step": ms / steps,
                        "roofline_frac": n * 2 * 19 * BYTES[storage] / (ms / steps * 1e-3) / 1e9
                        / peak}
        ens.close()
        if storage == "f32":
            k = max(4, steps // 50)
            ms1 = _timed(lambda: [l.step(1) for _ in range(k) for l in lats], lats[0].stream)
            out["f32"]["one_at_a_time_mlups"] = n * k / ms1 / 1e3
        for l in lats:
            l.close()
    out["sites"] = n
    out["members"] = len(members)
    out["steps"] = steps
    out["errors"] = ensemble_error_table(members)
    return out


def run_ensemble(args):
    """The ensemble as the main line (FP16S batched)."""
    k_steps = min(max(args.steps, 1), ENSEMBLE_STEPS)
    out = ensemble_study(args, k_steps, args.warmup)
    line = {
        "metric": METRIC, "value": out["f16s"]["batched_mlups"], "unit": "MLUPS", "n_gpus": 1,
        "steps": k_steps, "warmup": args.warmup,
        "ms_per_step": out["f16s"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ensemble of 256 seeded elastic tubes (%d sites), FP16S storage"
                   % out["sites"], "sites": out["sites"]},
        "ensemble": out,
    }
    print(json.dumps(line), flush=True)


def run_config(args, name, n, ws):
    """The `config` object of both arms (same keys and values for one workload)."""
    return {"workload": name, "sites": n, "storage": args.storage, "wall": "elastic GZS",
            "l2": "populations (%.0f MB) exceed L2; no flush" % (19 * BYTES[args.storage] * n / 1e6),
            "parallelism": "replicas x%d" % ws}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    geo, params, name = workload(args)
    from oracle import Oracle
    from oracle.oracle import default_threads
    threads = default_threads()
    orc = Oracle(geo.labels, geo.iolets, tau=params["tau"], wall_model=1, F=params["F"],
                 kappa=params["kappa"], rho0=params["rho0"], threads=threads)
    # each step of this arm is one oracle step over the whole lattice; the run
    # is bounded to ~2 minutes of host time (steps beyond that are not run,
    # and the line says how many were)
    orc.run(min(args.warmup, 3))
    budget = 120.0
    t0 = time.perf_counter()
    done = 0
    while done < args.steps and (done == 0 or time.perf_counter() - t0 < budget):
        orc.run(1)
        done += 1
    dt = time.perf_counter() - t0
    mlups = orc.n * done / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / done * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": run_config(args, name, int(orc.n), ws),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": "%d of %d full oracle steps of the workload (%.1f s budget)"
                         % (done, args.steps, budget)},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    ws, rank, local = dist_init()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2108_08783_gb300 import Lattice
    import lbm_inputs as I

    geo, params, name = workload(args)
    lat = Lattice(geo.labels, geo.iolets, storage=args.storage, tau=params["tau"], device=local)
    lat.set_wall("elastic", rho0=params["rho0"], F=params["F"], kappa=params["kappa"])
    info = lat.info()
    n = lat.n
    stream = lat.stream
    # ---------------------------------------------------------------- device timing
    # warm-up: at least W steps, and two blocks of the library's captured step
    # graph (lbm_step replays 20-step graphs), so that the graph is captured
    # before the timed region and the timed region starts on an even step
    warm = max(args.warmup, 40)
    warm += warm & 1
    lat.step(warm)
    lat.sync()
    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    # The timed region carries events at its two ends only: per-step events
    # (lbm_profile) cost a few per cent, so they are taken in a short run after it.
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if rank == 0 else None
    ms_max = max_over_ranks(ws, ms)
    value = ws * n * args.steps / (ms_max * 1e-3) / 1e6
    # Per-step detail (fork-to-join and bulk-kernel windows, launch counts).
    pk = min(args.steps, 200)
    lat.profile(True)
    lat.step(pk)
    (step_ms_sum, bulk_ms_sum), (n_bulk_l, n_bnd_l) = lat.profile_read()
    lat.profile(False)
    lat.sync()
    launches_per_step = (n_bulk_l + n_bnd_l) / pk
    # the timed region's graph bookkeeping: one k_advance per replayed block, and
    # one k_set_step when the warm-up ended on direct steps (the counter is stale)
    graph_launches = 0
    if args.steps >= GRAPH_STEPS:
        graph_launches = args.steps // GRAPH_STEPS + (1 if warm % GRAPH_STEPS else 0)
    # ---------------------------------------------------------------- roofline
    peak, peak_kind = measured_peaks()
    s = BYTES[args.storage]
    # The step's two kernels (k_boundary on a side stream beside k_bulk) run
    # concurrently, so the unit is the step: every site read and written once
    # (19 populations each way).  Its duration is the timed region's mean step,
    # launch gaps included.
    bulk_sites = int(info[11])
    step_ms = ms_max / args.steps
    algo = n * 2 * 19 * s
    achieved = algo / (step_ms * 1e-3) / 1e9
    traffic = kernel_traffic(args.storage, args.config)
    roof = {"bound": "hbm", "kernel": "step: k_bulk + k_boundary (concurrent)", "achieved": achieved,
            "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "traffic_kind": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one step's "
                             "launches; per-launch counters leave out write-back of lines "
                             "still dirty in L2 when a launch ends"),
            "algorithmic_bytes_per_launch": algo, "launch_ms": step_ms,
            "event_step_ms": step_ms_sum / max(1, n_bulk_l),
            "k_bulk_window_ms": bulk_ms_sum / max(1, n_bulk_l), "bulk_sites": bulk_sites,
            "bulk_tiles": int(info[4]), "boundary_tiles": int(info[5] + info[6])}
    # ---------------------------------------------------------------- end to end
    e2e = None
    if not args.no_e2e:
        rho_g, u_g = I.random_fields(1, geo.shape, drho=1e-3, umax=0.02)
        c = lat.coords()
        rho_h = torch.from_numpy(I.gather(rho_g, c)).pin_memory()
        u_h = torch.from_numpy(I.gather(u_g, c)).pin_memory()
        rho_o = torch.empty(n, dtype=torch.float64).pin_memory()
        u_o = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        k = args.e2e_steps
        # every step's mass and iolet fluxes (lbm_step_diag: reduced by the step
        # kernels themselves), copied into a page-locked ring row by row
        ring = torch.empty((k, 1 + len(geo.iolets)), dtype=torch.float64).pin_memory()
        row = ring.stride(0) * ring.element_size()
        import ctypes
        barrier(ws)
        t0 = time.perf_counter()
        lat.init_fields(rho_h.numpy(), u_h.numpy())
        for i in range(k):
            lat._check(lat._lib.lbm_step_diag(lat.h, 1, ctypes.c_void_p(ring.data_ptr() + i * row)))
        lat._check(lat._lib.lbm_moments(lat.h, _addr(rho_o), _addr(u_o), 0))
        dt = time.perf_counter() - t0
        dt = max_over_ranks(ws, dt)
        diag = ring.numpy()
        if not np.isfinite(diag).all():
            raise SystemExit("e2e: non-finite diagnostics")
        e2e = {"value": ws * n * k / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": (rho_h.numel() + u_h.numel()) * 8 / k,
               "d2h_bytes_per_step": ring.shape[1] * 8 + (rho_o.numel() + u_o.numel()) * 8 / k,
               "steps": k,
               "per_step_result": "mass and iolet fluxes of every step (lbm_step_diag), FP64",
               "mass_first_last": [float(diag[0, 0]), float(diag[-1, 0])]}
    # ---------------------------------------------------------------- mixed precision
    prec = None
    if rank == 0 and not args.no_precision:
        prec = precision_study(args, geo, params, args.precision_steps)
    walls = wall_cost(args, geo, params) if rank == 0 and not args.no_precision else None
    tree = None
    if rank == 0 and not args.no_tree and args.config != "tree":
        tree = tree_study(args, max(args.steps, args.section_steps))
    ens = None
    if rank == 0 and not args.no_ensemble:
        ens = ensemble_study(args, min(max(args.steps, args.section_steps), ENSEMBLE_STEPS),
                             args.warmup)
    # ---------------------------------------------------------------- CPU baseline
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        mlups, threads, steps, dt = cpu_oracle(geo, params, seconds=args.cpu_seconds)
        m1, _, steps1, dt1 = cpu_oracle(geo, params, seconds=3.0, max_steps=50, threads=1)
        c1_s, c1_n = cpu_short_tube_full_run()
        cpu = {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "%d FP64 oracle steps of the same workload (%.1f s)" % (steps, dt),
               "single_thread_mlups": m1,
               "single_thread_sample": "%d steps (%.1f s)" % (steps1, dt1),
               "cpu_model": cpu_model(),
               "short_tube_full_run_s": c1_s,
               "short_tube": "R=8 L=64 tube (%d sites), 2000 steps from rest, all cores" % c1_n}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "warmup_steps_run": warm,
            "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.storage], "data": "synthetic",
            "config": run_config(args, name, n, ws),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "mixed_precision": prec,
            "wall_cost": walls, "tree": tree, "ensemble": ens,
            "gpu_launches": int(round(launches_per_step * args.steps)) + graph_launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _addr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=list(BYTES))
    ap.add_argument("--config", default="tube40", choices=["tube40", "tree", "tube8", "ensemble"])
    ap.add_argument("--e2e-steps", type=int, default=4000,
                    help="steps of the end-to-end run (the workload's usual length)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--precision-steps", type=int, default=4000)
    ap.add_argument("--section-steps", type=int, default=400,
                    help="timed steps (at least) of the tree and ensemble sections")
    ap.add_argument("--no-tree", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "ensemble":
        run_ensemble(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
