"""Learned warm start of elastic tubes: data, training and evaluation.

A family of straight elastic tubes (radius, length, wall stiffness Eh/r0,
steady inflow and relaxation time drawn per tube) is solved to steady state
by the method itself (batched lattices, ``Ensemble``); the network
(``MLP``, 4 x 256, bfloat16 with FP32 accumulation) learns
(tube parameters, axial and radial position) -> (rho, u_r, u_z) from those
converged fields with the library's own forward/backward/Adam kernels; a run
then starts from the network's proposal (``Lattice.warm_start``) instead of
from rest.  The zero-velocity start stays the fallback, and the network's
error is measured against the method's own converged solution.

Convergence: the relative change of u per step, measured over a window of
``window`` steps, ||u(t) - u(t - window)|| / (window ||u(t)||), falls below
``tol`` (1e-6).  Device tensors and norms are torch plumbing; every step of
the method and of the network runs in the library's kernels.
"""
import math

import numpy as np

import lbm_inputs as I

#: run-level feature normalisation: (R / 24, L / 512, log10(Eh/r0), u_in / 0.04, 2 (tau - 0.5))
N_GLOBAL = 5
F_WALL = 0.85


def family(seed, count, radius=(6.0, 24.0), length=(64, 512), stiffness=(0.05, 5.0),
           u_in=(0.01, 0.04), tau=(0.55, 1.0)):
    """Seeded tube parameters: the ensemble family (radius, length, Eh/r0, tau)
    with a steady parabolic inflow of mean velocity u_in."""
    base = I.tube_ensemble(seed=seed, count=count, radius=radius, length=length,
                           stiffness=stiffness, tau=tau)
    rng = np.random.default_rng(seed + 7919)
    amp = rng.uniform(*u_in, count)
    for p, a in zip(base, amp):
        p["u_in"] = float(a)
        p.pop("period", None)
    return base


def features(p):
    return [p["radius"] / 24.0, p["length"] / 512.0, math.log10(p["eh_r0"]), p["u_in"] / 0.04,
            2.0 * (p["tau"] - 0.5)]


def scales(p):
    """(rho_scale, u_scale): the inflow velocity, and the density drop of a
    rigid Poiseuille tube of the same size, 3 * 8 nu L u / R^2."""
    nu = (p["tau"] - 0.5) / 3.0
    return 24.0 * nu * p["length"] * p["u_in"] / p["radius"] ** 2, p["u_in"]


def build(p, storage="f32"):
    """(Geometry, Lattice, frame) of one tube, at rest."""
    from . import Lattice, warm_frame
    geo = I.tube(p["radius"], p["length"], u_mean=p["u_in"])
    lat = Lattice(geo.labels, geo.iolets, storage=storage, tau=p["tau"])
    lat.set_wall("elastic", rho0=1.0, F=F_WALL, kappa=p["kappa"])
    c = geo.meta["centre"]
    rs, us = scales(p)
    frame = warm_frame((c[0], c[1], 0.0), (0.0, 0.0, 1.0), 0.5, p["length"], p["radius"],
                       features(p), rs, us)
    return geo, lat, frame


class Monitor:
    """Relative change of u per step over a window, per lattice."""

    def __init__(self, lats):
        import torch
        self.lats = lats
        self.rho = [torch.empty(l.n, dtype=torch.float64, device=l.device) for l in lats]
        self.u = [torch.empty((l.n, 3), dtype=torch.float64, device=l.device) for l in lats]
        self.prev = None

    def sample(self):
        for lat, r, u in zip(self.lats, self.rho, self.u):
            lat.moments_into(r, u)
        cur = [u.clone() for u in self.u]
        out = None
        if self.prev is not None:
            out = np.array([float((c - p).norm() / c.norm().clamp_min(1e-300))
                            for c, p in zip(cur, self.prev)])
        self.prev = cur
        return out


def converge(lats, ens, tol=1e-6, window=100, max_steps=40000):
    """Advance the ensemble until every member's change per step is below tol
    (or max_steps); returns the step at which each member first met it
    (max_steps + window if never)."""
    mon = Monitor(lats)
    ens.sync()
    mon.sample()
    done = np.full(len(lats), -1, np.int64)
    steps = 0
    while steps < max_steps and (done < 0).any():
        ens.step(window)
        steps += window
        ens.sync()
        d = mon.sample() / window
        hit = (done < 0) & (d < tol)
        done[hit] = steps
    done[done < 0] = max_steps + window
    return done


def solve(params, storage="f32", tol=1e-6, window=100, max_steps=40000, start=None):
    """Build and converge a batch of tubes; returns (lattices, frames, steps).
    ``start(i, lat, frame)`` initialises member i (default: rest)."""
    from . import Ensemble
    geos, lats, frames = [], [], []
    for i, p in enumerate(params):
        g, lat, fr = build(p, storage)
        if start is not None:
            start(i, lat, fr)
        geos.append(g)
        lats.append(lat)
        frames.append(fr)
    ens = Ensemble(lats)
    steps = converge(lats, ens, tol, window, max_steps)
    ens.sync()
    del ens
    return lats, frames, steps


def dataset(params, samples_per_tube=1024, seed=0, batch=256, **kw):
    """Training pairs (x [m][7], t [m][3]) from converged tubes, sampled
    uniformly over each tube's sites; also returns the steps each needed."""
    import torch
    xs, ts, all_steps = [], [], []
    gen = torch.Generator(device="cpu").manual_seed(seed)
    for b in range(0, len(params), batch):
        lats, frames, steps = solve(params[b:b + batch], **kw)
        all_steps.append(steps)
        for lat, fr in zip(lats, frames):
            x, t = lat.warm_features(fr)
            idx = torch.randint(0, lat.n, (samples_per_tube,), generator=gen).to(x.device)
            xs.append(x[idx])
            ts.append(t[idx])
        for lat in lats:
            lat.close()
    return torch.cat(xs), torch.cat(ts), np.concatenate(all_steps)


def train(net, x, t, iters=3000, batch=4096, lr=2e-3, lr_end=1e-4, seed=0, log_every=0):
    """Adam over random minibatches with a cosine-decayed step size; returns
    the loss history [(iteration, loss)] sampled every ``log_every``."""
    import torch
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    m = x.shape[0]
    for it in range(iters):
        idx = torch.randint(0, m, (min(batch, m),), generator=gen).to(x.device)
        a = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * it / max(1, iters - 1)))
        want = log_every and (it % log_every == 0 or it == iters - 1)
        loss = net.train_step(x[idx], t[idx], lr=a, want_loss=bool(want))
        if want:
            hist.append((it, loss))
    net.sync()
    return hist


def evaluate(net, params, storage="f32", tol=1e-6, window=100, max_steps=40000):
    """Held-out tubes from rest and from the network's start: steps to
    converge, and the relative L2 error of each start's u against the
    converged solution of the zero start."""
    import torch
    lats0, frames0, steps0 = solve(params, storage, tol, window, max_steps)
    conv = []
    err0 = []
    for lat in lats0:
        rho, u = lat.moments()
        conv.append((rho, u))
        err0.append(1.0)  # ||0 - u|| / ||u||
    init_err = []

    def start(i, lat, fr):
        lat.warm_start(net, fr)
        _, u = lat.moments()
        uc = conv[i][1]
        init_err.append(float(np.linalg.norm(u - uc) / np.linalg.norm(uc)))

    lats1, _, steps1 = solve(params, storage, tol, window, max_steps, start=start)
    final_err = []
    for l0, l1 in zip(lats0, lats1):
        u1 = l1.moments()[1]
        u0 = l0.moments()[1]
        final_err.append(float(np.linalg.norm(u1 - u0) / np.linalg.norm(u0)))
    for lat in lats0 + lats1:
        lat.close()
    torch.cuda.synchronize()
    return dict(steps_zero=steps0, steps_warm=steps1, init_err_warm=np.array(init_err),
                init_err_zero=np.array(err0), final_err=np.array(final_err))


def study(n_train=2000, n_eval=200, seed=0, storage="f32", samples_per_tube=1024, iters=4000,
          batch=4096, max_steps=40000, window=100, tol=1e-6, family_kw=None, log=print):
    """Train on n_train tubes of the family and evaluate on n_eval held-out
    ones; returns a summary dict."""
    import time

    import torch
    from . import MLP
    fk = family_kw or {}
    train_p = family(seed, n_train, **fk)
    eval_p = family(seed + 100003, n_eval, **fk)
    t0 = time.time()
    x, t, steps_train = dataset(train_p, samples_per_tube, seed, storage=storage, tol=tol,
                                window=window, max_steps=max_steps)
    t1 = time.time()
    log("solved %d training tubes in %.1f s (steps to converge: median %d, max %d); %d samples"
        % (n_train, t1 - t0, np.median(steps_train), steps_train.max(), x.shape[0]))
    net = MLP(N_GLOBAL + 2, 256, 4, 3, max_batch=batch)
    net.set_params(I.mlp_init(seed, N_GLOBAL + 2, 256, 4, 3))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(net.stream)
    hist = train(net, x, t, iters=iters, batch=batch, seed=seed, log_every=max(1, iters // 10))
    e1.record(net.stream)
    e1.synchronize()
    train_ms = e0.elapsed_time(e1)
    log("trained %d Adam steps of %d samples in %.1f ms; loss %s" % (
        iters, batch, train_ms, " ".join("%.2e" % l for _, l in hist)))
    t2 = time.time()
    res = evaluate(net, eval_p, storage, tol, window, max_steps)
    t3 = time.time()
    sz, sw = res["steps_zero"], res["steps_warm"]
    out = dict(n_train=n_train, n_eval=n_eval, storage=storage, tol=tol, window=window,
               max_steps=max_steps, samples=int(x.shape[0]), iters=iters, batch=batch,
               train_ms=train_ms, loss_first=hist[0][1], loss_last=hist[-1][1],
               steps_zero_mean=float(sz.mean()), steps_warm_mean=float(sw.mean()),
               steps_zero_median=float(np.median(sz)), steps_warm_median=float(np.median(sw)),
               step_ratio_mean=float(np.mean(sw / sz)),
               unconverged_zero=int((sz > max_steps).sum()),
               unconverged_warm=int((sw > max_steps).sum()),
               init_err_warm_median=float(np.median(res["init_err_warm"])),
               init_err_warm_mean=float(np.mean(res["init_err_warm"])),
               final_err_max=float(res["final_err"].max()),
               solve_s=t1 - t0, eval_s=t3 - t2)
    log("held-out: steps zero mean %.0f median %.0f | warm mean %.0f median %.0f | "
        "mean ratio %.3f | warm-start error vs converged u: median %.3f | final agreement %.1e"
        % (out["steps_zero_mean"], out["steps_zero_median"], out["steps_warm_mean"],
           out["steps_warm_median"], out["step_ratio_mean"], out["init_err_warm_median"],
           out["final_err_max"]))
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start study on the tube family")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--max-steps", type=int, default=40000)
    ap.add_argument("--samples", type=int, default=1024)
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--small", action="store_true", help="radius 4-8, length 24-64, tau 0.7-1")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    fk = dict(radius=(4.0, 8.0), length=(24, 64), tau=(0.7, 1.0)) if a.small else None
    r = study(a.train, a.eval, storage=a.storage, samples_per_tube=a.samples, iters=a.iters,
              max_steps=a.max_steps, family_kw=fk)
    print(json.dumps(r))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
