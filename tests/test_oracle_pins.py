"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests touches the GPU path.  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand) fails at least one of them:

* velocity set / weights: isotropy identities up to fourth order;
* equilibrium: moment identities (and the reading of Eq. feq with the 1/2 factors);
* collision: exact mass and momentum conservation, fixed point at equilibrium;
* streaming + bounce-back: rest state invariant, exact mass conservation in a
  closed box, second-order Poiseuille convergence in a duct against the
  textbook series solution;
* elastic GZS wall: F = 0, kappa = 0 puts a no-slip wall on the wall nodes
  (Poiseuille again, wider duct); F = 1 preserves a uniform plug flow exactly;
  kappa -> infinity reproduces F = 1; rho0 above every density reproduces
  kappa = 0 bit for bit (the clamp);
* velocity inlet: rigid Womersley flow at alpha = 4 (the M = 1, c -> infinity
  limit of the Sec. 2.2 solution) within 5 %;
* complex Bessel series against scipy;
* the tube-law expansion and the wall velocity exported per wall site against
  the moments the step read (bit for bit for the expansion);
* the F ratio against the radial mode of the Womersley momentum balance
  integrated numerically;
* unit conversions against Table A1 and Sec. 2.4.
"""
import os

import numpy as np
import pytest

import lbm_inputs as I
from oracle import Oracle, bessel_j01, collide, equilibrium, velocity_set, womersley_shape
from oracle import analytic as A

from analytic_ref import duct_velocity, rel_l2, womersley_rigid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------- velocity set

def test_velocity_set_isotropy():
    c, w, opp = velocity_set()
    c = c.astype(np.float64)
    assert c.shape == (19, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w @ c, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-16)
    # 1 rest + 6 axis + 12 face diagonals, each listed once, opposite pairs
    assert sorted(map(tuple, c.astype(int).tolist())) == sorted(
        {(a, b, e) for a in (-1, 0, 1) for b in (-1, 0, 1) for e in (-1, 0, 1)
         if abs(a) + abs(b) + abs(e) <= 2})
    for i in range(19):
        assert opp[opp[i]] == i
        np.testing.assert_array_equal(c[opp[i]], -c[i])


# ----------------------------------------------------------- equilibrium

@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.9, 1.1)
    u = rng.uniform(-0.1, 0.1, 3)
    c, w, _ = velocity_set()
    c = c.astype(np.float64)
    feq = equilibrium(rho, u)
    assert abs(feq.sum() - rho) < 1e-15
    np.testing.assert_allclose(feq @ c, rho * u, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", feq, c, c),
                               rho * np.eye(3) / 3.0 + rho * np.outer(u, u), atol=2e-16)


def test_printed_equilibrium_without_halves_breaks_momentum_flux():
    """The reading of Eq. (feq): as printed (no 1/2 factors) the second moment
    would be rho c_s^2 I + 2 rho u u, not the Navier-Stokes rho c_s^2 I + rho u u."""
    c, w, _ = velocity_set()
    c = c.astype(np.float64)
    rho, u = 1.02, np.array([0.03, -0.02, 0.05])
    cu = c @ u
    printed = w * rho * (1 + 3 * cu + 9 * cu ** 2 - 3 * u @ u)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", printed, c, c),
                               rho * np.eye(3) / 3 + 2 * rho * np.outer(u, u), atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", equilibrium(rho, u), c, c),
                               rho * np.eye(3) / 3 + rho * np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("tau", [0.51, 0.8, 1.0, 1.7])
def test_collision_conserves_and_relaxes(tau):
    rng = np.random.default_rng(7)
    c, w, _ = velocity_set()
    c = c.astype(np.float64)
    f = w * (1 + rng.uniform(-0.2, 0.2, 19))
    out = collide(f, tau)
    assert abs(out.sum() - f.sum()) < 1e-15
    np.testing.assert_allclose(out @ c, f @ c, atol=1e-16)
    rho = f.sum()
    u = f @ c / rho
    feq = equilibrium(rho, u)
    # Eq. (LBE_SRT): the non-equilibrium part shrinks by exactly (1 - 1/tau)
    np.testing.assert_allclose(out - feq, (1 - 1 / tau) * (f - feq), atol=1e-16)
    np.testing.assert_allclose(collide(feq, tau), feq, atol=1e-16)


# ----------------------------------------------------------- lattice build

@pytest.mark.parametrize("seed", range(4))
def test_builder_brute_force(seed):
    g = I.random_labels(seed, (7, 6, 9), fill=0.6)
    o = Oracle(g.labels, g.iolets)
    ex = o.export()
    lab = g.labels
    fluid = np.argwhere(lab == 1)
    # canonical order: ascending (x*ny + y)*nz + z, which argwhere already gives
    np.testing.assert_array_equal(ex["coords"], fluid)
    idx = {tuple(p): k for k, p in enumerate(fluid.tolist())}
    c, _, _ = velocity_set()
    walls = []
    for s, p in enumerate(fluid):
        nwall = 0
        for i in range(1, 19):
            q = p + c[i]
            if np.any(q < 0) or np.any(q >= lab.shape) or lab[tuple(q)] == 0:
                want = -1
                nwall += 1
                walls.append((s, i))
            elif lab[tuple(q)] == 1:
                want = idx[tuple(q)]
            else:
                want = -2 - (int(lab[tuple(q)]) - 2)
            assert ex["nbr"][s, i - 1] == want
    np.testing.assert_array_equal(ex["wall_links"], np.array(walls, np.int64).reshape(-1, 2))
    np.testing.assert_array_equal(ex["wall_sites"], np.unique([s for s, _ in walls]))


def test_builder_rejects_unknown_iolet_label():
    g = I.tube(4, 8)
    with pytest.raises(ValueError):
        Oracle(g.labels, g.iolets[:1])


# ----------------------------------------------------------- invariants of the step

@pytest.mark.parametrize("wall_model", [0, 1])
def test_rest_state_is_invariant(wall_model):
    g = I.tube(6, 16, u_mean=0.0, rho_out=1.0)
    o = Oracle(g.labels, g.iolets, tau=0.7, wall_model=wall_model, F=0.85, kappa=12.0)
    f0 = o.populations()
    o.run(50)
    np.testing.assert_allclose(o.populations(), f0, rtol=0, atol=1e-15)


def test_closed_box_conserves_mass_exactly():
    g = I.closed_box(12, 10, 14)
    o = Oracle(g.labels, [], tau=0.6, wall_model=0)
    rho, u = I.random_fields(3, g.shape, drho=5e-3, umax=0.03)
    c = o.coords()
    o.init_equilibrium(I.gather(rho, c), I.gather(u, c))
    m0 = o.reduce()[0]
    o.run(3000)
    m1 = o.reduce()[0]
    # exact up to rounding: the collision's sum is off by about one ulp per
    # site and step (sum of f^eq is rho only to rounding), so the bound is
    # steps * 4 eps; a lost or duplicated population would show as ~1e-4
    assert abs(m1 - m0) / m0 < 3000 * 4 * np.finfo(float).eps
    # and the flow decays (walls take momentum out)
    assert np.abs(o.moments()[1]).max() < 0.03


def test_elastic_wall_does_not_conserve_mass_in_closed_box():
    """Reading R6: the wall velocity scales the full u_f, so the elastic wall
    exchanges mass; documented, not a defect of the oracle."""
    g = I.closed_box(10, 10, 10)
    o = Oracle(g.labels, [], tau=0.6, wall_model=1, F=0.85, kappa=5.0)
    rho, u = I.random_fields(4, g.shape, drho=5e-3, umax=0.03)
    c = o.coords()
    o.init_equilibrium(I.gather(rho, c), I.gather(u, c))
    m0 = o.reduce()[0]
    o.run(200)
    assert abs(o.reduce()[0] - m0) / m0 > 1e-9


# ----------------------------------------------------------- Poiseuille

def _duct_error(n, wall_model, tau=1.0):
    nu = A.viscosity(tau)
    L = 2 * n
    G0 = 0.01 * nu / (0.0737 * n * n)
    d = 1.5 * G0 * L
    g = I.duct(n, n, L, rho_in=1 + d, rho_out=1 - d)
    o = Oracle(g.labels, g.iolets, tau=tau, wall_model=wall_model, F=0.0, kappa=0.0)
    o.run(int(2.5 * n * n / nu))
    rho, u = o.moments()
    c = o.coords()
    zm = L // 2 + 1
    plane = lambda z: c[:, 2] == z
    G = -(rho[plane(zm + 1)].mean() - rho[plane(zm - 1)].mean()) / 2.0 / 3.0
    m = plane(zm)
    mu = rho[m].mean() * nu
    cx = (n + 1) / 2.0
    # half-way bounce-back puts the wall half a node out; the GZS wall at
    # Delta = 1 with zero wall velocity puts it on the wall nodes
    a = n / 2.0 if wall_model == 0 else (n + 1) / 2.0
    ua = duct_velocity(c[m, 0] - cx, c[m, 1] - cx, a, a, G, mu)
    return rel_l2(u[m, 2], ua)


@pytest.mark.parametrize("wall_model,tol", [(0, 2e-3), (1, 1.5e-2)])
def test_duct_poiseuille_second_order(wall_model, tol):
    e = [_duct_error(n, wall_model) for n in (5, 10, 20)]
    assert e[2] < tol
    order = np.log2(e[1] / e[2])
    assert 1.5 < order < 2.6, e


# ----------------------------------------------------------- elastic wall special cases

def _plug_run(F, kappa, rho0=1.0, steps=150):
    u0 = 0.02
    n, L = 6, 12
    cx = (n + 1) / 2.0
    inlet = I.Iolet(kind=0, centre=(cx, cx, 0.0), axis=(0.0, 0.0, 1.0), radius=10.0, profile=2,
                    u_mean=u0)
    g = I.duct(n, n, L, inlet=inlet, rho_out=1.0)
    o = Oracle(g.labels, g.iolets, tau=0.8, wall_model=1, F=F, kappa=kappa, rho0=rho0)
    u = np.zeros((o.n, 3))
    u[:, 2] = u0
    o.init_equilibrium(None, u)
    o.run(steps)
    return o


def test_f_one_preserves_plug_flow():
    """F = 1, kappa = 0 gives U_w = u_f: a uniform plug is an exact steady state."""
    o = _plug_run(F=1.0, kappa=0.0)
    rho, u = o.moments()
    np.testing.assert_allclose(rho, 1.0, atol=1e-13)
    np.testing.assert_allclose(u[:, 2], 0.02, atol=1e-13)
    np.testing.assert_allclose(u[:, :2], 0.0, atol=1e-13)
    # with F < 1 the wall slows the fluid next to it
    rho, u = _plug_run(F=0.85, kappa=0.0).moments()
    assert np.abs(u[:, 2] - 0.02).max() > 1e-4


def test_kappa_limits():
    """kappa -> infinity with p > P0 everywhere makes (F + dE)/(1 + dE) -> 1 (same as F = 1);
    rho0 above every density clamps dE to 0 (same as kappa = 0, bit for bit)."""
    base = dict(F=0.3)
    f_one = _plug_run(F=1.0, kappa=0.0).populations()
    big = _plug_run(kappa=1e13, rho0=0.5, **base).populations()
    assert np.abs(big - f_one).max() < 1e-11
    zero = _plug_run(kappa=0.0, **base).populations()
    clamped = _plug_run(kappa=50.0, rho0=2.0, **base).populations()
    np.testing.assert_array_equal(clamped, zero)
    loose = _plug_run(kappa=50.0, rho0=0.9, **base).populations()
    assert np.abs(loose - zero).max() > 1e-8


def test_wall_state_export():
    g = I.tube(6, 16, u_mean=0.02)
    o = Oracle(g.labels, g.iolets, tau=0.8, wall_model=1, F=0.85, kappa=12.0, rho0=0.999)
    o.run(40)
    dE, Uw = o.wall_state()
    assert dE.shape == (o.n_wall,) and np.all(dE >= 0) and dE.max() > 0
    # U_w is parallel to the fluid velocity and no larger than it (0 <= F <= 1)
    assert np.all(np.isfinite(Uw))


def test_wall_state_is_the_tube_law_of_the_local_pressure():
    """Sec. 2.4 tube law dE = kappa (p - P0), clamped at 0, with the lattice
    pressure p - P0 = c_s^2 (rho - rho0) (Eq. Pressure), and Sec. 2.3's
    U_w = (F + dr - dx)/dr u_f with dr = dx + dE.

    The moments are read from the populations held before the last step
    (summed here in the oracle's order, so the expansion is compared bit for
    bit), c_s^2 comes from the velocity set's own second moment, kappa is
    large enough that dE is O(0.1 - 1) (a dropped or doubled c_s^2 changes
    it by a factor 3), rho0 sits inside the range of the wall densities so
    that the clamp acts on some sites and not on others, and F and kappa vary
    per wall site (a shuffled site index fails)."""
    c, w, _ = velocity_set()
    cs2 = float(np.sum(w * c[:, 0].astype(np.float64) ** 2))
    inv_cs2 = float(round(1.0 / cs2))
    assert abs(1.0 / cs2 - inv_cs2) < 1e-14 and inv_cs2 == 3.0
    g = I.tube(6, 24, u_mean=0.02)
    o = Oracle(g.labels, g.iolets, tau=0.8, wall_model=1)
    ws = o.export()["wall_sites"]
    coords = o.coords()
    rng = np.random.default_rng(4)
    F = rng.uniform(0.0, 1.0, ws.size)
    kappa = rng.uniform(30.0, 300.0, ws.size)
    rho_g, u_g = I.random_fields(3, g.shape, drho=2e-3, umax=0.02)
    o.init_equilibrium(I.gather(rho_g, coords), I.gather(u_g, coords))
    o.run(5)
    f = o.populations()[ws]
    rho = np.zeros(ws.size)
    j = np.zeros((ws.size, 3))
    for i in range(19):  # the oracle's summation order
        rho = rho + f[:, i]
        j = j + f[:, i:i + 1] * c[i].astype(np.float64)
    u = j / rho[:, None]
    rho0 = float(np.median(rho))
    o.configure(0.8, 1, rho0, F, kappa)
    o.run(1)
    dE, Uw = o.wall_state()
    want = kappa * np.maximum(0.0, (rho - rho0) / inv_cs2)
    np.testing.assert_array_equal(dE, want)
    assert 0.1 < dE.max() < 3.0 and np.count_nonzero(dE == 0.0) > ws.size // 4
    ratio = (F + dE) / (1.0 + dE)
    np.testing.assert_allclose(Uw, ratio[:, None] * u, rtol=0, atol=1e-15)
    # the expansion moves U_w from F u_f (dE = 0) toward u_f
    big = dE > 0.1
    assert np.all(np.abs(Uw[big, 2]) > np.abs(F[big] * u[big, 2]) - 1e-18)


# ----------------------------------------------------------- Womersley

def test_bessel_series_matches_scipy():
    from scipy.special import jv
    rng = np.random.default_rng(0)
    for _ in range(60):
        z = complex(*rng.uniform(-9, 9, 2))
        j0, j1 = bessel_j01(z)
        assert abs(j0 - jv(0, z)) <= 1e-11 * max(1.0, abs(jv(0, z)))
        assert abs(j1 - jv(1, z)) <= 1e-11 * max(1.0, abs(jv(1, z)))


def test_womersley_shape_limits():
    xi = np.linspace(0, 1, 41)
    # alpha -> 0: Poiseuille 2 (1 - xi^2)
    s = np.array([womersley_shape(1e-3, x) for x in xi])
    np.testing.assert_allclose(s.real, 2 * (1 - xi ** 2), atol=1e-6)
    for alpha in (2.0, 4.0, 8.68):
        s = np.array([womersley_shape(alpha, x) for x in np.linspace(0, 1, 2001)])
        r = np.linspace(0, 1, 2001)
        mean = np.trapezoid(2 * s * r, r)  # unit mean over the disc
        assert abs(mean - 1) < 1e-5
        assert abs(s[-1]) < 1e-12  # no slip at r = R


def test_rigid_womersley_tube():
    """Velocity inlet carrying the alpha = 4 Womersley profile; mid-plane
    profiles at 5 phases of the third period agree within 5 % of the peak."""
    tau, R, L, alpha = 0.55, 10, 30, 4.0
    nu = A.viscosity(tau)
    T = 2 * np.pi / (alpha ** 2 * nu / R ** 2)
    g = I.tube(R, L, u_mean=0.01, u_amp=0.01, period=T, profile=1)
    o = Oracle(g.labels, g.iolets, tau=tau, wall_model=0)
    c = o.coords()
    m = c[:, 2] == L // 2
    cx = g.meta["centre"][0]
    xi = np.sqrt((c[m, 0] - cx) ** 2 + (c[m, 1] - cx) ** 2) / R
    o.run(int(2 * T))
    got, want, shifted = [], [], []
    for ph in range(5):
        o.run(int(np.ceil(2 * T + ph * T / 5)) - o.step)
        u = o.moments()[1][m, 2]
        th = 2 * np.pi * o.step / T
        got.append(u)
        want.append(womersley_rigid(xi, alpha, 0.01, 0.01, th))
        shifted.append(womersley_rigid(xi, alpha, 0.01, 0.01, th + np.pi / 2))
    peak = max(np.linalg.norm(w) for w in want)
    err = [np.linalg.norm(a - b) / peak for a, b in zip(got, want)]
    assert max(err) < 0.05, err
    # a quarter-period phase error would be caught
    assert max(np.linalg.norm(a - b) / peak for a, b in zip(got, shifted)) > 0.15


# ----------------------------------------------------------- elastic vs rigid trend

def test_elastic_vs_rigid_trend_short_tube():
    """Short tube (R = 8, L = 64, tau = 0.8, peak 0.05, kappa = 12, F = 0.85):
    the elastic wall moves fluid faster next to the wall and needs a smaller
    pressure drop than bounce-back (Sec. 2.4 comparison)."""
    g = I.tube(8, 64, u_mean=0.025)
    res = {}
    for wm in (0, 1):
        o = Oracle(g.labels, g.iolets, tau=0.8, wall_model=wm, F=0.85, kappa=12.0)
        o.run(2000)
        rho, u = o.moments()
        c = o.coords()
        m = c[:, 2] == 32
        r = np.hypot(c[m, 0] - 9.5, c[m, 1] - 9.5)
        near = r > 6.5
        res[wm] = (u[m, 2][near].mean(), rho[c[:, 2] == 8].mean() - rho[c[:, 2] == 56].mean())
    assert res[1][0] > res[0][0]
    assert res[1][1] < res[0][1]


# ----------------------------------------------------------- unit conversions

def _table_a1():
    rows = []
    for line in open(os.path.join(GOLDEN, "table_a1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, dx, dt, tau, steps, sites, cores = line.split()
        rows.append((name, float(dx), float(dt), float(tau), int(steps), int(sites), int(cores)))
    return rows


def test_table_a1_tau_from_units():
    nu = 0.004 / 1000.0  # Sec. 2.4 fluid
    for name, dx, dt, tau, *_ in _table_a1():
        got = A.tau_from_physical(nu, dx, dt)
        if name == "arteries_orig":
            # printed 0.527 does not follow from dx, dt (0.524); recorded as a paper inconsistency
            assert abs(got - 0.524) < 5e-4
            continue
        assert abs(got - tau) < 5e-4, (name, got, tau)


def test_sec24_cylinder_numbers():
    vals = {}
    for line in open(os.path.join(GOLDEN, "sec24_cylinder.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        vals[k] = float(v)
    omega = 2 * np.pi / vals["period"]
    alpha = A.womersley_number(vals["radius"], omega, vals["rho"], vals["mu"])
    assert abs(alpha - vals["womersley"]) < 1e-12
    h = vals["thickness_over_R"] * vals["radius"]
    k = A.tube_law_coefficient(vals["radius"], vals["young"], h, vals["poisson"])
    assert abs(k - 1.125e-6) < 1e-18
    # the same coefficient through the stiffness parameter Eh/r0 used by the workloads
    assert abs(A.kappa_lattice(vals["radius"], vals["young"] * h / vals["radius"]) - k) < 1e-18
    # the short tube: r0 = 8, Eh/r0 = 0.5 (lattice units) -> kappa = 12
    assert A.kappa_lattice(8.0, 0.5) == 12.0


def test_f_ratio_limits():
    for alpha in (1.0, 3.0, 8.0):
        assert abs(A.f_ratio(alpha, 1e-9, 0.7) - 1.0) < 1e-6  # F -> 1 as dr -> 0
        assert abs(A.f_ratio(alpha, 0.05, 0.0) - 1.0) < 1e-15  # M = 0


def _womersley_radial_mode(alpha, xi):
    """y(xi) / y(1) for the radial part of the oscillating Womersley velocity,
    integrated numerically from the momentum balance rather than taken from a
    Bessel function: with time dependence e^(i omega t) (Sec. 2.2), the
    homogeneous part of rho dw/dt = -dp/dz + mu (w'' + w'/r) is
    y'' + y'/xi = i alpha^2 y in xi = r/R (alpha^2 = R^2 omega rho / mu),
    regular at the axis (y(0) = 1, y'(0) = 0)."""
    from scipy.integrate import solve_ivp
    a2 = 1j * alpha * alpha
    x0 = 1e-4  # start off the axis on the regular series y = 1 + a2 x^2/4 + a2^2 x^4/64
    y0 = np.array([1 + a2 * x0 ** 2 / 4 + a2 ** 2 * x0 ** 4 / 64,
                   a2 * x0 / 2 + a2 ** 2 * x0 ** 3 / 16], complex)
    sol = solve_ivp(lambda x, y: [y[1], a2 * y[0] - y[1] / x], (x0, 1.0), y0, method="DOP853",
                    rtol=1e-12, atol=1e-15, dense_output=True)
    assert sol.success
    return sol.sol(xi)[0] / sol.sol(1.0)[0]


def test_f_ratio_matches_the_womersley_momentum_balance():
    """Sec. 2.3's F = w(R) / w(R - dr) with w proportional to 1 - M J0(Lambda r/R)/J0(Lambda),
    Lambda = i^(3/2) alpha, against the same ratio built from the radial mode
    integrated from the momentum balance (no Bessel function, no Lambda): a
    wrong phase of Lambda (i^(1/2) alpha gives the complex conjugate mode), a
    dropped (1 - dr/R) or a swapped numerator fails."""
    for alpha in (1.0, 3.0, 8.0):
        for d in (0.02, 0.1, 0.3):
            for M in (0.5, 0.9, 1.3 - 0.2j):
                want = (1.0 - M) / (1.0 - M * _womersley_radial_mode(alpha, 1.0 - d))
                got = A.f_ratio(alpha, d, M)
                assert abs(got - want) <= 1e-8 * abs(want), (alpha, d, M, got, want)
                # the conjugate mode (e^(-i omega t) convention) is distinguishable
                if M == 0.9 and alpha >= 3.0:
                    wrong = (1.0 - M) / (1.0 - M * np.conj(_womersley_radial_mode(alpha, 1.0 - d)))
                    assert abs(got - wrong) > 1e-3 * abs(want)


# ----------------------------------------------------------- wall shear stress

def test_wss_matches_viscous_stress_of_duct_flow():
    """The stress read from f^neq at a wall-adjacent node equals mu du/dn of
    the textbook duct solution there (pins the -(1 - 1/(2 tau)) factor, the
    second moment of f^neq and the tangential projection)."""
    tau, n = 1.0, 16
    nu = A.viscosity(tau)
    L = 2 * n
    G0 = 0.01 * nu / (0.0737 * n * n)
    d = 1.5 * G0 * L
    g = I.duct(n, n, L, rho_in=1 + d, rho_out=1 - d)
    o = Oracle(g.labels, g.iolets, tau=tau, wall_model=0)
    o.run(int(2.5 * n * n / nu))
    rho, u = o.moments()
    c = o.coords()
    zm = L // 2 + 1
    G = -(rho[c[:, 2] == zm + 1].mean() - rho[c[:, 2] == zm - 1].mean()) / 2.0 / 3.0
    mu = rho[c[:, 2] == zm].mean() * nu
    cx = (n + 1) / 2.0
    sel = np.where((c[:, 2] == zm) & (c[:, 1] == 1) & (np.abs(c[:, 0] - cx) < n / 4))[0]
    normals = np.tile([0.0, -1.0, 0.0], (sel.size, 1))
    wss = o.wss(sel, normals)
    h = 1e-4
    xs, ys = c[sel, 0] - cx, c[sel, 1] - cx
    dudy = (duct_velocity(xs, ys + h, n / 2, n / 2, G, mu)
            - duct_velocity(xs, ys - h, n / 2, n / 2, G, mu)) / (2 * h)
    np.testing.assert_allclose(wss, mu * np.abs(dudy), rtol=0.03)


def test_rigid_wall_shear_exceeds_elastic():
    """Sec. 3: the elastic wall lowers wall shear stress relative to bounce-back."""
    g = I.tube(8, 64, u_mean=0.025)
    out = {}
    for wm in (0, 1):
        o = Oracle(g.labels, g.iolets, tau=0.8, wall_model=wm, F=0.85, kappa=12.0)
        o.run(600)
        ex = o.export()
        s = ex["wall_sites"]
        out[wm] = o.wss(s, I.wall_normals(g, ex["coords"][s]))
    assert out[0].mean() > 2 * out[1].mean()
    assert np.mean(out[0] >= out[1]) > 0.9


def test_reduce_flux_balances_and_matches_the_duct_flow_rate():
    """Steady pressure-driven duct (bounce-back): the oracle's per-iolet flux
    (sum of rho u . axis over the sites touching the iolet) is the same at
    inlet and outlet (mass balance) and equals the node sum of rho times the
    rectangular-duct series velocity on the end planes."""
    n, tau = 10, 1.0
    nu = A.viscosity(tau)
    L = 2 * n
    G0 = 0.01 * nu / (0.0737 * n * n)
    d = 1.5 * G0 * L
    g = I.duct(n, n, L, rho_in=1 + d, rho_out=1 - d)
    o = Oracle(g.labels, g.iolets, tau=tau, wall_model=0, F=0.0, kappa=0.0)
    o.run(int(3.0 * n * n / nu))
    red = o.reduce()
    q_in, q_out = red[1], red[2]
    assert q_in > 0 and q_out > 0
    assert abs(q_in - q_out) < 1e-6 * q_in
    rho, u = o.moments()
    c = o.coords()
    zm = L // 2 + 1
    plane = lambda z: c[:, 2] == z
    G = -(rho[plane(zm + 1)].mean() - rho[plane(zm - 1)].mean()) / 2.0 / 3.0
    m = plane(zm)
    mu = rho[m].mean() * nu
    cx = (n + 1) / 2.0
    ua = duct_velocity(c[m, 0] - cx, c[m, 1] - cx, n / 2.0, n / 2.0, G, mu)
    q_series = float(np.sum(rho[m] * ua))
    assert abs(q_in - q_series) < 1e-2 * q_series
    # the site sum over the mid plane carries the same flux
    assert abs(float(np.sum(rho[m] * u[m, 2])) - q_in) < 1e-3 * q_in


def _steady_tube(rho_out, u0=0.01, R=6.0, L=24):
    g = I.tube(R, L, u_mean=u0, rho_out=rho_out)
    o = Oracle(g.labels, g.iolets, tau=0.8, wall_model=0, F=0.0, kappa=0.0)
    o.run(2500)
    rho, u = o.moments()
    return o, rho, u, o.coords()


def test_parabolic_inlet_carries_its_mean_velocity():
    """A steady parabolic velocity inlet of mean u (R9: 2(1 - r^2/R^2) scaled to
    unit mean over the disc) delivers a flux of about rho u per inlet-plane
    node once the tube is steady (the node sum of the profile differs from
    its disc mean by the discretisation only)."""
    u0 = 0.01
    o, rho, u, c = _steady_tube(1.0, u0)
    first = c[:, 2] == 1
    per_node = o.reduce()[1] / first.sum()
    assert abs(per_node / (rho[first].mean() * u0) - 1.0) < 0.02


def test_density_outlet_sets_the_pressure_level():
    """Raising the outlet density by delta raises the density everywhere in a
    steady, incompressible-regime tube by delta (the flow, set by the inlet,
    does not change): the outlet fixes the pressure level."""
    delta = 1e-3
    _, r0, u0, c = _steady_tube(1.0)
    _, r1, u1, _ = _steady_tube(1.0 + delta)
    shift = r1 - r0
    assert abs(shift.mean() / delta - 1.0) < 0.05
    assert np.std(shift) < 0.05 * delta
    assert np.max(np.abs(u1 - u0)) < 1e-3 * np.max(np.abs(u0))


# ----------------------------------------------------------- wall times (Sec. 2.4)

def _walltimes():
    rows = []
    for line in open(os.path.join(GOLDEN, "walltimes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        r, el, ri, sites, cores = line.split()
        rows.append((int(r), float(el), float(ri), int(sites), int(cores)))
    return rows


def test_walltime_table_is_consistent_with_table_a1_and_the_papers_claim():
    """Table WallTimes (Sec. 2.4, wall time of 1000 iterations, elastic wall vs
    rigid bounce-back on the same domain and cores) against Table A1's sites and
    cores for the three cylinders, the paper's statement that the elastic wall
    is no slower than the rigid one, and the site-update rates the two tables
    imply (sites x 1000 / wall time): 5,318 / 13,168 / 31,235 MLUPS elastic,
    1.73 / 2.19 / 2.60 MLUPS per core."""
    a1 = {name: (sites, cores) for name, _, _, _, _, sites, cores in _table_a1()}
    want = {50: (5318, 1.73), 100: (13168, 2.19), 200: (31235, 2.60)}
    for r, elastic, rigid, sites, cores in _walltimes():
        assert a1["cylinder_R%d" % r] == (sites, cores)
        assert elastic <= rigid
        mlups = sites * 1000 / elastic / 1e6
        assert abs(mlups - want[r][0]) < 1.0
        assert abs(mlups / cores - want[r][1]) < 0.005
