"""Seeded vessel geometries voxelised into label grids.

Label convention (shared by the oracle and the library): 0 solid, 1 fluid,
2+k ghost node of iolet k.  A node is fluid iff it lies strictly inside the
vessel; ghost nodes are the nodes just beyond an end cap that lie radially
inside it.  Grids are indexed ``labels[x, y, z]`` (C order, z fastest).
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Iolet:
    """An inlet (kind 0, prescribed velocity) or outlet (kind 1, prescribed density).

    ``axis`` is the unit direction of the mean flow (into the domain at an
    inlet, out of it at an outlet); ``centre`` is a point on the vessel axis;
    ``profile`` selects the inlet shape (0 parabolic, 1 rigid Womersley,
    2 plug).  The inlet velocity is ``axis * (u_mean p0(r) + u_amp (ps(r)
    sin(theta) + pc(r) cos(theta)))`` with ``theta = 2 pi n / period + phase``;
    ``period <= 0`` means steady.
    """
    kind: int
    centre: tuple
    axis: tuple
    radius: float
    profile: int = 0
    rho: float = 1.0
    u_mean: float = 0.0
    u_amp: float = 0.0
    period: float = 0.0
    phase: float = 0.0


@dataclass
class Geometry:
    labels: np.ndarray
    iolets: list
    name: str = ""
    radius: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.labels.shape

    def n_fluid(self):
        return int(np.count_nonzero(self.labels == 1))


def _disc(n, radius, centre):
    ii = np.arange(n, dtype=np.float64) - centre
    return ii[:, None] ** 2 + ii[None, :] ** 2 < radius * radius


def tube(radius, length, margin=2, u_mean=0.025, u_amp=0.0, period=0.0, phase=0.0, rho_out=1.0,
         profile=0, closed=False):
    """Straight z-aligned cylinder of ``length`` fluid planes with ghost planes at both ends.

    Box: ``(2R + 2 margin) x (2R + 2 margin) x (length + 2)``; axis at the box
    centre ``(n - 1)/2``; fluid planes ``z = 1..length``; inlet ghosts at
    ``z = 0`` (iolet 0, velocity), outlet ghosts at ``z = length + 1``
    (iolet 1, density ``rho_out``).  ``closed=True`` makes both caps solid and
    drops the iolets.
    """
    n = int(2 * np.ceil(radius) + 2 * margin)
    c = (n - 1) / 2.0
    disc = _disc(n, radius, c)
    labels = np.zeros((n, n, length + 2), np.uint8)
    labels[disc, 1:length + 1] = 1
    iolets = []
    if not closed:
        labels[disc, 0] = 2
        labels[disc, length + 1] = 3
        iolets = [
            Iolet(kind=0, centre=(c, c, 0.0), axis=(0.0, 0.0, 1.0), radius=float(radius),
                  profile=profile, u_mean=u_mean, u_amp=u_amp, period=period, phase=phase),
            Iolet(kind=1, centre=(c, c, float(length + 1)), axis=(0.0, 0.0, 1.0),
                  radius=float(radius), rho=rho_out),
        ]
    return Geometry(labels, iolets, name="tube_R%g_L%d" % (radius, length), radius=float(radius),
                    meta={"centre": (c, c), "length": length})


def duct(width, height, length, rho_in=1.001, rho_out=0.999, inlet=None):
    """Rectangular duct: fluid ``x = 1..width``, ``y = 1..height``, ``z = 1..length``.

    Solid walls at ``x = 0, width+1`` and ``y = 0, height+1``; ghost planes at
    ``z = 0`` (iolet 0) and ``z = length+1`` (iolet 1).  By default both ends
    are fixed-density (pressure-driven flow); ``inlet`` replaces iolet 0.
    """
    nx, ny, nz = width + 2, height + 2, length + 2
    labels = np.zeros((nx, ny, nz), np.uint8)
    labels[1:width + 1, 1:height + 1, 1:length + 1] = 1
    labels[1:width + 1, 1:height + 1, 0] = 2
    labels[1:width + 1, 1:height + 1, length + 1] = 3
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    r = float(max(width, height))
    io0 = inlet if inlet is not None else Iolet(kind=1, centre=(cx, cy, 0.0), axis=(0.0, 0.0, 1.0),
                                                radius=r, rho=rho_in)
    io1 = Iolet(kind=1, centre=(cx, cy, float(length + 1)), axis=(0.0, 0.0, 1.0), radius=r,
                rho=rho_out)
    return Geometry(labels, [io0, io1], name="duct_%dx%dx%d" % (width, height, length),
                    meta={"width": width, "height": height, "length": length})


def closed_box(nx, ny, nz):
    """Fluid interior of a box whose one-node shell is solid (no iolets)."""
    labels = np.zeros((nx, ny, nz), np.uint8)
    labels[1:-1, 1:-1, 1:-1] = 1
    return Geometry(labels, [], name="box_%dx%dx%d" % (nx, ny, nz))


def random_labels(seed, shape, fill=0.7, n_iolets=2):
    """Random label grid for integer-build fuzzing and short parity runs.

    Fluid with probability ``fill``; a random subset of the remaining nodes on
    the two z faces become ghosts of iolet 0 (velocity inlet, plug profile) and
    iolet 1 (density outlet).
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    labels = (rng.random(shape) < fill).astype(np.uint8)
    iolets = []
    if n_iolets >= 1:
        face = labels[:, :, 0]
        face[(face == 0) & (rng.random((nx, ny)) < 0.6)] = 2
        iolets.append(Iolet(kind=0, centre=((nx - 1) / 2.0, (ny - 1) / 2.0, 0.0),
                            axis=(0.0, 0.0, 1.0), radius=float(max(nx, ny)), profile=2,
                            u_mean=0.01))
    if n_iolets >= 2:
        face = labels[:, :, nz - 1]
        face[(face == 0) & (rng.random((nx, ny)) < 0.6)] = 3
        iolets.append(Iolet(kind=1, centre=((nx - 1) / 2.0, (ny - 1) / 2.0, float(nz - 1)),
                            axis=(0.0, 0.0, 1.0), radius=float(max(nx, ny)), rho=1.0))
    return Geometry(labels, iolets, name="random_%d" % seed)


# ----------------------------------------------------------------- vessel trees

def _orthonormal(d):
    d = d / np.linalg.norm(d)
    a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(d, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    return d, e1, e2


def _tree_segments(seed, depth, root_radius, split=(0.4, 0.6), angle=(30.0, 60.0),
                   length=(8.0, 12.0), taper=0.10):
    """Segments (start, direction, length, r_start, r_end, level) of a seeded Murray tree.

    Murray's law r_p^3 = r_c1^3 + r_c2^3 with split ratio s ~ U(split) in r^3;
    the two children leave at angles U(angle) on either side of the parent axis,
    in a plane turned 90 degrees from the parent's branching plane; each segment
    is U(length) times its start radius long and its radius falls linearly by
    ``taper`` along it; children start from the parent's end radius.
    """
    rng = np.random.default_rng(seed)
    segs = []
    d0, e1, _ = _orthonormal(np.array([0.0, 0.0, 1.0]))
    stack = [(np.zeros(3), d0, e1, float(root_radius), 0)]
    while stack:
        p, d, plane, r0, lev = stack.pop(0)
        L = rng.uniform(*length) * r0
        r1 = r0 * (1.0 - taper)
        segs.append((p.copy(), d.copy(), L, r0, r1, lev))
        if lev == depth:
            continue
        end = p + L * d
        s = rng.uniform(*split)
        radii = (r1 * s ** (1.0 / 3.0), r1 * (1.0 - s) ** (1.0 / 3.0))
        _, a, b = _orthonormal(d)
        # branching plane spanned by d and `plane`; next level turns it by 90 degrees
        n_plane = np.cross(d, plane)
        for sign, rc in zip((1.0, -1.0), radii):
            th = np.deg2rad(rng.uniform(*angle))
            dc = np.cos(th) * d + sign * np.sin(th) * plane
            dc /= np.linalg.norm(dc)
            stack.append((end.copy(), dc, n_plane / np.linalg.norm(n_plane), rc, lev + 1))
    return segs


def murray_tree(seed=0, depth=6, root_radius=48.0, margin=3, max_voxels=4_000_000_000, **kw):
    """Voxelised seeded bifurcating tree: root inlet (iolet 0), one outlet per leaf.

    Returns a Geometry whose ``meta['segments']`` lists the frusta and whose
    ``meta['segment_of_voxel']`` (uint8, 255 = none) gives the segment that owns
    each fluid node, from which the local rest radius is found by
    :func:`rest_radius`.
    """
    segs = _tree_segments(seed, depth, root_radius, **kw)
    lo = np.full(3, np.inf)
    hi = np.full(3, -np.inf)
    for p, d, L, r0, r1, lev in segs:
        for q in (p, p + L * d):
            lo = np.minimum(lo, q - r0 - 2)
            hi = np.maximum(hi, q + r0 + 2)
    lo = np.floor(lo) - margin
    hi = np.ceil(hi) + margin
    shape = tuple(int(v) for v in (hi - lo + 1))
    if int(np.prod(shape, dtype=np.int64)) > max_voxels:
        raise ValueError("tree box %s exceeds max_voxels" % (shape,))
    labels = np.zeros(shape, np.uint8)
    owner = np.full(shape, 255, np.uint8)
    iolets = []
    for k, (p, d, L, r0, r1, lev) in enumerate(segs):
        pl = p - lo
        e = pl + L * d
        rmax = max(r0, r1)
        bl = np.maximum(np.floor(np.minimum(pl, e) - rmax - 1), 0).astype(int)
        bh = np.minimum(np.ceil(np.maximum(pl, e) + rmax + 1), np.array(shape) - 1).astype(int)
        X, Y, Z = np.meshgrid(*[np.arange(bl[a], bh[a] + 1, dtype=np.float64) for a in range(3)],
                              indexing="ij")
        rel = np.stack([X - pl[0], Y - pl[1], Z - pl[2]], -1)
        t = rel @ d
        rad2 = np.einsum("...i,...i->...", rel, rel) - t * t
        rt = r0 + (r1 - r0) * np.clip(t / L, 0.0, 1.0)
        inside = (t >= 0.0) & (t <= L) & (rad2 < rt * rt)
        # children overlap their parent's end; joints are filled by both
        sub = labels[bl[0]:bh[0] + 1, bl[1]:bh[1] + 1, bl[2]:bh[2] + 1]
        osub = owner[bl[0]:bh[0] + 1, bl[1]:bh[1] + 1, bl[2]:bh[2] + 1]
        newf = inside & (sub != 1)
        sub[inside] = 1
        osub[newf] = k
    # caps: the root's start (inlet) and every leaf's end (outlets)
    caps = [(0, segs[0][0] - lo, -segs[0][1], segs[0][3])]
    caps += [(k, s[0] - lo + s[2] * s[1], s[1], s[4]) for k, s in enumerate(segs) if s[5] == depth]
    # ghost layers beyond the caps: nodes within sqrt(3) past the cap plane, radially inside
    for ci, (k, centre_l, outward, rc) in enumerate(caps):
        bl = np.maximum(np.floor(centre_l - rc - 3), 0).astype(int)
        bh = np.minimum(np.ceil(centre_l + rc + 3), np.array(shape) - 1).astype(int)
        X, Y, Z = np.meshgrid(*[np.arange(bl[a], bh[a] + 1, dtype=np.float64) for a in range(3)],
                              indexing="ij")
        rel = np.stack([X - centre_l[0], Y - centre_l[1], Z - centre_l[2]], -1)
        ta = rel @ outward
        r2 = np.einsum("...i,...i->...", rel, rel) - ta * ta
        ghost = (ta > 0.0) & (ta <= np.sqrt(3.0) + 1e-9) & (r2 < rc * rc)
        sub = labels[bl[0]:bh[0] + 1, bl[1]:bh[1] + 1, bl[2]:bh[2] + 1]
        ghost &= sub == 0
        code = 2 + len(iolets)
        sub[ghost] = code
        centre = tuple(float(v) for v in centre_l)
        if ci == 0:
            iolets.append(Iolet(kind=0, centre=centre, axis=tuple(float(v) for v in -outward),
                                radius=float(rc), profile=0))
        else:
            iolets.append(Iolet(kind=1, centre=centre, axis=tuple(float(v) for v in outward),
                                radius=float(rc), rho=1.0))
    return Geometry(labels, iolets, name="tree_seed%d_d%d" % (seed, depth), radius=root_radius,
                    meta={"segments": segs, "origin": lo, "segment_of_voxel": owner})


def rest_radius(geom, coords):
    """Local rest radius r0 at the given integer node coordinates of a tree or tube."""
    coords = np.asarray(coords)
    if "segments" not in geom.meta:
        return np.full(len(coords), geom.radius)
    owner = geom.meta["segment_of_voxel"][coords[:, 0], coords[:, 1], coords[:, 2]]
    segs = geom.meta["segments"]
    lo = geom.meta["origin"]
    out = np.zeros(len(coords))
    for k in np.unique(owner):
        if k == 255:
            continue
        p, d, L, r0, r1, lev = segs[k]
        m = owner == k
        t = (coords[m] - (p - lo)) @ d
        out[m] = r0 + (r1 - r0) * np.clip(t / L, 0.0, 1.0)
    return out


def tube_ensemble(seed=0, count=256, radius=(6.0, 24.0), length=(64, 512), stiffness=(0.05, 5.0),
                  period=(1000.0, 5000.0), tau=(0.55, 1.0), sigma=0.5):
    """Seeded parameters of an ensemble of independent elastic tubes.

    Radii U(radius), lengths U(length), Eh/r0 log-uniform in ``stiffness``,
    inlet periods U(period), relaxation times U(tau).  Each member's stiffness
    is returned both as Eh/r0 and as the lattice tube-law coefficient
    ``kappa = (1 - sigma^2) r0 / (Eh/r0)``.
    """
    rng = np.random.default_rng(seed)
    R = rng.uniform(*radius, count)
    L = rng.integers(length[0], length[1] + 1, count)
    Eh = np.exp(rng.uniform(np.log(stiffness[0]), np.log(stiffness[1]), count))
    T = rng.uniform(*period, count)
    taus = rng.uniform(*tau, count)
    return [dict(radius=float(R[i]), length=int(L[i]), eh_r0=float(Eh[i]), period=float(T[i]),
                 tau=float(taus[i]), kappa=float((1 - sigma ** 2) * R[i] / Eh[i]))
            for i in range(count)]


def wall_normals(geom, coords):
    """Outward unit normals of the vessel surface nearest to the given node coordinates.

    Tubes: the radial direction from the axis; trees: the radial direction from
    the axis of the segment that owns the node (its axial component removed).
    Used to evaluate wall shear stress at wall sites.
    """
    coords = np.asarray(coords, np.float64)
    if "segments" not in geom.meta:
        c = np.array(geom.meta["centre"], np.float64)
        v = np.zeros_like(coords)
        v[:, 0] = coords[:, 0] - c[0]
        v[:, 1] = coords[:, 1] - c[1]
    else:
        ic = coords.astype(np.int64)
        owner = geom.meta["segment_of_voxel"][ic[:, 0], ic[:, 1], ic[:, 2]]
        lo = geom.meta["origin"]
        v = np.zeros_like(coords)
        for k in np.unique(owner):
            if k == 255:
                continue
            p, d, L, r0, r1, lev = geom.meta["segments"][k]
            m = owner == k
            rel = coords[m] - (p - lo)
            v[m] = rel - np.outer(rel @ d, d)
    nrm = np.linalg.norm(v, axis=1)
    nrm[nrm == 0] = 1.0
    return v / nrm[:, None]
