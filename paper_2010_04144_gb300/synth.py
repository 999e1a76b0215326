"""Seeded synthetic inputs: voxelised vessel geometries and request streams.

This module produces *inputs only*: lists of fluid lattice points plus the
descriptors of their inlets/outlets ("iolets"), and seeded request streams.
It holds none of the lattice-Boltzmann arithmetic (no velocity set, no
neighbour table, no boundary rule, no collision, no coupling factor); both
the CUDA path and the FP64 oracle start from what it returns.

The paper's geometries (the circle-of-Willis data set of Section 2.2 and the
Yoon-sun leg vasculature of Section 3.1) are not available.  Seeded
bifurcating trees stand in for them: Section 3.1 describes vessel trees
clipped flat and perpendicular at their tips, which is what the leaves here
are.

Conventions shared with the iolet descriptor format of the C-ABI:
  * fluid sites are integer lattice points (x, y, z) with 0 <= x, y, z < 2^21;
  * an iolet centre, axis and radius are fixed-point integers in units of
    2^-10 lattice units; the axis points OUT of the fluid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FIX = 1024  # fixed-point scale of iolet descriptors (2^-10 lattice units)

PRESSURE, VELOCITY = 0, 1
PLUG, PARABOLIC = 0, 1
PULSE_CONST, PULSE_COSINE, PULSE_SINE = 0, 1, 2

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood 2014); uniform() = top 53 bits / 2^53."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) / float(1 << 53)


@dataclass
class Iolet:
    """Inlet/outlet descriptor (same fields as the C-ABI's hg_iolet)."""
    kind: int                 # PRESSURE or VELOCITY
    centre: tuple             # fixed point (2^-10)
    axis: tuple               # fixed point, outward
    radius: int               # fixed point
    value: float = 0.0        # density deviation (pressure) or peak speed (velocity)
    profile: int = PLUG       # velocity iolets: PLUG or PARABOLIC
    pulse: int = PULSE_CONST  # time modulation of value
    period: float = 0.0       # steps (pulsed iolets)

    def area(self) -> float:
        r = self.radius / FIX
        return math.pi * r * r

    def centre_lu(self) -> np.ndarray:
        return np.asarray(self.centre, dtype=np.float64) / FIX


@dataclass
class Geometry:
    xyz: np.ndarray                  # (n, 3) int32, any order, no duplicates
    iolets: list                     # list[Iolet]
    origin: tuple = (0, 0, 0)        # integer lattice offset of this geometry in a shared frame
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


# --------------------------------------------------------------------------
# point-set helpers
# --------------------------------------------------------------------------

def _pack(x, y, z):
    return (x.astype(np.int64) | (y.astype(np.int64) << 21) | (z.astype(np.int64) << 42))


def _unpack(k):
    m = (1 << 21) - 1
    return np.stack([(k & m), ((k >> 21) & m), ((k >> 42) & m)], axis=1).astype(np.int32)


def _expand_rows(xs, ys, zlo, zhi):
    cnt = np.maximum(zhi - zlo + 1, 0)
    keep = cnt > 0
    xs, ys, zlo, cnt = xs[keep], ys[keep], zlo[keep], cnt[keep]
    if cnt.size == 0:
        return np.zeros(0, dtype=np.int64)
    tot = int(cnt.sum())
    rx = np.repeat(xs, cnt)
    ry = np.repeat(ys, cnt)
    start = np.repeat(zlo, cnt)
    offs = np.arange(tot, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    return _pack(rx, ry, start + offs)


def _rows(lo, hi):
    xs = np.arange(lo[0], hi[0] + 1, dtype=np.int64)
    ys = np.arange(lo[1], hi[1] + 1, dtype=np.int64)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return X.ravel(), Y.ravel()


def cylinder_points(P, Q, r):
    """Lattice points X with 0 <= (X-P).a <= |Q-P| and distance to the axis <= r.

    Works row by row: for each (x, y) the admissible z form one interval
    (quadratic radial condition intersected with the axial slab).
    """
    P = np.asarray(P, np.float64)
    Q = np.asarray(Q, np.float64)
    ax = Q - P
    ell = float(np.linalg.norm(ax))
    a = ax / ell
    lo = np.floor(np.minimum(P, Q) - r - 1).astype(np.int64)
    hi = np.ceil(np.maximum(P, Q) + r + 1).astype(np.int64)
    X, Y = _rows(lo, hi)
    dx = X - P[0]
    dy = Y - P[1]
    alpha = dx * a[0] + dy * a[1]
    A = 1.0 - a[2] * a[2]
    B = -2.0 * alpha * a[2]
    C = dx * dx + dy * dy - alpha * alpha - r * r
    if A > 1e-12:
        disc = B * B - 4.0 * A * C
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        s_lo = np.where(ok, (-B - sq) / (2 * A), np.inf)
        s_hi = np.where(ok, (-B + sq) / (2 * A), -np.inf)
    else:
        ok = C <= 0
        s_lo = np.where(ok, -np.inf, np.inf)
        s_hi = np.where(ok, np.inf, -np.inf)
    if abs(a[2]) > 1e-12:
        t0 = (0.0 - alpha) / a[2]
        t1 = (ell - alpha) / a[2]
        s_lo = np.maximum(s_lo, np.minimum(t0, t1))
        s_hi = np.minimum(s_hi, np.maximum(t0, t1))
    else:
        inside = (alpha >= 0) & (alpha <= ell)
        s_lo = np.where(inside, s_lo, np.inf)
        s_hi = np.where(inside, s_hi, -np.inf)
    s_lo = np.clip(s_lo, lo[2] - P[2] - 1, hi[2] - P[2] + 1)
    s_hi = np.clip(s_hi, lo[2] - P[2] - 1, hi[2] - P[2] + 1)
    zlo = np.ceil(s_lo + P[2]).astype(np.int64)
    zhi = np.floor(s_hi + P[2]).astype(np.int64)
    return _expand_rows(X, Y, zlo, zhi)


def sphere_points(Cn, r):
    Cn = np.asarray(Cn, np.float64)
    lo = np.floor(Cn - r - 1).astype(np.int64)
    hi = np.ceil(Cn + r + 1).astype(np.int64)
    X, Y = _rows(lo, hi)
    rem = r * r - (X - Cn[0]) ** 2 - (Y - Cn[1]) ** 2
    ok = rem >= 0
    h = np.sqrt(np.where(ok, rem, 0.0))
    zlo = np.where(ok, np.ceil(Cn[2] - h), 1).astype(np.int64)
    zhi = np.where(ok, np.floor(Cn[2] + h), 0).astype(np.int64)
    return _expand_rows(X, Y, zlo, zhi)


def _fix3(v):
    return tuple(int(round(float(c) * FIX)) for c in v)


# --------------------------------------------------------------------------
# straight tube and closed box
# --------------------------------------------------------------------------

def cylinder(radius=8, length=64, axis=2, margin=2, inlet=None, outlet=None):
    """Straight voxelised tube: points with (u-c)^2 + (v-c)^2 <= R^2, axial index 0..length-1.

    The tube's axis lies on lattice points (c = margin + R).  Both ends are cut
    flat half a lattice unit beyond the last fluid layer; the inlet sits at the
    low end with outward axis -e_axis, the outlet at the high end.
    ``inlet`` / ``outlet`` are dicts of Iolet fields (kind, value, ...).
    """
    R = int(radius)
    c = margin + R
    u, v = np.meshgrid(np.arange(c - R, c + R + 1), np.arange(c - R, c + R + 1), indexing="ij")
    m = (u - c) ** 2 + (v - c) ** 2 <= R * R
    u, v = u[m], v[m]
    w = np.arange(margin, margin + length)
    U = np.repeat(u, length)
    V = np.repeat(v, length)
    Wc = np.tile(w, u.size)
    pts = [None, None, None]
    others = [d for d in range(3) if d != axis]
    pts[others[0]], pts[others[1]], pts[axis] = U, V, Wc
    xyz = np.stack(pts, axis=1).astype(np.int32)
    ctr = [0.0, 0.0, 0.0]
    ctr[others[0]] = c
    ctr[others[1]] = c
    e = [0, 0, 0]
    e[axis] = 1
    io = []
    inl = dict(kind=PRESSURE, value=0.001) if inlet is None else dict(inlet)
    out = dict(kind=PRESSURE, value=0.0) if outlet is None else dict(outlet)
    c_in = list(ctr)
    c_in[axis] = margin - 0.5
    c_out = list(ctr)
    c_out[axis] = margin + length - 0.5
    io.append(Iolet(centre=_fix3(c_in), axis=tuple(-FIX * x for x in e), radius=R * FIX, **inl))
    io.append(Iolet(centre=_fix3(c_out), axis=tuple(FIX * x for x in e), radius=R * FIX, **out))
    meta = dict(kind="cylinder", radius=R, length=length, axis=axis, centre=c, margin=margin)
    return Geometry(xyz=xyz, iolets=io, meta=meta)


def box(nx, ny, nz, margin=2):
    """Closed rectangular box of fluid (every boundary link is a wall)."""
    X, Y, Z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.int32) + margin
    return Geometry(xyz=xyz, iolets=[], meta=dict(kind="box", shape=(nx, ny, nz)))


def parallel_tubes(n_tubes, radius=6, length=48, spacing=None, margin=2, inlet=None, outlet=None):
    """``n_tubes`` identical straight tubes along z, side by side in x (one domain)."""
    R = int(radius)
    sp = spacing if spacing is not None else 2 * R + 4
    parts, io = [], []
    for j in range(n_tubes):
        g = cylinder(radius=R, length=length, axis=2, margin=margin, inlet=inlet, outlet=outlet)
        shift = np.array([j * sp, 0, 0], dtype=np.int32)
        parts.append(g.xyz + shift)
        for d in g.iolets:
            cx, cy, cz = d.centre
            io.append(Iolet(kind=d.kind, centre=(cx + j * sp * FIX, cy, cz), axis=d.axis,
                            radius=d.radius, value=d.value, profile=d.profile,
                            pulse=d.pulse, period=d.period))
    # order iolets: all inlets first (tube order), then all outlets
    io = io[0::2] + io[1::2]
    return Geometry(xyz=np.concatenate(parts), iolets=io,
                    meta=dict(kind="tubes", n=n_tubes, radius=R, length=length, spacing=sp))


# --------------------------------------------------------------------------
# bifurcating trees
# --------------------------------------------------------------------------

def _perp_basis(d):
    ref = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(d, ref)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    return e1, e2


def _rotate(v, k, th):
    """Rodrigues rotation of v about unit axis k by angle th."""
    return v * math.cos(th) + np.cross(k, v) * math.sin(th) + k * np.dot(k, v) * (1 - math.cos(th))


@dataclass
class TreeSpec:
    depth: int = 6
    root_radius: float = 24.0
    seed: int = 2010041442
    scale: float = 1.0                 # multiplies every length (radii and segment lengths)
    len_range: tuple = (6.0, 10.0)     # segment length in units of its radius
    angle_range: tuple = (30.0, 70.0)  # branching angle, degrees
    murray: float = 2.0 ** (-1.0 / 3.0)


def tree_centrelines(spec: TreeSpec):
    """Heap-ordered segments (P, Q, r) of a seeded binary tree, in lattice units (float)."""
    rng = SplitMix64(spec.seed)
    nseg = 2 ** spec.depth - 1
    P = [None] * nseg
    Q = [None] * nseg
    D = [None] * nseg
    r = [0.0] * nseg
    P[0] = np.zeros(3)
    D[0] = np.array([0.0, 0.0, 1.0])
    r[0] = spec.root_radius * spec.scale
    lo_l, hi_l = spec.len_range
    lo_a, hi_a = spec.angle_range
    for n in range(nseg):
        ell = lo_l + (hi_l - lo_l) * rng.uniform()
        Q[n] = P[n] + D[n] * ell * r[n]
        c1, c2 = 2 * n + 1, 2 * n + 2
        if c1 < nseg:
            phi = 2.0 * math.pi * rng.uniform()
            th1 = math.radians(lo_a + (hi_a - lo_a) * rng.uniform())
            th2 = math.radians(lo_a + (hi_a - lo_a) * rng.uniform())
            e1, e2 = _perp_basis(D[n])
            b = math.cos(phi) * e1 + math.sin(phi) * e2
            for c, th in ((c1, th1), (c2, -th2)):
                d = _rotate(D[n], b, th)
                D[c] = d / np.linalg.norm(d)
                r[c] = r[n] * spec.murray
                P[c] = Q[n]
    return P, Q, r


def tree(spec: TreeSpec = TreeSpec(), venous: bool = False, radius_factor: float = 1.2,
         inlet_speed: float = 0.05, period: float = 1000.0, pulse: int = PULSE_COSINE,
         venous_offset: float = 0.0):
    """Voxelised bifurcating tree with flat-cut root and leaves.

    Arterial form: the root start is a velocity inlet (parabolic profile, peak
    ``inlet_speed`` modulated by ``pulse`` with ``period``), every leaf end is a
    pressure outlet at zero density deviation.  Iolet 0 is the root; leaves
    follow in heap (breadth-first) order.

    Venous form (``venous=True``): the mirror image x -> -x of the same
    centrelines with radii multiplied by ``radius_factor``; the leaves become
    velocity inlets (plug profile, value 0 until coupled) and the root becomes
    a pressure outlet.  Iolet 0 is still the root.
    """
    P, Q, r = tree_centrelines(spec)
    nseg = len(P)
    if venous:
        mir = np.array([-1.0, 1.0, 1.0])
        P = [p * mir for p in P]
        Q = [q * mir for q in Q]
        r = [x * radius_factor for x in r]
    Pq = [np.round(p * FIX) / FIX for p in P]
    Qq = [np.round(q * FIX) / FIX for q in Q]
    lows = np.array([np.minimum(Pq[n], Qq[n]) - r[n] - 2.0 for n in range(nseg)]).min(axis=0)
    shift = -np.floor(lows)
    Pq = [p + shift for p in Pq]
    Qq = [q + shift for q in Qq]
    keys = []
    first_leaf = 2 ** (spec.depth - 1) - 1
    for n in range(nseg):
        keys.append(cylinder_points(Pq[n], Qq[n], r[n]))
        if n < first_leaf:
            keys.append(sphere_points(Qq[n], r[n]))
    k = np.unique(np.concatenate(keys))
    xyz = _unpack(k)
    io = []
    root_axis = _fix3(-(Qq[0] - Pq[0]) / np.linalg.norm(Qq[0] - Pq[0]))
    leaves = list(range(first_leaf, nseg))
    if not venous:
        io.append(Iolet(kind=VELOCITY, centre=_fix3(Pq[0]), axis=root_axis,
                        radius=int(round(r[0] * FIX)), value=inlet_speed, profile=PARABOLIC,
                        pulse=pulse, period=period))
        for n in leaves:
            a = (Qq[n] - Pq[n]) / np.linalg.norm(Qq[n] - Pq[n])
            io.append(Iolet(kind=PRESSURE, centre=_fix3(Qq[n]), axis=_fix3(a),
                            radius=int(round(r[n] * FIX)), value=0.0))
    else:
        io.append(Iolet(kind=PRESSURE, centre=_fix3(Pq[0]), axis=root_axis,
                        radius=int(round(r[0] * FIX)), value=0.0))
        for n in leaves:
            a = (Qq[n] - Pq[n]) / np.linalg.norm(Qq[n] - Pq[n])
            io.append(Iolet(kind=VELOCITY, centre=_fix3(Qq[n]), axis=_fix3(a),
                            radius=int(round(r[n] * FIX)), value=0.0, profile=PLUG))
    # shared frame: the venous tree is placed beside the arterial one
    origin = tuple(int(v) for v in (-shift + np.array([venous_offset, 0.0, 0.0])))
    meta = dict(kind="tree", depth=spec.depth, root_radius=spec.root_radius, seed=spec.seed,
                scale=spec.scale, venous=venous, n_segments=nseg, leaves=leaves,
                radii=[float(x) for x in r], shift=[float(x) for x in shift],
                segments=[(tuple(float(x) for x in Pq[n]), tuple(float(x) for x in Qq[n]))
                          for n in range(nseg)])
    return Geometry(xyz=xyz, iolets=io, origin=origin, meta=meta)


def tree_volume_estimate(spec: TreeSpec) -> float:
    """Sum of segment cylinder volumes (overlaps ignored): a cheap size estimate."""
    P, Q, r = tree_centrelines(spec)
    return float(sum(math.pi * r[n] ** 2 * np.linalg.norm(Q[n] - P[n]) for n in range(len(P))))


def scale_for_sites(spec: TreeSpec, target_sites: float) -> float:
    """Length scale that makes a tree of this shape hold about ``target_sites`` sites."""
    base = TreeSpec(**{**spec.__dict__, "scale": 1.0})
    return (target_sites / tree_volume_estimate(base)) ** (1.0 / 3.0)


# --------------------------------------------------------------------------
# seeded perturbations and request streams
# --------------------------------------------------------------------------

def random_state(n, seed, amplitude=1e-3, dtype=np.float64):
    """Seeded uniform perturbation, shape (19, n), in (-amplitude, amplitude)."""
    g = np.random.default_rng(seed)
    return (amplitude * (2.0 * g.random((19, n)) - 1.0)).astype(dtype)


def uniform_draws(seed, n):
    """n SplitMix64 uniforms in [0, 1) (used for the coupling pressure-drop draws)."""
    rng = SplitMix64(seed)
    return np.array([rng.uniform() for _ in range(n)])


@dataclass
class Request:
    rid: int
    arrival_s: float
    spec: TreeSpec
    coupled: bool
    steps: int


def request_stream(n_requests=256, rate_per_s=4.0, arrival_seed=7, steps=2000,
                   depth_range=(3, 8), sites_range=(5e4, 4e7), root_radius=24.0):
    """Seeded serving workload: tree requests with Poisson arrivals.

    Request i uses seed i: depth ~ U{3..8}, target sites log-uniform in
    ``sites_range`` (realised through the tree's length scale), coupled
    arterial/venous pair with probability 1/2.
    """
    arr = SplitMix64(arrival_seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += -math.log(1.0 - arr.uniform()) / rate_per_s
        g = SplitMix64(i)
        d = depth_range[0] + int(g.uniform() * (depth_range[1] - depth_range[0] + 1))
        lo, hi = math.log(sites_range[0]), math.log(sites_range[1])
        target = math.exp(lo + (hi - lo) * g.uniform())
        coupled = g.uniform() < 0.5
        spec = TreeSpec(depth=d, root_radius=root_radius, seed=1_000_003 * (i + 1))
        per_domain = target / (2.44 if coupled else 1.0)
        spec.scale = scale_for_sites(spec, per_domain)
        out.append(Request(rid=i, arrival_s=t, spec=spec, coupled=coupled, steps=steps))
    return out
