"""Post-processing of read-back fields (Section 3.3 analysis and unit mapping).

Nothing here runs on the device or touches the stepping path: these helpers
take the macroscopic fields a domain returns (``Domain.macroscopic()``:
(drho, ux, uy, uz) per canonical site) and the seeded geometry they came from.

* ``lattice_parameters`` / ``physical_step``: the two relations Section 3.3
  states for single-relaxation-time LB, nu = (tau - 1/2) dx^2 / (3 dt) and
  Ma = sqrt(3) v_max dt / dx (< 0.1), solved for whichever quantity is asked.
* ``velocity_vs_area_planes``: mean speed against vessel cross-section area, the
  quantity Section 3.3 plots for the coupled arterial and venous trees, measured
  as the paper describes: lattice planes at 1/4, 1/2 and 3/4 of the domain's
  length, separated into vessels, area from the convex hull around each
  vessel's lattice points (each point as its unit cell).
* ``velocity_vs_area``: the same quantity per tree segment.  The
  paper cuts measurement planes through the whole domain and separates them
  into vessels; a synthetic tree knows its centrelines, so each segment is cut
  by the plane through its mid-point normal to its axis.  The cross-section is
  the set of sites within half a lattice unit of that plane and within the
  segment radius (+1) of the axis; area = number of those sites (lattice
  units^2, the discrete counterpart of the paper's convex hull), speed = mean
  |u| over them.  Arterial areas are returned negative, as the paper plots
  them, when ``arterial_negative`` is set.
"""
from __future__ import annotations

import math

import numpy as np

from . import synth as S


def lattice_parameters(dx, dt, nu, v_max):
    """(tau, Ma) of a run with spacing dx [m], step dt [s], viscosity nu [m^2/s] and peak
    speed v_max [m/s]: tau = 1/2 + 3 nu dt / dx^2, Ma = sqrt(3) v_max dt / dx."""
    tau = 0.5 + 3.0 * nu * dt / (dx * dx)
    ma = math.sqrt(3.0) * v_max * dt / dx
    return tau, ma


def physical_step(dx, nu, tau):
    """Time step [s] that makes relaxation time tau reproduce viscosity nu at spacing dx."""
    if not tau > 0.5:
        raise ValueError("tau must exceed 1/2")
    return (tau - 0.5) * dx * dx / (3.0 * nu)


def lattice_speed(v_phys, dx, dt):
    """A physical speed [m/s] in lattice units (dx per dt)."""
    return v_phys * dt / dx


class _CellIndex:
    """Sites bucketed into cubes of side C for bounding-box queries."""

    C = 16

    def __init__(self, xyz):
        c = (np.asarray(xyz, np.int64) // self.C)
        self.key = (c[:, 0] << 42) | (c[:, 1] << 21) | c[:, 2]
        self.order = np.argsort(self.key, kind="stable")
        self.sorted = self.key[self.order]

    def query(self, lo, hi):
        lo = np.floor(np.asarray(lo) / self.C).astype(np.int64)
        hi = np.floor(np.asarray(hi) / self.C).astype(np.int64)
        out = []
        for cx in range(lo[0], hi[0] + 1):
            for cy in range(lo[1], hi[1] + 1):
                for cz in range(lo[2], hi[2] + 1):
                    k = (cx << 42) | (cy << 21) | cz
                    a, b = np.searchsorted(self.sorted, [k, k + 1])
                    if b > a:
                        out.append(self.order[a:b])
        return np.concatenate(out) if out else np.zeros(0, np.int64)


def velocity_vs_area(geo, fields, xyz, arterial_negative=False):
    """Rows (segment, area, mean |u|, sites) for every segment of a seeded tree.

    geo: the synth.tree geometry (its segment end points in the lattice frame are
    in ``geo.meta["segments"]``); fields: (n, 4) macroscopic fields in canonical
    order; xyz: (n, 3) canonical site coordinates (``Domain.sites()``)."""
    if geo.meta.get("kind") != "tree":
        raise ValueError("velocity_vs_area needs a seeded tree geometry")
    fields = np.asarray(fields)
    cells = _CellIndex(xyz)
    rows = []
    for n, ((p, q), r) in enumerate(zip(geo.meta["segments"], geo.meta["radii"])):
        p, q = np.array(p), np.array(q)
        a = (q - p) / np.linalg.norm(q - p)
        mid = 0.5 * (p + q)
        cand = cells.query(mid - (r + 2.0), mid + (r + 2.0))
        rel = xyz[cand].astype(np.float64) - mid
        along = rel @ a
        near = np.abs(along) <= 0.5
        perp2 = (rel[near] ** 2).sum(1) - along[near] ** 2
        sel = cand[near][perp2 <= (r + 1.0) ** 2]
        if sel.size == 0:
            continue
        speed = np.linalg.norm(fields[sel, 1:4].astype(np.float64), axis=1)
        area = float(sel.size)
        rows.append((n, -area if arterial_negative else area, float(speed.mean()), int(sel.size)))
    return np.array(rows, dtype=np.float64).reshape(-1, 4)


def _plane_components(P):
    """Connected components of lattice points P (m, 2) under 8-neighbour adjacency."""
    m = P.shape[0]
    parent = np.arange(m)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    index = {(int(x), int(y)): i for i, (x, y) in enumerate(P)}
    for i, (x, y) in enumerate(P):
        for dx, dy in ((1, 0), (0, 1), (1, 1), (1, -1)):
            j = index.get((int(x) + dx, int(y) + dy))
            if j is not None:
                a, b = find(i), find(j)
                if a != b:
                    parent[max(a, b)] = min(a, b)
    roots = np.array([find(i) for i in range(m)])
    _, labels = np.unique(roots, return_inverse=True)
    return labels


def _hull_area(P):
    """Area of the convex hull of 2-D points (0 for fewer than 3 or collinear points)."""
    if P.shape[0] < 3:
        return 0.0
    pts = np.unique(P.astype(np.float64), axis=0)
    if pts.shape[0] < 3:
        return 0.0
    # Andrew's monotone chain, then the shoelace formula
    pts = pts[np.lexsort((pts[:, 1], pts[:, 0]))]

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in pts[::-1]:
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    hull = np.array(lower[:-1] + upper[:-1])
    if hull.shape[0] < 3:
        return 0.0
    x, y = hull[:, 0], hull[:, 1]
    return 0.5 * abs(float(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1))))


def _cell_hull_area(P):
    """Area of the convex hull around lattice points P (m, 2), each point taken as the unit
    square it stands for: one rule for every vessel size (one site: 1; a one-site-wide line
    of k sites: k; never 0), and within half a lattice unit of the hull through the points'
    centres along the rim of a large vessel."""
    P = np.asarray(P, np.float64)
    corners = np.concatenate([P + d for d in ((-0.5, -0.5), (-0.5, 0.5), (0.5, -0.5), (0.5, 0.5))])
    return _hull_area(corners)


def velocity_vs_area_planes(fields, xyz, fractions=(0.25, 0.5, 0.75), axis=None,
                            arterial_negative=False):
    """Section 3.3's measurement as the paper describes it: lattice planes normal to the
    domain's longest extent (or ``axis``) at the given fractions of its length, each cut
    separated into vessels (8-connected groups of sites in the plane), each vessel's area
    the convex hull around its lattice points (each point as its unit cell, so vessels one
    site wide keep a non-zero area), its speed the mean |u| over them.

    Returns rows (fraction, vessel, area, mean |u|, sites); areas negative when
    ``arterial_negative`` is set, as the paper plots the arterial vessels."""
    X = np.asarray(xyz, np.int64)
    fields = np.asarray(fields)
    if axis is None:
        axis = int(np.argmax(X.max(axis=0) - X.min(axis=0)))
    others = [a for a in range(3) if a != axis]
    lo, hi = int(X[:, axis].min()), int(X[:, axis].max())
    rows = []
    for f in fractions:
        level = int(round(lo + f * (hi - lo)))
        sel = np.nonzero(X[:, axis] == level)[0]
        if sel.size == 0:
            continue
        P = X[sel][:, others]
        labels = _plane_components(P)
        for c in range(labels.max() + 1):
            mem = sel[labels == c]
            Pc = X[mem][:, others]
            area = _cell_hull_area(Pc)
            speed = float(np.linalg.norm(fields[mem, 1:4].astype(np.float64), axis=1).mean())
            rows.append((f, c, -area if arterial_negative else area, speed, int(mem.size)))
    return np.array(rows, dtype=np.float64).reshape(-1, 5)
