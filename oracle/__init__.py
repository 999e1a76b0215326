"""FP64 CPU oracle of the sparse D3Q19 LBGK hot path (arXiv 2010.04144).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2010_04144_gb300``) and never imports it; the
two meet only through the seeded inputs of ``paper_2010_04144_gb300.synth``.

The arithmetic lives in ``hemeoracle.c`` (plain C, double precision, see the
readings R1-R6 listed at its top); this module only marshals arrays and
sequences the time steps:

  * step t (t = 1, 2, ...) maps F_{t-1} to F_t with boundary values of time t;
  * boundary values of an uncoupled iolet at time t are value * pulse(t);
  * a coupled venous inlet at time t takes factor * M_{t-1}[src].mean_un, the
    arterial outlet mean of the previous time level (Section 3, forward
    direction: scaled average velocity becomes the paired inlet's velocity);
    M_0 is taken over the moments of the initial state;
  * with alternation on (Section 3 alternates the exchange direction), the
    exchange after step e is forward for even e and reverse for odd e.  A
    reverse exchange sets, for every arterial outlet k with coupled venous
    inlets J_k, the speed v_k = mean over j in J_k of (inflow speed at j) /
    factor_j and the force density F_k = -(1/2) v_k |v_k| n_k (n_k the outward
    unit axis): the dynamic pressure of that flow, per lattice unit, opposing
    outflow.  F_k acts, through the Guo forcing of R7, on every site next to
    outlet k from the next step on.  Each exchange leaves the values of the
    other direction as they were.  The paper states this direction in words
    only (no formula, no number); the mapping is pinned by the properties the
    reading fixes (zero inflow gives zero force; the force opposes outflow and
    is quadratic in the speed; fed inlets are averaged, not summed; a forward
    then reverse exchange on a steady pair returns the outlet mean), and the
    forcing itself (R7) by its conservation laws and closed-form flows.

Parity status of each function is listed in ``oracle/coupling.py`` and the
test files under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

PRESSURE, VELOCITY = 0, 1
PLUG, PARABOLIC = 0, 1
PULSE_CONST, PULSE_COSINE, PULSE_SINE = 0, 1, 2


class OrIolet(C.Structure):
    _fields_ = [("kind", C.c_int32), ("profile", C.c_int32), ("pulse", C.c_int32),
                ("pad", C.c_int32), ("value", C.c_double), ("period", C.c_double),
                ("centre", C.c_int64 * 3), ("axis", C.c_int64 * 3), ("radius", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.or_lattice.argtypes = [P, P, P]
        L.or_feq.argtypes = [C.c_double] * 4 + [P]
        L.or_morton.argtypes = [C.c_int32] * 3
        L.or_morton.restype = C.c_uint64
        L.or_classify.argtypes = [C.c_int32] * 3 + [P, C.c_int32]
        L.or_classify.restype = C.c_int
        L.or_build.argtypes = [P, C.c_int64, P, C.c_int32, P, P, P, P]
        L.or_build.restype = C.c_int
        L.or_nbr_rows.argtypes = [P, C.c_int64, P, C.c_int32, P, C.c_int64, P]
        L.or_step.argtypes = [C.c_int64, P, P, P, P, C.c_double, P, P, P, P]
        L.or_step_sites.argtypes = [C.c_int64, P, P, P, C.c_double, P, P, P, P, C.c_int64, P, P]
        L.or_collide.argtypes = [P, C.c_double, P, P, P]
        L.or_moments.argtypes = [C.c_int64, P, P]
        L.or_iolet_means.argtypes = [C.c_int64, P, P, P, C.c_int32, P]
        L.or_mass.argtypes = [C.c_int64, P]
        L.or_mass.restype = C.c_double
        L.or_num_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None and a.size else None


def iolet_array(iolets):
    arr = (OrIolet * max(1, len(iolets)))()
    for k, d in enumerate(iolets):
        e = arr[k]
        e.kind, e.profile, e.pulse = int(d.kind), int(d.profile), int(d.pulse)
        e.value, e.period = float(d.value), float(d.period)
        for j in range(3):
            e.centre[j] = int(d.centre[j])
            e.axis[j] = int(d.axis[j])
        e.radius = int(d.radius)
    return arr


def lattice():
    """(c[19,3], w[19], opp[19]) as the oracle holds them."""
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19, np.float64)
    o = np.zeros(19, np.int32)
    lib().or_lattice(_p(c), _p(w), _p(o))
    return c, w, o


def feq(drho, u):
    out = np.zeros(19, np.float64)
    lib().or_feq(float(drho), float(u[0]), float(u[1]), float(u[2]), _p(out))
    return out


def collide(g, tau, force=None):
    """Collision of one site's streamed values g[19] (R4; R7 with a force): (out[19], mom[4])."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    F = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    out = np.zeros(19, np.float64)
    mom = np.zeros(4, np.float64)
    lib().or_collide(_p(g), float(tau), _p(F), _p(out), _p(mom))
    return out, mom


def morton(x, y, z):
    return int(lib().or_morton(int(x), int(y), int(z)))


def classify(q, iolets):
    arr = iolet_array(iolets)
    return int(lib().or_classify(int(q[0]), int(q[1]), int(q[2]), C.byref(arr), len(iolets)))


def pulse(kind, t, period):
    """Time modulation of an iolet value (reading: the paper gives no waveform)."""
    if kind == PULSE_CONST:
        return 1.0
    if kind == PULSE_COSINE:
        return 0.5 * (1.0 - math.cos(2.0 * math.pi * t / period))
    if kind == PULSE_SINE:
        return math.sin(2.0 * math.pi * t / period)
    raise ValueError(kind)


class Domain:
    """One sparse fluid domain: canonical site order, neighbour table, state."""

    def __init__(self, xyz, iolets, tau=0.8, with_nbr=True):
        xyz = np.ascontiguousarray(xyz, dtype=np.int32)
        n = xyz.shape[0]
        self.n = n
        self.iolets = list(iolets)
        self.tau = float(tau)
        self._io = iolet_array(self.iolets)
        self.perm = np.zeros(n, np.int64)
        self.xyz = np.zeros((n, 3), np.int32)
        self.keys = np.zeros(n, np.uint64)
        self.nbr = np.zeros((18, n), np.int32) if with_nbr else None
        rc = lib().or_build(_p(xyz), n, C.byref(self._io), len(self.iolets), _p(self.perm),
                            _p(self.xyz), _p(self.keys), _p(self.nbr) if with_nbr else None)
        if rc != 0:
            raise ValueError(f"oracle build failed with code {rc}")
        self.F = np.zeros((19, n), np.float64)
        self.mom = np.zeros((n, 4), np.float64)

    def nbr_rows(self, pts):
        pts = np.ascontiguousarray(pts, dtype=np.int32)
        out = np.zeros((pts.shape[0], 18), np.int32)
        lib().or_nbr_rows(_p(self.keys), self.n, C.byref(self._io), len(self.iolets), _p(pts),
                          pts.shape[0], _p(out))
        return out

    def moments(self, F=None):
        F = self.F if F is None else np.ascontiguousarray(F, dtype=np.float64)
        out = np.zeros((self.n, 4), np.float64)
        lib().or_moments(self.n, _p(F), _p(out))
        return out

    def iolet_means(self, mom):
        out = np.zeros((max(1, len(self.iolets)), 3), np.float64)
        if self.iolets:
            mom = np.ascontiguousarray(mom, dtype=np.float64)
            lib().or_iolet_means(self.n, _p(self.nbr), _p(mom), C.byref(self._io),
                                 len(self.iolets), _p(out))
        return out[: len(self.iolets)]

    def mass(self, F=None):
        F = self.F if F is None else np.ascontiguousarray(F, dtype=np.float64)
        return float(lib().or_mass(self.n, _p(F)))

    def adjacent(self, k):
        """Canonical indices of the sites with a link into iolet k."""
        return np.nonzero((self.nbr == -(2 + k)).any(axis=0))[0]

    def step_into(self, Fin, Fout, bcval, mom=None, force=None):
        """One step; force (None = none) is a per-site force density [n, 3] (R7)."""
        bc = np.ascontiguousarray(bcval if len(bcval) else [0.0], dtype=np.float64)
        F = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
        lib().or_step(self.n, _p(self.nbr), _p(self.xyz), _p(Fin), _p(Fout), self.tau,
                      C.byref(self._io), _p(bc), _p(F), _p(mom) if mom is not None else None)

    def step_sites(self, Fin, bcval, sites, force=None):
        """Update of selected sites from state Fin: (out[p,19], mom[p,4])."""
        Fin = np.ascontiguousarray(Fin, dtype=np.float64)
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        bc = np.ascontiguousarray(bcval if len(bcval) else [0.0], dtype=np.float64)
        F = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
        out = np.zeros((sites.size, 19), np.float64)
        mom = np.zeros((sites.size, 4), np.float64)
        lib().or_step_sites(self.n, _p(self.nbr), _p(self.xyz), _p(Fin), self.tau,
                            C.byref(self._io), _p(bc), _p(F), _p(sites), sites.size, _p(out), _p(mom))
        return out, mom


class System:
    """Domains stepped in lockstep, with coupling pairs.

    pairs: iterable of (src_domain, src_iolet, dst_domain, dst_iolet, factor);
    the destination is a velocity iolet whose value at time t becomes
    factor * (mean u.n over the source iolet at time t-1) after a forward
    exchange.  alternate=True alternates forward and reverse exchanges (see
    the module docstring); the default exchanges forward after every step.
    """

    def __init__(self, domains, pairs=(), alternate=False):
        self.domains = list(domains)
        self.pairs = list(pairs)
        self.alternate = bool(alternate)
        self.t = 0
        self._coupled = {}
        for (sd, sk, dd, dk, f) in self.pairs:
            self._coupled[(dd, dk)] = (sd, sk, float(f))
        self._buf = [np.zeros_like(d.F) for d in self.domains]
        self.M = [d.iolet_means(d.moments()) for d in self.domains]
        self.cbv = {key: 0.0 for key in self._coupled}          # coupled inlet values
        self.iolet_force = [np.zeros((len(d.iolets), 3)) for d in self.domains]
        self._adj = {}
        self._exchange(0)

    def forward_exchange(self, e):
        return not self.alternate or e % 2 == 0

    def _exchange(self, e):
        """Exchange after step e (e = 0: the initial state), from the means M_e."""
        if self.forward_exchange(e):
            for (dd, dk), (sd, sk, f) in self._coupled.items():
                self.cbv[(dd, dk)] = f * self.M[sd][sk][0]
            return
        groups = {}
        for (dd, dk), (sd, sk, f) in self._coupled.items():
            inflow = -self.M[dd][dk][0]          # u.n is outward: inflow is its negative
            groups.setdefault((sd, sk), []).append(inflow / f)
        for (sd, sk), speeds in groups.items():
            v = sum(speeds) / len(speeds)
            a = np.array(self.domains[sd].iolets[sk].axis, dtype=np.float64)
            self.iolet_force[sd][sk] = -0.5 * v * abs(v) * (a / np.linalg.norm(a))

    def site_force(self, di):
        """Per-site force density [n, 3] of domain di for the next step, or None."""
        f = self.iolet_force[di]
        forced = np.nonzero(np.abs(f).sum(axis=1))[0]
        if forced.size == 0:
            return None
        d = self.domains[di]
        out = np.zeros((d.n, 3), np.float64)
        for k in forced:
            if (di, k) not in self._adj:
                self._adj[(di, k)] = d.adjacent(k)
            out[self._adj[(di, k)]] += f[k]
        return out

    def bc_values(self, di, t):
        d = self.domains[di]
        out = np.zeros(len(d.iolets), np.float64)
        for k, io in enumerate(d.iolets):
            if (di, k) in self.cbv:
                out[k] = self.cbv[(di, k)]
            else:
                out[k] = io.value * pulse(io.pulse, t, io.period)
        return out

    def step(self, nsteps=1, callback=None):
        for _ in range(nsteps):
            t = self.t + 1
            bcs = [self.bc_values(i, t) for i in range(len(self.domains))]
            forces = [self.site_force(i) for i in range(len(self.domains))]
            for i, d in enumerate(self.domains):
                d.step_into(d.F, self._buf[i], bcs[i], d.mom, forces[i])
                d.F, self._buf[i] = self._buf[i], d.F
            self.M = [d.iolet_means(d.mom) for d in self.domains]
            self.t = t
            self._exchange(t)
            if callback is not None:
                callback(self)


def num_threads():
    return int(lib().or_num_threads())


def set_threads(n):
    lib().or_set_threads(int(n))
