"""Coupling map and scale factors of the arterial-venous self-coupling (Section 3).

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).

greedy_map   Section 3, coupling-map paragraph: arteries are visited in
             ascending order and each takes the closest venous inlet still
             unassigned (which is then removed); afterwards every venous inlet
             left over joins its closest artery.  Distances are Euclidean
             between iolet centres.  Readings: ties go to the lowest index;
             distances are compared exactly as squared fixed-point integers.
velocity_factors
             Eq. (1) dP_i = k_i q_i L_i with k_i proportional to 1/A_i, plus
             mass conservation q_0 = sum_i q_i, give the velocity scale factor
             printed after Eq. (1); it is evaluated here exactly in that form,
             normalised by pair 1 as printed.
pressure_drops
             Section 3: each pair's pressure-drop factor dP_i/P_0 is drawn
             uniformly in [0.3, 0.7]; the uniform numbers are an input.
"""
from __future__ import annotations

import math


def _d2(a, b):
    return sum((int(a[j]) - int(b[j])) ** 2 for j in range(3))


def greedy_map(art_centres, ven_centres):
    """Return (assign, dist): assign[v] = artery of venous inlet v, dist[v] = L_v (lattice units).

    Centres are fixed-point integer triples (units of 2^-10 lattice units).
    """
    na, nv = len(art_centres), len(ven_centres)
    if na == 0:
        raise ValueError("no arterial outlets")
    assign = [-1] * nv
    remaining = list(range(nv))
    for a in range(na):
        if not remaining:
            break
        best = min(remaining, key=lambda v: (_d2(art_centres[a], ven_centres[v]), v))
        assign[best] = a
        remaining.remove(best)
    for v in sorted(remaining):
        assign[v] = min(range(na), key=lambda a: (_d2(art_centres[a], ven_centres[v]), a))
    dist = [math.sqrt(_d2(art_centres[assign[v]], ven_centres[v])) / 1024.0 for v in range(nv)]
    return assign, dist


def velocity_factors(A0, dP, L, A):
    """v_i / v_0 for the N inlets coupled to one outlet of area A0 (printed form after Eq. (1)).

    dP[i] = dP_i / P_0, L[i] = distance, A[i] = inlet area, i = 0..N-1 (the
    paper's i = 1..N; its normalising pair "1" is index 0 here).
    """
    N = len(dP)
    if N == 0:
        return []
    if any(l <= 0 for l in L) or any(a <= 0 for a in A) or A0 <= 0:
        raise ValueError("lengths and areas must be positive")
    ratio = [dP[i] * L[0] * A[i] / (dP[0] * L[i] * A[0]) for i in range(N)]
    total = 0.0
    for r in ratio:
        total += r
    return [(A0 / A[i]) * ratio[i] / total for i in range(N)]


def pressure_drops(uniforms):
    """dP_i / P_0 ~ U(0.3, 0.7) from given uniforms in [0, 1)."""
    return [0.3 + 0.4 * u for u in uniforms]


def coupling_table(art_centres, art_areas, ven_centres, ven_areas, uniforms):
    """Greedy map + drawn pressure drops + factors: list of (artery, vein, L, dP, factor)."""
    assign, dist = greedy_map(art_centres, ven_centres)
    dP = pressure_drops(uniforms)
    out = []
    for a in range(len(art_centres)):
        vs = [v for v in range(len(ven_centres)) if assign[v] == a]
        if not vs:
            continue
        f = velocity_factors(art_areas[a], [dP[v] for v in vs], [dist[v] for v in vs],
                             [ven_areas[v] for v in vs])
        for v, fv in zip(vs, f):
            out.append((a, v, dist[v], dP[v], fv))
    return out
