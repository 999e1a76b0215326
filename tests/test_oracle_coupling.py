"""Pins of the coupling map and scale factors (Section 3), CPU only."""
import math
import os

import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "coupling_1to3.txt")


def _golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return [(float(r[1]), float(r[2]), float(r[3])) for r in rows]


def test_paper_1to3_example():
    from oracle import coupling as CP

    rows = _golden()
    dP = [r[0] for r in rows]
    printed = [r[1] for r in rows]
    L = [r[2] for r in rows]
    f = CP.velocity_factors(1.0, dP, L, [1.0, 1.0, 1.0])
    assert [round(x, 2) for x in f] == printed
    assert abs(sum(f) - 1.0) < 1e-15


def test_single_inlet_is_area_ratio():
    from oracle import coupling as CP

    for A0, A1 in [(1.0, 1.0), (2.0, 3.0), (math.pi * 8 ** 2, math.pi * 9.6 ** 2)]:
        f = CP.velocity_factors(A0, [0.42], [17.0], [A1])
        assert abs(f[0] - A0 / A1) < 1e-15 * (A0 / A1)


def test_equal_inlets_split_evenly():
    from oracle import coupling as CP

    for N in (2, 3, 7, 13):
        f = CP.velocity_factors(1.0, [0.5] * N, [10.0] * N, [1.0] * N)
        assert np.allclose(f, 1.0 / N, rtol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_mass_conservation_of_factors(seed):
    """sum_i A_i v_i = A_0 v_0 (q_0 = sum q_i) and factor ratios follow dP_i A_i / L_i."""
    from oracle import coupling as CP

    g = np.random.default_rng(seed)
    N = int(g.integers(1, 14))
    dP = list(CP.pressure_drops(g.random(N)))
    L = list(1 + 50 * g.random(N))
    A = list(1 + 100 * g.random(N))
    A0 = float(1 + 100 * g.random())
    f = CP.velocity_factors(A0, dP, L, A)
    assert abs(sum(a * x for a, x in zip(A, f)) - A0) < 1e-12 * A0
    for i in range(N):
        assert 0.3 <= dP[i] <= 0.7
        # q_i / q_j = (dP_i A_i / L_i) / (dP_j A_j / L_j)
        qi, q0 = A[i] * f[i], A[0] * f[0]
        assert abs(qi / q0 - (dP[i] * A[i] / L[i]) / (dP[0] * A[0] / L[0])) < 1e-12 * qi / q0
    # invariance under a common scaling of distances and areas
    f2 = CP.velocity_factors(A0 * 4, dP, [3 * l for l in L], [4 * a for a in A])
    assert np.allclose(f, f2, rtol=1e-13)


def _c(x, y, z):
    return (int(x * 1024), int(y * 1024), int(z * 1024))


def test_greedy_map_by_hand():
    from oracle import coupling as CP

    art = [_c(0, 0, 0), _c(10, 0, 0)]
    ven = [_c(9, 0, 0), _c(1, 0, 0), _c(2, 0, 0), _c(12, 0, 0), _c(30, 0, 0)]
    assign, dist = CP.greedy_map(art, ven)
    # artery 0 takes vein 1 (d=1); artery 1 takes vein 0 (d=1); then veins 2, 3, 4
    # join their closest artery: 2 -> 0 (d=2), 3 -> 1 (d=2), 4 -> 1 (d=20)
    assert assign == [1, 0, 0, 1, 1]
    assert dist == [1.0, 1.0, 2.0, 2.0, 20.0]


def test_greedy_map_ties_and_more_arteries():
    from oracle import coupling as CP

    art = [_c(0, 0, 0), _c(4, 0, 0)]
    ven = [_c(2, 0, 0), _c(-2, 0, 0)]          # vein 0 equidistant from both arteries
    assign, _ = CP.greedy_map(art, ven)
    assert assign == [0, 1]                    # artery 0 first: tie on distance -> vein 0
    art = [_c(0, 0, 0), _c(5, 0, 0), _c(9, 0, 0)]
    ven = [_c(6, 0, 0)]
    assign, _ = CP.greedy_map(art, ven)        # fewer veins than arteries
    assert assign == [0]
    ven = [_c(2, 0, 0), _c(2, 0, 0)]           # identical veins: lowest index first
    assign, _ = CP.greedy_map([_c(0, 0, 0), _c(0, 0, 0)], ven)
    assert assign == [0, 1]
    ven = [_c(0, 3, 0), _c(0, 0, 3)]
    assign, _ = CP.greedy_map([_c(0, 0, 0)], ven)
    assert assign == [0, 0]                    # 1:N map, every vein covered


def test_every_artery_gets_a_vein():
    from oracle import coupling as CP

    g = np.random.default_rng(9)
    art = [_c(*(g.random(3) * 100)) for _ in range(5)]
    ven = [_c(*(g.random(3) * 100)) for _ in range(65)]    # 13x more venous inlets
    assign, dist = CP.greedy_map(art, ven)
    assert set(assign) == set(range(5))
    table = CP.coupling_table(art, [1.0] * 5, ven, [1.0] * 65, g.random(65))
    for a in range(5):
        fs = [r[4] for r in table if r[0] == a]
        assert abs(sum(fs) - 1.0) < 1e-12


def test_coupled_1to3_simulation(oracle_mod):
    """One tube feeding three (equal sizes): coupled inlets follow the factors.

    The venous inlet values are factor x arterial-outlet mean of the previous
    step (exactly); the measured venous means, over the sites next to each
    inlet, are proportional to the factors (common geometric factor).
    """
    from oracle import coupling as CP

    rows = _golden()
    f = CP.velocity_factors(1.0, [r[0] for r in rows], [r[2] for r in rows], [1.0] * 3)
    art = S.cylinder(radius=6, length=48, inlet=dict(kind=S.PRESSURE, value=0.001))
    ven = S.parallel_tubes(3, radius=6, length=48,
                           inlet=dict(kind=S.VELOCITY, value=0.0, profile=S.PLUG))
    da = oracle_mod.Domain(art.xyz, art.iolets)
    dv = oracle_mod.Domain(ven.xyz, ven.iolets)
    s = oracle_mod.System([da, dv], [(0, 1, 1, j, f[j]) for j in range(3)])
    s.step(3000)
    ua = s.M[0][1][0]
    assert ua > 0
    bc = s.bc_values(1, s.t + 1)
    for j in range(3):
        assert bc[j] == f[j] * ua
    meas = np.array([-s.M[1][j][0] / ua for j in range(3)])
    ratio = meas / np.array(f)
    assert np.ptp(ratio) < 0.005 * ratio.mean()
    assert 0.85 < ratio.mean() <= 1.0
