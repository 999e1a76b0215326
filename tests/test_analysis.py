"""Analysis helpers (Section 3.3), CPU only.

  * unit relations against the claims Section 3.3 makes about the numbers it
    prints (tests/golden/units_section33.txt): the aorta parameters lie at the
    cusp of the Mach bound (valid, but a factor 2 in speed or step breaks it);
    the coupled run's step follows from 1,000,000 steps = 100 s and its inlet
    speed is valid while a physiological 1 m/s would not be; and the round trip
    of the two relations;
  * velocity against vessel area: on a single steady tube fed by a parabolic
    inlet of peak U, mass conservation fixes the cross-section mean speed at
    the inlet profile's mean over the inlet's lattice points (U/2 in the
    continuum; 0.4805 U on the 81 points of a radius-5 disc); the moving-wall
    rule evaluates the profile at link mid-points, which loses ~2 % at the rim,
    so the bar is 4 % (the oracle supplies the flow field).
"""
import os

import numpy as np
import pytest

from paper_2010_04144_gb300 import analysis as A
from paper_2010_04144_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden", "units_section33.txt")


def _cases():
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            name, dx, dt, v, claim = line.split()
            yield name, float(dx), float(dt), float(v), claim


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_mach_claims_of_section_3_3(case):
    _, dx, dt, v, claim = case
    ma = lambda vv, tt: A.lattice_parameters(dx, tt, 4e-6, vv)[1]
    assert ma(v, dt) < 0.1                       # every printed run respects the bound
    if claim == "cusp":                          # "the cusp of achievable": twice the speed or
        assert ma(2 * v, dt) > 0.1               # twice the step leaves the valid range
        assert ma(v, 2 * dt) > 0.1
    else:                                        # valid only because the inlet was slowed down
        assert ma(1.0, dt) > 0.1


def test_coupled_run_step_from_printed_duration():
    steps, seconds = 1_000_000, 100.0            # Section 3.3: 1,000,000 steps = 100 s
    dt = {c[0]: c[2] for c in _cases()}["coupled"]
    assert abs(seconds / steps - dt) < 1e-18


def test_unit_round_trip():
    for dx, nu, tau in [(25e-6, 4e-6, 0.52), (75e-6, 3.5e-6, 0.8), (1e-3, 1e-6, 1.0)]:
        dt = A.physical_step(dx, nu, tau)
        t2, _ = A.lattice_parameters(dx, dt, nu, 1.0)
        assert abs(t2 - tau) < 1e-12
        assert abs(A.lattice_speed(dx / dt, dx, dt) - 1.0) < 1e-15
    with pytest.raises(ValueError):
        A.physical_step(1e-4, 1e-6, 0.5)


def test_mean_speed_of_steady_tube_is_half_the_peak(oracle_mod):
    U = 0.02
    geo = S.tree(S.TreeSpec(depth=1, root_radius=5.0, seed=11), inlet_speed=U,
                 pulse=S.PULSE_CONST)
    d = oracle_mod.Domain(geo.xyz, geo.iolets, tau=0.8)
    oracle_mod.System([d]).step(1500)
    rows = A.velocity_vs_area(geo, d.moments(), d.xyz)
    assert rows.shape[0] == 1
    _, area, speed, n = rows[0]
    x, y = np.meshgrid(np.arange(-5, 6), np.arange(-5, 6))
    r2 = (x ** 2 + y ** 2)[x ** 2 + y ** 2 <= 25]
    assert area == r2.size                                # the disc's lattice points
    expect = U * np.mean(1.0 - r2 / 25.0)
    assert abs(speed - expect) / expect < 0.04
    neg = A.velocity_vs_area(geo, d.moments(), d.xyz, arterial_negative=True)
    assert neg[0, 1] == -area


def test_hull_area_matches_a_library_hull():
    from scipy.spatial import ConvexHull

    rng = np.random.default_rng(5)
    for _ in range(20):
        P = rng.integers(-20, 20, size=(rng.integers(3, 60), 2))
        if np.linalg.matrix_rank(P - P[0]) < 2:
            continue
        assert abs(A._hull_area(P) - ConvexHull(P.astype(float)).volume) < 1e-9
    assert A._hull_area(np.array([[0, 0], [1, 1], [2, 2]])) == 0.0     # collinear


def test_plane_cuts_separate_vessels():
    g = S.parallel_tubes(3, radius=5, length=30)
    fields = np.zeros((g.n, 4))
    fields[:, 3] = 0.25
    rows = A.velocity_vs_area_planes(fields, g.xyz, axis=2)
    assert rows.shape[0] == 9                                  # 3 planes x 3 tubes
    x, y = np.meshgrid(np.arange(-5, 6), np.arange(-5, 6))
    disc = np.stack([x.ravel(), y.ravel()], 1)[(x ** 2 + y ** 2).ravel() <= 25]
    assert np.allclose(rows[:, 2], A._cell_hull_area(disc))    # each cut: one lattice disc
    from scipy.spatial import ConvexHull

    corners = np.concatenate([disc + d for d in ((-.5, -.5), (-.5, .5), (.5, -.5), (.5, .5))])
    assert abs(A._cell_hull_area(disc) - ConvexHull(corners).volume) < 1e-9
    assert A._cell_hull_area(disc) >= disc.shape[0] > A._hull_area(disc)
    assert np.allclose(rows[:, 3], 0.25) and np.all(rows[:, 4] == disc.shape[0])
    neg = A.velocity_vs_area_planes(fields, g.xyz, axis=2, arterial_negative=True)
    assert np.allclose(neg[:, 2], -rows[:, 2])
    t = S.tree(S.TreeSpec(depth=4, root_radius=5, seed=7))
    rt = A.velocity_vs_area_planes(np.ones((t.n, 4)), t.xyz)
    ax = int(np.argmax(t.xyz.max(0) - t.xyz.min(0)))
    for f in (0.25, 0.5, 0.75):
        level = int(round(t.xyz[:, ax].min() + f * (t.xyz[:, ax].max() - t.xyz[:, ax].min())))
        assert rt[rt[:, 0] == f, 4].sum() == np.sum(t.xyz[:, ax] == level)   # every site in a vessel


def test_thin_vessels_have_consistent_areas():
    """A vessel one site wide has the area of its sites, whatever their number; a square
    block of sites has its full area; no cut yields a zero area."""
    for k in range(1, 8):
        line = np.stack([np.arange(k), np.zeros(k, int)], 1)
        assert A._cell_hull_area(line) == float(k)
        assert A._cell_hull_area(line[:, ::-1]) == float(k)
    block = np.stack(np.meshgrid(np.arange(3), np.arange(3)), -1).reshape(-1, 2)
    assert A._cell_hull_area(block) == 9.0
    # a plane cut through a one-voxel-wide straight vessel next to a wide one
    thin = np.stack([np.full(6, 3), np.full(6, 3), np.arange(6)], 1)
    wide = S.cylinder(radius=3, length=6, margin=10).xyz
    xyz = np.concatenate([thin, wide]).astype(np.int32)
    rows = A.velocity_vs_area_planes(np.ones((xyz.shape[0], 4)), xyz, axis=2)
    assert np.all(rows[:, 2] > 0)
    assert sorted(set(rows[:, 4].astype(int))) == [1, 29]
