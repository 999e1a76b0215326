"""Pins of the oracle's body-force collision (reading R7: Guo, Zheng and Shi
forcing, named by Section 3 for the reverse coupling direction), CPU only.

  * conservation: the forced collision keeps the mass and raises the momentum
    by exactly the force density (what makes the scheme first-order exact);
  * zero force: bit-identical to the unforced update;
  * hydrostatics: a closed box under a uniform force settles at rest with the
    density gradient of an ideal gas of sound speed 1/sqrt(3), d(drho)/dz = 3 g;
  * body-force Poiseuille: a tube with both ends at the same pressure, driven by
    a uniform axial force density G, carries u = G (R^2 - r^2) / (4 nu);
  * reverse exchange: forces appear only after odd exchanges and only at the
    sites next to the forced outlet, and the alternation holds each direction's
    values (the mapping itself is a reading: parity unpinned).
"""
import math

import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

TAU = 0.8
NU = (TAU - 0.5) / 3.0


def _lattice(oracle_mod):
    c, w, _ = oracle_mod.lattice()
    return c.astype(np.float64), w


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_forced_collision_conserves_mass_adds_force(oracle_mod, seed):
    c, w = _lattice(oracle_mod)
    rng = np.random.default_rng(seed)
    g = rng.uniform(-1e-2, 1e-2, 19) * w * 18
    F = rng.uniform(-1e-3, 1e-3, 3)
    for tau in (0.55, 0.8, 1.7):
        out, mom = oracle_mod.collide(g, tau, F)
        assert abs(out.sum() - g.sum()) <= 1e-16
        j_in, j_out = c.T @ g, c.T @ out
        np.testing.assert_allclose(j_out - j_in, F, rtol=0, atol=2e-17)
        # the reported velocity is the momentum average over the step, (j + F/2) / rho
        rho = 1.0 + g.sum()
        np.testing.assert_allclose(mom[1:] * rho, 0.5 * (j_in + j_out), rtol=0, atol=1e-17)
        out0, _ = oracle_mod.collide(g, tau)
        assert np.abs(out - out0).max() > 0


def test_zero_force_is_bitwise_unforced(oracle_mod):
    geo = S.tree(S.TreeSpec(depth=3, root_radius=4, seed=5), inlet_speed=0.04, period=50.0)
    a = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    b = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    a.F[:] = b.F[:] = S.random_state(a.n, seed=9, amplitude=1e-3)
    bc = [io.value for io in geo.iolets]
    outa, outb = np.zeros_like(a.F), np.zeros_like(b.F)
    a.step_into(a.F, outa, bc, a.mom)
    b.step_into(b.F, outb, bc, b.mom, np.zeros((b.n, 3)))
    assert np.array_equal(outa, outb) and np.array_equal(a.mom, b.mom)
    g = np.linspace(-1e-3, 1e-3, 19)
    x, mx = oracle_mod.collide(g, TAU)
    y, my = oracle_mod.collide(g, TAU, np.zeros(3))
    assert np.array_equal(x, y) and np.array_equal(mx, my)


def test_hydrostatic_box(oracle_mod):
    nz, g0 = 12, 2e-5
    geo = S.box(6, 6, nz)
    d = oracle_mod.Domain(geo.xyz, [], tau=TAU)
    force = np.tile([0.0, 0.0, g0], (d.n, 1))
    out = np.zeros_like(d.F)
    for _ in range(2500):
        d.step_into(d.F, out, [], d.mom, force)
        d.F, out = out, d.F
    m = d.mom
    z = d.xyz[:, 2].astype(np.float64)
    slope, _ = np.polyfit(z, m[:, 0], 1)
    assert abs(slope - 3.0 * g0) / (3.0 * g0) < 0.01
    assert np.abs(m[:, 1:]).max() < 1e-3 * g0 * nz      # at rest
    assert abs(d.mass()) < 1e-15 * d.n                    # mass stays zero


def test_body_force_poiseuille(oracle_mod):
    R, L, G = 8, 48, 4e-6
    geo = S.cylinder(radius=R, length=L, inlet=dict(kind=S.PRESSURE, value=0.0))
    d = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    force = np.tile([0.0, 0.0, G], (d.n, 1))
    out = np.zeros_like(d.F)
    for _ in range(1500):
        d.step_into(d.F, out, [0.0] * len(geo.iolets), d.mom, force)
        d.F, out = out, d.F
    c, mg = geo.meta["centre"], geo.meta["margin"]
    z = d.xyz[:, 2]
    mid = (z >= mg + L // 4) & (z < mg + 3 * L // 4)
    r2 = ((d.xyz[mid, 0] - c) ** 2 + (d.xyz[mid, 1] - c) ** 2).astype(np.float64)
    uz = d.mom[mid, 3]
    A = np.stack([np.ones_like(r2), -r2], 1)
    a, b = np.linalg.lstsq(A, uz, rcond=None)[0]
    assert abs(4 * NU * b - G) / G < 0.03
    assert abs(math.sqrt(a / b) - R) < 0.5


def _coupled_pair(oracle_mod, alternate):
    art = S.cylinder(radius=4, length=24, inlet=dict(kind=S.VELOCITY, value=0.02, profile=S.PARABOLIC,
                                                     pulse=S.PULSE_CONST))
    ven = S.cylinder(radius=4, length=24, inlet=dict(kind=S.VELOCITY, value=0.0, profile=S.PLUG))
    da = oracle_mod.Domain(art.xyz, art.iolets, tau=TAU)
    dv = oracle_mod.Domain(ven.xyz, ven.iolets, tau=TAU)
    return oracle_mod.System([da, dv], [(0, 1, 1, 0, 0.8)], alternate=alternate), da, dv


def test_reverse_exchange_schedule_and_sites(oracle_mod):
    sf, _, _ = _coupled_pair(oracle_mod, alternate=False)
    sa, da, _ = _coupled_pair(oracle_mod, alternate=True)
    sf.step(120)          # flow reaches the outlet and the coupled venous inlet
    sa.step(120)
    seen = []
    for t in range(121, 129):
        sf.step(1)
        sa.step(1)
        assert sa.t == t
        f = sa.iolet_force[0][1]
        seen.append(np.abs(f).sum() > 0)
        if t % 2 == 1:          # a reverse exchange just ran: the force follows the venous inflow
            vin = -sa.M[1][0][0]
            v = vin / 0.8
            ax = np.array(sa.domains[0].iolets[1].axis, float)
            np.testing.assert_allclose(f, -0.5 * v * abs(v) * ax / np.linalg.norm(ax), rtol=1e-15)
        else:                   # a forward exchange: the venous inlet follows the arterial outlet
            assert sa.cbv[(1, 0)] == 0.8 * sa.M[0][1][0]
        assert not np.any(sf.iolet_force[0])      # forward-only mode never forces
    assert all(seen)
    F = sa.site_force(0)
    forced = np.nonzero(np.abs(F).sum(1))[0]
    assert np.array_equal(forced, da.adjacent(1))
    assert sa.site_force(1) is None


# ---- reverse-exchange mapping (reading 13), pinned on the properties the reading fixes:
# the outlet force is the dynamic pressure 1/2 v|v| of the speed the fed venous inlets map
# back to, directed against the outlet's outward axis for inflow, averaged (not summed) over
# the inlets an outlet feeds, with each inlet's factor undone.

def _fan_system(oracle_mod, factors):
    """Arterial tube (outlet = iolet 1, outward +z) feeding len(factors) venous tube inlets."""
    art = S.cylinder(radius=3, length=12, inlet=dict(kind=S.VELOCITY, value=0.01, profile=S.PLUG))
    ven = S.parallel_tubes(len(factors), radius=3, length=12,
                           inlet=dict(kind=S.VELOCITY, value=0.0, profile=S.PLUG))
    da = oracle_mod.Domain(art.xyz, art.iolets, tau=TAU)
    dv = oracle_mod.Domain(ven.xyz, ven.iolets, tau=TAU)
    pairs = [(0, 1, 1, j, f) for j, f in enumerate(factors)]
    return oracle_mod.System([da, dv], pairs, alternate=True)


def _reverse(sysm, inlet_means):
    """Reverse exchange (odd e) with the venous inlets' mean u.n set to `inlet_means`."""
    for j, m in enumerate(inlet_means):
        sysm.M[1][j][0] = m
    sysm._exchange(1)
    return np.array(sysm.iolet_force[0][1])


def test_reverse_zero_inflow_gives_zero_force(oracle_mod):
    s = _fan_system(oracle_mod, [0.6, 0.9])
    assert np.array_equal(_reverse(s, [0.0, 0.0]), np.zeros(3))


def test_reverse_force_opposes_outflow(oracle_mod):
    s = _fan_system(oracle_mod, [0.7])
    n = np.array([0.0, 0.0, 1.0])                 # the arterial outlet's outward axis
    F = _reverse(s, [-0.01])                        # inflow at the venous inlet (u.n < 0)
    assert F @ n < 0 and np.allclose(np.cross(F, n), 0.0, atol=0)
    F = _reverse(s, [+0.01])                        # backflow out of the venous inlet
    assert F @ n > 0


def test_reverse_force_quadratic_in_speed(oracle_mod):
    s = _fan_system(oracle_mod, [0.45])
    F1 = _reverse(s, [-0.004])
    F2 = _reverse(s, [-0.008])
    assert abs(np.linalg.norm(F2) / np.linalg.norm(F1) - 4.0) < 1e-14


def test_reverse_mean_over_fed_inlets(oracle_mod):
    one = _reverse(_fan_system(oracle_mod, [0.5]), [-0.006])
    three = _reverse(_fan_system(oracle_mod, [0.5, 0.5, 0.5]), [-0.006, -0.006, -0.006])
    np.testing.assert_allclose(three, one, rtol=1e-15, atol=0)
    assert np.linalg.norm(one) > 0


def test_forward_then_reverse_round_trip(oracle_mod):
    """A steady 1:1 pair whose venous inlet carries exactly the imposed inflow maps back to
    the arterial outlet mean: the reverse direction undoes the forward factor."""
    f, m = 0.37, 0.0123
    s = _fan_system(oracle_mod, [f])
    s.M[0][1][0] = m                               # arterial outlet mean u.n (outflow)
    s._exchange(0)                                 # forward: venous inlet speed f * m
    imposed = s.cbv[(1, 0)]
    assert imposed == f * m
    F = _reverse(s, [-imposed])                    # the inlet's mean u.n is the imposed inflow
    v = math.sqrt(2.0 * np.linalg.norm(F))
    assert abs(v - m) <= 1e-15 * m
    assert F[2] < 0
