"""Physics pins of the FP64 oracle (CPU only).

Each test checks the oracle against something the mathematics or the paper
fixes, not against itself:
  * rest state: f~ = 0 is an exact fixed point (deviation storage, reading R4);
  * mass: a closed box conserves total mass to round-off (LBGK collision
    conserves mass, bounce-back walls return every population);
  * Poiseuille: steady tube flow driven by a density difference matches the
    analytic parabola u = G (R^2 - r^2) / (4 nu), G = drho / (3 L),
    nu = (tau - 1/2) / 3 (the viscosity relation quoted in Section 3.3);
  * Womersley: oscillating pressure drop, complex velocity amplitude against
    the Bessel-function solution;
  * velocity inlet: steady mass flux through every interior plane equals the
    mass the moving-wall rule injects, sum over inlet links of 6 w_i c_i.u_w;
  * axis symmetry: the same tube along x and along z gives the same fields.
"""
import math

import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

TAU = 0.8
NU = (TAU - 0.5) / 3.0


def test_rest_state_exact(oracle_mod):
    geo = S.tree(S.TreeSpec(depth=3, root_radius=4, seed=5), inlet_speed=0.0)
    d = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    s = oracle_mod.System([d])
    s.step(300)
    assert np.all(d.F == 0.0)
    assert np.all(d.mom == 0.0)


def test_mass_conserved_closed_box(oracle_mod):
    geo = S.box(9, 7, 6)
    d = oracle_mod.Domain(geo.xyz, [], tau=TAU)
    d.F[:] = S.random_state(d.n, seed=3, amplitude=1e-3)
    m0 = d.mass()
    s = oracle_mod.System([d])
    drift = []
    s.step(1000, lambda st: drift.append(d.mass() - m0))
    scale = np.abs(d.F).sum()
    assert max(abs(x) for x in drift) <= 1e-13 * d.n * 19 * 1e-3
    assert abs(d.mass() - m0) <= 1e-12 * max(scale, 1e-3)
    assert not np.all(d.F == 0.0)


def _poiseuille(oracle_mod, R=8, L=64, drho=0.001, steps=2000):
    geo = S.cylinder(radius=R, length=L, inlet=dict(kind=S.PRESSURE, value=drho))
    d = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    s = oracle_mod.System([d])
    s.step(steps)
    return geo, d, d.moments()


@pytest.fixture(scope="module")
def poiseuille(oracle_mod):
    return _poiseuille(oracle_mod)


def test_poiseuille_profile(poiseuille):
    geo, d, m = poiseuille
    R, L, c, mg = geo.meta["radius"], geo.meta["length"], geo.meta["centre"], geo.meta["margin"]
    z = d.xyz[:, 2]
    mid = (z >= mg + L // 4) & (z < mg + 3 * L // 4)
    r2 = ((d.xyz[mid, 0] - c) ** 2 + (d.xyz[mid, 1] - c) ** 2).astype(np.float64)
    uz = m[mid, 3]
    G = 0.001 / (3.0 * L)
    # fitted parabola u = a - b r^2: b = G / (4 nu), R_eff^2 = a / b
    A = np.stack([np.ones_like(r2), -r2], 1)
    a, b = np.linalg.lstsq(A, uz, rcond=None)[0]
    G_fit = 4 * NU * b
    R_eff = math.sqrt(a / b)
    assert abs(G_fit - G) / G < 0.03
    assert abs(R_eff - R) < 0.5
    # analytic profile with the radius of the staircase cross-section's area
    n_cross = int(np.sum(z == mg))
    R_area = math.sqrt(n_cross / math.pi)
    ua = G * (R_area ** 2 - r2) / (4 * NU)
    assert np.linalg.norm(uz - ua) / np.linalg.norm(ua) < 0.06
    # no transverse flow, positive axial flow everywhere
    assert np.max(np.abs(m[mid, 1:3])) < 1e-3 * np.max(uz)
    assert np.all(uz > 0)


def test_poiseuille_pressure_drop(poiseuille):
    geo, d, m = poiseuille
    L, mg = geo.meta["length"], geo.meta["margin"]
    z = d.xyz[:, 2]
    # density deviation falls linearly from the inlet value to the outlet value
    zs = np.arange(mg + 4, mg + L - 4)
    prof = np.array([m[z == zz, 0].mean() for zz in zs])
    slope = np.polyfit(zs, prof, 1)[0]
    assert abs(slope - (-0.001 / L)) / (0.001 / L) < 0.03
    mid = m[z == mg + L // 2, 0].mean()
    assert abs(mid - 0.0005) < 0.05 * 0.0005


def _j0(zz, terms=60):
    s, term = 0j, 1 + 0j
    for k in range(terms):
        if k:
            term *= -(zz * zz / 4) / (k * k)
        s += term
    return s


def test_womersley(oracle_mod):
    """Complex velocity amplitude over the last period vs the Womersley solution.

    The driving gradient amplitude is measured between two planes around the
    central cross-section, so the test does not depend on the acoustic
    response of the short tube.
    """
    T = 1000.0
    geo = S.cylinder(inlet=dict(kind=S.PRESSURE, value=0.001, pulse=S.PULSE_SINE, period=T))
    d = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    s = oracle_mod.System([d])
    c, mg, R = geo.meta["centre"], geo.meta["margin"], geo.meta["radius"]
    z = d.xyz[:, 2]
    zc = mg + 32
    sec = z == zc
    r = np.sqrt((d.xyz[sec, 0] - c) ** 2 + (d.xyz[sec, 1] - c) ** 2)
    p1, p2 = z == zc - 8, z == zc + 8
    w = 2 * math.pi / T
    acc = {"U": np.zeros(int(sec.sum()), complex), "G": 0j}

    def cb(st):
        if st.t > 3 * T:
            e = np.exp(-1j * w * st.t) * 2 / T
            acc["G"] += (d.mom[p1, 0].mean() - d.mom[p2, 0].mean()) / 3.0 / 16.0 * e
            acc["U"] += d.mom[sec, 3] * e

    s.step(int(4 * T), cb)
    Gh, U = acc["G"], acc["U"]
    # the measured gradient oscillates with the imposed amplitude drho / (3 L), to within 10%
    assert abs(abs(Gh) - 0.001 / (3 * 64)) / (0.001 / (3 * 64)) < 0.1
    R_area = math.sqrt(sec.sum() / math.pi)
    alpha = R_area * math.sqrt(w / NU)
    assert 1.9 < alpha < 2.1
    k = (1j) ** 1.5 * alpha
    Ua = (Gh / (1j * w)) * (1 - np.array([_j0(k * ri / R_area) for ri in r]) / _j0(k))
    assert np.linalg.norm(U - Ua) / np.linalg.norm(Ua) < 0.08
    # the centreline lags the gradient by more than the quasi-steady (zero) phase
    lag = np.angle(Gh) - np.angle(U[np.argmin(r)])
    lag_a = np.angle(Gh) - np.angle(Ua[np.argmin(r)])
    assert abs(((lag - lag_a + math.pi) % (2 * math.pi)) - math.pi) < 0.1


@pytest.mark.parametrize("profile", [S.PLUG, S.PARABOLIC])
def test_velocity_inlet_flux_balance(oracle_mod, profile):
    R, L, U = 5, 30, 0.01
    geo = S.cylinder(radius=R, length=L, inlet=dict(kind=S.VELOCITY, value=U, profile=profile))
    d = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    s = oracle_mod.System([d])
    s.step(3000)
    c, w, opp = oracle_mod.lattice()
    key = {tuple(p): i for i, p in enumerate(d.xyz)}

    def plane_flux(zp):
        tot = 0.0
        for i in range(19):
            if c[i, 2] == 0:
                continue
            layer = zp if c[i, 2] > 0 else zp + 1
            for sidx in np.nonzero(d.xyz[:, 2] == layer)[0]:
                if tuple(d.xyz[sidx] + c[i]) in key:
                    tot += c[i, 2] * d.F[i, sidx]
        return tot

    io = geo.iolets[0]
    ctr = np.array(io.centre) / 1024.0
    ah = np.array(io.axis, float) / np.linalg.norm(io.axis)
    inj = 0.0
    for i in range(1, 19):
        for sidx in np.nonzero(d.nbr[i - 1] == -2)[0]:
            mpt = d.xyz[sidx] - 0.5 * c[i] - ctr
            perp = mpt - mpt.dot(ah) * ah
            phi = 1.0 if profile == S.PLUG else max(0.0, 1 - perp.dot(perp) / R ** 2)
            inj += 6 * w[i] * c[i].dot(-ah * U * phi)
    assert inj > 0
    for zp in (6, 16, 26):
        assert abs(plane_flux(zp) - inj) / inj < 1e-4


def test_axis_symmetry(oracle_mod):
    gz = S.cylinder(radius=4, length=20, axis=2)
    gx = S.cylinder(radius=4, length=20, axis=0)
    dz = oracle_mod.Domain(gz.xyz, gz.iolets, tau=TAU)
    dx = oracle_mod.Domain(gx.xyz, gx.iolets, tau=TAU)
    sz, sx = oracle_mod.System([dz]), oracle_mod.System([dx])
    sz.step(200)
    sx.step(200)
    mz, mx = dz.moments(), dx.moments()
    # map x-tube coordinates (a, b, c) -> z-tube coordinates (c, b, a)
    kz = {tuple(p): i for i, p in enumerate(dz.xyz)}
    idx = np.array([kz[(p[2], p[1], p[0])] for p in dx.xyz])
    np.testing.assert_allclose(mx[:, 0], mz[idx, 0], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(mx[:, 1], mz[idx, 3], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(mx[:, 2], mz[idx, 2], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(mx[:, 3], mz[idx, 1], rtol=1e-9, atol=1e-15)
    assert np.max(np.abs(mx[:, 1])) > 1e-5
