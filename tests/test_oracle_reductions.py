"""Brute-force pins of the oracle's reductions: moments, iolet means, mass (CPU only)."""
import numpy as np

from paper_2010_04144_gb300 import synth as S


def test_moments_bruteforce(oracle_mod):
    c, w, opp = oracle_mod.lattice()
    F = S.random_state(40, seed=1, amplitude=1e-2)
    d = oracle_mod.Domain(S.box(4, 5, 2).xyz, [])
    m = d.moments(F)
    for s in range(40):
        f = F[:, s]
        drho = sum(f[i] for i in range(19))
        j = [sum(c[i][a] * f[i] for i in range(19)) for a in range(3)]
        assert abs(m[s, 0] - drho) < 1e-16
        for a in range(3):
            assert abs(m[s, 1 + a] - j[a] / (1 + drho)) < 1e-15


def test_iolet_means_bruteforce(oracle_mod):
    geo = S.tree(S.TreeSpec(depth=3, root_radius=4, seed=2))
    d = oracle_mod.Domain(geo.xyz, geo.iolets)
    g = np.random.default_rng(0)
    mom = g.normal(size=(d.n, 4))
    out = d.iolet_means(mom)
    for k, io in enumerate(geo.iolets):
        adj = [s for s in range(d.n) if any(d.nbr[i, s] == -(2 + k) for i in range(18))]
        nh = np.array(io.axis, float) / np.linalg.norm(io.axis)
        assert out[k, 2] == len(adj)
        assert len(adj) > 0
        un = [mom[s, 1:] @ nh for s in adj]
        assert abs(out[k, 0] - np.mean(un)) < 1e-12
        assert abs(out[k, 1] - np.mean(mom[adj, 0])) < 1e-12
    # an iolet nobody touches reports zeros
    far = list(geo.iolets) + [S.Iolet(kind=S.PRESSURE, centre=(10 ** 6, 0, 0),
                                      axis=(1024, 0, 0), radius=1024)]
    d2 = oracle_mod.Domain(geo.xyz, far)
    assert np.all(d2.iolet_means(mom)[-1] == 0.0)


def test_mass_bruteforce(oracle_mod):
    F = S.random_state(33, seed=4)
    d = oracle_mod.Domain(S.box(3, 11, 1).xyz, [])
    assert abs(d.mass(F) - float(np.sum(F))) < 1e-15


def test_step_sites_equals_step(oracle_mod):
    geo = S.tree(S.TreeSpec(depth=3, root_radius=4, seed=2))
    d = oracle_mod.Domain(geo.xyz, geo.iolets)
    F = S.random_state(d.n, seed=8, amplitude=1e-3)
    bc = np.array([0.01] + [0.0005] * (len(geo.iolets) - 1))
    Fo = np.zeros_like(F)
    mom = np.zeros((d.n, 4))
    d.step_into(F, Fo, bc, mom)
    sites = np.arange(0, d.n, 7)
    out, mo = d.step_sites(F, bc, sites)
    assert np.array_equal(out, Fo[:, sites].T)
    assert np.array_equal(mo, mom[sites])
