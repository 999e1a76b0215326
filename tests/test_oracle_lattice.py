"""Pins of the oracle's lattice, equilibrium and site ordering (CPU only).

The paper names the D3Q19 lattice and single-relaxation-time collision
(Section 2) but prints no table; these tests pin the oracle's tables against
the mathematical facts any D3Q19/LBGK implementation must satisfy.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest


def _frac_w(w):
    f = [Fraction(x).limit_denominator(100) for x in w]
    assert all(abs(float(a) - b) < 1e-16 for a, b in zip(f, w))
    return f


def test_velocity_set_is_d3q19(oracle_mod):
    c, w, opp = oracle_mod.lattice()
    vs = {tuple(v) for v in c}
    expect = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in v) <= 2}
    assert vs == expect and len(vs) == 19
    assert tuple(c[0]) == (0, 0, 0)
    # axis directions first, then diagonals (reading R1)
    assert all(np.abs(c[i]).sum() == 1 for i in range(1, 7))
    assert all(np.abs(c[i]).sum() == 2 for i in range(7, 19))


def test_opposites(oracle_mod):
    c, w, opp = oracle_mod.lattice()
    for i in range(19):
        assert np.array_equal(c[opp[i]], -c[i])
        assert opp[opp[i]] == i
    # opposite pairs are adjacent: (1,2), (3,4), ...
    for i in range(1, 19, 2):
        assert opp[i] == i + 1


def test_weight_moments_exact(oracle_mod):
    c, w, opp = oracle_mod.lattice()
    W = _frac_w(w)
    assert sum(W) == 1
    for a in range(3):
        assert sum(W[i] * c[i, a] for i in range(19)) == 0
        for b in range(3):
            m2 = sum(W[i] * c[i, a] * c[i, b] for i in range(19))
            assert m2 == (Fraction(1, 3) if a == b else 0)
            for g in range(3):
                assert sum(W[i] * c[i, a] * c[i, b] * c[i, g] for i in range(19)) == 0
                for d in range(3):
                    m4 = sum(W[i] * c[i, a] * c[i, b] * c[i, g] * c[i, d] for i in range(19))
                    iso = Fraction(int(a == b and g == d) + int(a == g and b == d)
                                   + int(a == d and b == g), 9)
                    assert m4 == iso


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(oracle_mod, seed):
    """Deviation-form equilibrium: mass drho, momentum rho u, momentum flux drho/3 I + rho u u."""
    c, w, opp = oracle_mod.lattice()
    g = np.random.default_rng(seed)
    drho = 1e-2 * (2 * g.random() - 1)
    u = 0.05 * (2 * g.random(3) - 1)
    fe = oracle_mod.feq(drho, u)
    rho = 1 + drho
    assert abs(fe.sum() - drho) < 1e-15
    np.testing.assert_allclose(c.T @ fe, rho * u, atol=1e-16, rtol=1e-13)
    pi = np.einsum("i,ia,ib->ab", fe, c, c)
    np.testing.assert_allclose(pi, drho / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-16,
                               rtol=1e-12)
    # rest: all zeros
    assert np.all(oracle_mod.feq(0.0, [0, 0, 0]) == 0.0)


def _interleave(x, y, z):
    bits = []
    for b in range(20, -1, -1):
        bits += [(z >> b) & 1, (y >> b) & 1, (x >> b) & 1]
    return int("".join(str(v) for v in bits), 2)


def test_morton_key(oracle_mod):
    assert oracle_mod.morton(1, 0, 0) == 1
    assert oracle_mod.morton(0, 1, 0) == 2
    assert oracle_mod.morton(0, 0, 1) == 4
    assert oracle_mod.morton(2, 0, 0) == 8
    g = np.random.default_rng(5)
    for _ in range(200):
        x, y, z = (int(v) for v in g.integers(0, 1 << 21, 3))
        assert oracle_mod.morton(x, y, z) == _interleave(x, y, z)


def test_canonical_order_blocks(oracle_mod):
    """Ascending Morton order visits every aligned 8^3 block contiguously (Section 2.2 blocks)."""
    from paper_2010_04144_gb300 import synth

    geo = synth.tree(synth.TreeSpec(depth=3, root_radius=5, seed=3))
    d = oracle_mod.Domain(geo.xyz, geo.iolets, with_nbr=False)
    keys = d.keys.astype(np.uint64)
    assert np.all(np.diff(keys.astype(np.float64)) > 0) or np.all(keys[1:] > keys[:-1])
    blk = [tuple(v) for v in (d.xyz // 8)]
    seen, last = set(), None
    for b in blk:
        if b != last:
            assert b not in seen
            seen.add(b)
            last = b
    # perm maps canonical sites back to the input list
    assert np.array_equal(geo.xyz[d.perm], d.xyz)
