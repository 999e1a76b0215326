"""Pins of the oracle's neighbour table and iolet classification (CPU only).

Neighbour table: brute force over a coordinate dictionary on tiny geometries.
Iolet classification (reading R3 of the oracle; the paper only says vessel
tips are cut flat and perpendicular, Section 3.1): hand-placed points whose
answer is known.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S


def _brute_nbr(oracle_mod, xyz, iolets):
    c, w, opp = oracle_mod.lattice()
    key = {tuple(p): i for i, p in enumerate(xyz)}
    n = len(xyz)
    out = np.zeros((18, n), np.int32)
    for s in range(n):
        for i in range(1, 19):
            q = tuple(int(v) for v in xyz[s] - c[i])
            if q in key:
                out[i - 1, s] = key[q]
            else:
                out[i - 1, s] = oracle_mod.classify(q, iolets)
    return out


def _geoms():
    yield "box3", S.box(3, 3, 3), 0
    yield "voxel", S.Geometry(xyz=np.array([[5, 5, 5]], np.int32), iolets=[]), 0
    lb = [[2 + i, 2, 2] for i in range(5)] + [[6, 2 + j, 2] for j in range(1, 5)]
    yield "Lbend", S.Geometry(xyz=np.array(lb, np.int32), iolets=[]), 0
    # a single voxel touching two iolets (one below, one above)
    two = [S.Iolet(kind=S.PRESSURE, centre=(5120, 5120, 4608), axis=(0, 0, -1024), radius=1024),
           S.Iolet(kind=S.VELOCITY, centre=(5120, 5120, 5632), axis=(0, 0, 1024), radius=1024)]
    yield "twoiolets", S.Geometry(xyz=np.array([[5, 5, 5]], np.int32), iolets=two), 2
    yield "tube", S.cylinder(radius=3, length=6), 2
    yield "tree", S.tree(S.TreeSpec(depth=3, root_radius=3.5, seed=11)), 5


@pytest.mark.parametrize("name,geo,nio", list(_geoms()), ids=[g[0] for g in _geoms()])
def test_nbr_bruteforce(oracle_mod, name, geo, nio):
    d = oracle_mod.Domain(geo.xyz, geo.iolets)
    assert len(geo.iolets) == nio
    ref = _brute_nbr(oracle_mod, d.xyz, geo.iolets)
    assert np.array_equal(d.nbr, ref)
    # sampled rows agree with the full table
    pts = d.xyz[:: max(1, d.n // 50)]
    rows = d.nbr_rows(pts)
    assert np.array_equal(rows, d.nbr[:, :: max(1, d.n // 50)].T)


def test_small_cases_by_hand(oracle_mod):
    d = oracle_mod.Domain(np.array([[5, 5, 5]], np.int32), [])
    assert np.all(d.nbr == -1)
    box = S.box(3, 3, 3)
    d = oracle_mod.Domain(box.xyz, [])
    centre = int(np.nonzero((d.xyz == [3, 3, 3]).all(1))[0][0])
    assert np.all(d.nbr[:, centre] >= 0)
    corner = int(np.nonzero((d.xyz == [2, 2, 2]).all(1))[0][0])
    # corner site: sources x - c_i exist only when c_i has no positive component
    c, w, opp = oracle_mod.lattice()
    for i in range(1, 19):
        inside = np.all(c[i] <= 0)
        assert (d.nbr[i - 1, corner] >= 0) == inside
    two = list(_geoms())[3][1]
    d = oracle_mod.Domain(two.xyz, two.iolets)
    down = [i for i in range(1, 19) if c[i][2] == 1]   # source below (z - 1)
    up = [i for i in range(1, 19) if c[i][2] == -1]
    for i in range(1, 19):
        v = d.nbr[i - 1, 0]
        if i in down:
            assert v == -2
        elif i in up:
            assert v == -3
        else:
            assert v == -1


def test_classification_hand_points(oracle_mod):
    # flat cut at z = -0.5 (fixed point -512), outward -z, radius 8
    inlet = S.Iolet(kind=S.PRESSURE, centre=(10240, 10240, -512), axis=(0, 0, -1024),
                    radius=8 * 1024)
    io = [inlet]
    assert oracle_mod.classify((10, 10, -1), io) == -2      # right beyond the plane
    assert oracle_mod.classify((18, 10, -1), io) == -2      # on the rim: distance == radius
    assert oracle_mod.classify((19, 10, -1), io) == -1      # outside the radius
    assert oracle_mod.classify((10, 10, 0), io) == -1       # not beyond the plane
    assert oracle_mod.classify((10, 10, -2), io) == -2      # 1.5 units beyond
    assert oracle_mod.classify((10, 10, -3), io) == -1      # 2.5 units beyond: too deep
    # tilted axis (1, 1, 0) through the origin
    tilt = S.Iolet(kind=S.PRESSURE, centre=(0, 0, 0), axis=(1024, 1024, 0), radius=1024)
    # point (1, 0, 1): along = 1/sqrt2 (within depth), perp^2 = 1/2 + 1 = 1.5 > 1
    assert oracle_mod.classify((1, 0, 1), [tilt]) == -1
    # point (1, 0, 0): perp^2 = 1/2 <= 1
    assert oracle_mod.classify((1, 0, 0), [tilt]) == -2
    # radius just below sqrt(1/2): (1,0,0) falls outside
    tie = S.Iolet(kind=S.PRESSURE, centre=(0, 0, 0), axis=(1024, 1024, 0), radius=724)
    assert oracle_mod.classify((1, 0, 0), [tie]) == -1      # 724/1024 < sqrt(1/2)
    tie2 = S.Iolet(kind=S.PRESSURE, centre=(0, 0, 0), axis=(3 * 1024, 4 * 1024, 0),
                   radius=4 * 1024)
    # point (5, 0, 0): along = 3 units, i.e. beyond the 2-unit depth
    assert oracle_mod.classify((5, 0, 0), [tie2]) == -1     # 3 units beyond > depth 2
    tie3 = S.Iolet(kind=S.PRESSURE, centre=(4 * 1024, 0, 0), axis=(3 * 1024, 4 * 1024, 0),
                   radius=4 * 1024)
    # d = (1, 0, 0): along = 3/5, perp = 4/5 -> inside
    assert oracle_mod.classify((5, 0, 0), [tie3]) == -2
    tie4 = S.Iolet(kind=S.PRESSURE, centre=(0, 0, 0), axis=(3 * 1024, 4 * 1024, 0),
                   radius=int(4 * 1024 / 5))
    # d = (1, 0, 0): perp = 4/5 exactly = radius (819.2 not integer -> 819 < 819.2: outside)
    assert oracle_mod.classify((1, 0, 0), [tie4]) == -1
    tie5 = S.Iolet(kind=S.PRESSURE, centre=(0, 0, 0), axis=(3, 4, 0), radius=4096)
    # d = (5, 0, 0)*1024 -> along 3, perp 4 (radius 4): too deep again
    assert oracle_mod.classify((5, 0, 0), [tie5]) == -1
    tie6 = S.Iolet(kind=S.PRESSURE, centre=(3072, -4096, 0), axis=(3, 4, 0), radius=4096)
    # d = (2, 4, 0): along = (6+16)/5 = 4.4 > 2 -> too deep
    assert oracle_mod.classify((5, 0, 0), [tie6]) == -1
    tie7 = S.Iolet(kind=S.PRESSURE, centre=(4096, 0, 0), axis=(0, 1024, 0), radius=1024)
    # d = (1, 1, 0) -> along 1, perp exactly 1 == radius -> included
    assert oracle_mod.classify((5, 1, 0), [tie7]) == -2
    # lowest index wins when two openings overlap
    both = [tie7, S.Iolet(kind=S.VELOCITY, centre=(4096, 0, 0), axis=(0, 1024, 0),
                          radius=2048)]
    assert oracle_mod.classify((5, 1, 0), both) == -2
    assert oracle_mod.classify((6, 1, 0), both) == -3


def test_build_rejects_bad_input(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.Domain(np.array([[1, 1, 1], [1, 1, 1]], np.int32), [])
    with pytest.raises(ValueError):
        oracle_mod.Domain(np.array([[-1, 1, 1]], np.int32), [])
