"""Host build of the canonical order and neighbour table (hg_build_neighbours), CPU only.

The same code builds every domain's table before upload; here it is compared
bit for bit with the oracle's own construction (which is pinned by brute force
in test_oracle_geometry) on geometries with walls, iolet openings and ties:
a tube with both iolet kinds, a seeded tree, its venous twin, a closed box, a
single voxel; plus the error cases a domain build rejects.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

CASES = {
    "tube": lambda: S.cylinder(radius=5, length=20, inlet=dict(kind=S.VELOCITY, value=0.01,
                                                              profile=S.PARABOLIC)),
    "tree": lambda: S.tree(S.TreeSpec(depth=4, root_radius=5, seed=7)),
    "venous": lambda: S.tree(S.TreeSpec(depth=3, root_radius=4, seed=21), venous=True),
    "box": lambda: S.box(5, 4, 3),
    "voxel": lambda: S.Geometry(xyz=np.array([[3, 4, 5]], np.int32), iolets=[]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_matches_oracle_bitwise(hemegb_lib, oracle_mod, name):
    from paper_2010_04144_gb300 import hemegb as H

    geo = CASES[name]()
    rng = np.random.default_rng(3)
    xyz = geo.xyz[rng.permutation(geo.xyz.shape[0])]        # any input order
    xs, nbr = H.build_neighbours(xyz, geo.iolets)
    od = oracle_mod.Domain(xyz, geo.iolets)
    assert np.array_equal(xs, od.xyz)
    assert np.array_equal(nbr, od.nbr)
    if geo.iolets:
        assert (nbr < -1).any()                             # iolet links present


def test_rejects_what_a_domain_build_rejects(hemegb_lib):
    from paper_2010_04144_gb300 import hemegb as H

    with pytest.raises(H.HgError):
        H.build_neighbours(np.array([[1, 1, 1], [1, 1, 1]], np.int32), [])     # duplicate
    with pytest.raises(H.HgError):
        H.build_neighbours(np.array([[-1, 0, 0]], np.int32), [])               # out of range
    xs, nbr = H.build_neighbours(np.zeros((0, 3), np.int32), [])
    assert xs.shape == (0, 3) and nbr.shape == (18, 0)
