"""Iolet means (Section 2.3: only averages of macroscopic values cross between coupled
instances) held to 1e-12 relative against an FP64 sum of the very same per-site inputs.

The GPU reduces each iolet's sites in chunks of 256 with a fixed shuffle tree and adds the
chunk sums in order; the host here sums the same FP32 moments (read back through
hg_read_adjacent_moments) in FP64, sequentially in canonical order.  The two orders differ,
so the bar is 1e-12 of the terms' scale rather than bit equality; the count must be exact.
Cases span one and several chunks, both schemes, FP32 and FP16 storage and a reordered
device layout."""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _check_means(d, geo):
    nbr = d.neighbours()
    sites, mom = d.adjacent_moments()
    assert np.all(np.diff(sites) > 0)                           # canonical order
    M = d.iolet_stats()
    for k, io in enumerate(geo.iolets):
        mine = np.nonzero((nbr == -(2 + k)).any(axis=0))[0]
        rows = np.searchsorted(sites, mine)
        assert np.array_equal(sites[rows], mine)
        assert M[k, 2] == len(mine)
        if not len(mine):
            continue
        a = np.array(io.axis, dtype=np.float64)
        nh = a / np.sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2])
        m = mom[rows].astype(np.float64)
        terms = m[:, 1] * nh[0] + m[:, 2] * nh[1] + m[:, 3] * nh[2]
        su = sr = 0.0
        for t, r in zip(terms, m[:, 0]):                       # sequential, canonical order
            su += t
            sr += r
        ref_u, ref_r = su / len(mine), sr / len(mine)
        scale_u = max(abs(ref_u), float(np.mean(np.abs(terms))))
        scale_r = max(abs(ref_r), float(np.mean(np.abs(m[:, 0]))))
        assert abs(M[k, 0] - ref_u) <= 1e-12 * scale_u, (k, M[k, 0], ref_u)
        assert abs(M[k, 1] - ref_r) <= 1e-12 * scale_r, (k, M[k, 1], ref_r)
    return M


@pytest.mark.parametrize("storage,scheme,ordering", [("f32", "ab", "morton"), ("f16", "aa", "morton"),
                                                     ("f32", "aa", "rows")])
def test_iolet_means_same_inputs(gpu, storage, scheme, ordering):
    cases = [S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7), inlet_speed=0.05, period=200.0),
             S.cylinder(radius=12, length=16,
                        inlet=dict(kind=S.VELOCITY, value=0.02, profile=S.PARABOLIC))]
    for geo in cases:
        ctx = gpu.Context(storage=storage, scheme=scheme)
        try:
            d = ctx.domain(geo.xyz, geo.iolets, tau=0.8, ordering=ordering)
            for steps in (1, 36, 77):
                ctx.step(steps)
                M = _check_means(d, geo)
            assert np.abs(M[:, 0]).max() > 0
            assert max(M[:, 2]) > 256 or geo.meta.get("kind") != "cylinder"   # several chunks
        finally:
            ctx.close()
