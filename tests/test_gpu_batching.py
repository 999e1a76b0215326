"""Mixed plans: in a step over several domains, the large ones (≥ 2^20 sites) are launched
one by one with the single-domain kernel, chained by programmatic dependent launch, and
the small ones share one tile-table launch.  Each domain's result is bit-identical to the
same domain stepped alone, for both schemes and 32/16-bit storage, the table and the
run-encoded kernel variants, with coupling between a large and a small domain."""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _geoms():
    spec = S.TreeSpec(depth=5, root_radius=16.0, seed=3)
    spec.scale = S.scale_for_sites(spec, 1.3e6)
    big = S.tree(spec, inlet_speed=0.05, period=300.0)
    small = [S.tree(S.TreeSpec(depth=4, root_radius=6, seed=s), inlet_speed=0.04, period=200.0) for s in (7, 8)]
    assert big.n >= 1 << 20 and all(g.n < 1 << 20 for g in small)
    return [small[0], big, small[1]]


def _alone(gpu, geo, storage, scheme, steps, launch=None):
    ctx = gpu.Context(storage=storage, scheme=scheme)
    try:
        d = ctx.domain(geo.xyz, geo.iolets, ordering="rows")
        if launch:
            ctx.set_launch(*launch)
        ctx.step(steps)
        return d.state(), d.iolet_stats(), d.boundary_values()
    finally:
        ctx.close()


@pytest.mark.parametrize("storage,scheme,launch", [
    ("f32", "aa", None), ("f16", "ab", None), ("bf16", "aa", None),
    # run-encoded variants: the large domain in its own launch, the small ones in the
    # tile-table kernel; the reference is each domain alone with the table form
    ("f32", "ab", (128, 2, 13)), ("f32", "aa", (256, 1, 8)), ("f16", "aa", (128, 2, 10)),
    ("f16", "ab", (256, 2, 8))])
def test_mixed_plan_bit_identical_to_alone(gpu, storage, scheme, launch):
    geos = _geoms()
    steps = 37
    ref = [_alone(gpu, g, storage, scheme, steps) for g in geos]
    ctx = gpu.Context(storage=storage, scheme=scheme)
    try:
        ds = [ctx.domain(g.xyz, g.iolets, ordering="rows") for g in geos]
        assert all(d.info()["n_runs"] > 0 for d in ds)
        if launch:
            ctx.set_launch(*launch)
        ctx.step(steps)
        for d, r in zip(ds, ref):
            got = d.state(), d.iolet_stats(), d.boundary_values()
            for x, y in zip(r, got):
                assert np.array_equal(x, y)
    finally:
        ctx.close()


def test_mixed_plan_with_coupling(gpu):
    """A large arterial tree coupled to its larger venous twin (forward, every step), both
    launched separately: the pair's results are the same bits with and without an extra
    small domain sharing the steps through a tile-table launch."""
    spec = S.TreeSpec(depth=3, root_radius=16.0, seed=5)
    spec.scale = S.scale_for_sites(spec, 1.3e6)
    art = S.tree(spec, inlet_speed=0.05, period=300.0)
    ven = S.tree(spec, venous=True)
    extra = S.tree(S.TreeSpec(depth=4, root_radius=6, seed=9), inlet_speed=0.04, period=200.0)
    pairs = [(k, k, 0.7) for k in range(1, len(art.iolets))]
    out = []
    for with_extra in (False, True):
        ctx = gpu.Context(storage="f32", scheme="ab")
        try:
            da = ctx.domain(art.xyz, art.iolets)
            dv = ctx.domain(ven.xyz, ven.iolets)
            if with_extra:
                ctx.domain(extra.xyz, extra.iolets)
            ctx.couple(da, dv, pairs)
            ctx.step(2000)       # the inlet's wave needs ~1700 steps to reach every outlet
            out.append((da.state(), dv.state(), dv.boundary_values(), da.iolet_stats()))
        finally:
            ctx.close()
    for x, y in zip(*out):
        assert np.array_equal(x, y)
    assert np.abs(out[0][2]).max() > 0
