"""Device site orderings (Morton canonical, lexicographic rows, bricks) give bit-identical
results: the per-site arithmetic does not depend on where a site sits in memory, each
iolet's FP64 sums run over its sites in canonical order, and the mass sum runs in
canonical order.  Checked through the C ABI for both schemes, 32- and 16-bit storage,
several kernel variants, the pulsatile tree and a coupled pair with alternating
(forward / reverse, body-force) exchanges; neighbour tables decode to the oracle's."""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

pytestmark = pytest.mark.gpu

ORDERS = ("morton", "rows", "bricks")


def _run_tree(gpu, ordering, storage, scheme, steps, launch=None):
    geo = S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7), inlet_speed=0.05, period=200.0)
    ctx = gpu.Context(storage=storage, scheme=scheme)
    try:
        d = ctx.domain(geo.xyz, geo.iolets, tau=0.8, ordering=ordering)
        if launch:
            ctx.set_launch(*launch)
        ctx.step(steps)
        return (d.state(), d.macroscopic(), d.iolet_stats(), d.boundary_values(), d.mass(),
                d.adjacent_moments()[0], d.adjacent_moments()[1])
    finally:
        ctx.close()


@pytest.mark.parametrize("storage,scheme,launch", [
    ("f32", "ab", None), ("f32", "aa", None), ("f16", "aa", None), ("f16", "ab", (256, 2, 5)),
    ("f32", "ab", (256, 2, 3)), ("f32", "aa", (128, 1, 1)), ("bf16", "aa", (256, 1, 0))])
def test_orderings_bit_identical(gpu, storage, scheme, launch):
    for steps in (37, 120):
        ref = _run_tree(gpu, "morton", storage, scheme, steps, launch)
        for o in ORDERS[1:]:
            got = _run_tree(gpu, o, storage, scheme, steps, launch)
            for k, (x, y) in enumerate(zip(ref, got)):
                assert np.array_equal(x, y), (o, steps, k)


@pytest.mark.parametrize("storage,scheme,pairs", [
    ("f32", "ab", [((256, 2, 3), (256, 2, 8)), ((128, 1, 3), (128, 1, 8)), ((128, 2, 3), (128, 2, 13))]),
    ("f16", "ab", [((256, 2, 5), (256, 2, 9)), ((128, 2, 5), (128, 4, 8)), ((64, 4, 3), (64, 4, 13))]),
    ("f32", "aa", [((128, 2, 6), (128, 2, 10)), ((256, 2, 7), (256, 2, 11)), ((256, 1, 3), (256, 1, 8)),
                   ((256, 1, 3), (256, 1, 12)), ((128, 2, 3), (128, 2, 12)), ((128, 2, 3), (128, 2, 13)),
                   ((256, 2, 6), (256, 2, 14))]),
    ("f16", "aa", [((128, 2, 6), (128, 2, 10)), ((64, 2, 7), (64, 2, 11)), ((256, 1, 3), (256, 1, 12)),
                   ((128, 2, 6), (128, 2, 14))]),
    ("bf16", "aa", [((256, 2, 6), (256, 2, 10))])])
def test_run_encoded_table_bit_identical(gpu, storage, scheme, pairs):
    """Variants 8..14 read the run-encoded neighbour table, which a rows- or bricks-ordered
    domain has: same bits as their table-reading counterparts (3, 5, 6, 7, 3, 3, 6), odd and even
    step counts, through graph replays and direct steps."""
    for o in ("rows", "bricks"):
        geo = S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7), inlet_speed=0.05, period=200.0)
        ctx = gpu.Context(storage=storage, scheme=scheme)
        try:
            d = ctx.domain(geo.xyz, geo.iolets, tau=0.8, ordering=o)
            assert d.info()["n_runs"] > 0 and d.n / d.info()["n_runs"] > 4.5, o
        finally:
            ctx.close()
        for base, runs in pairs:
            for steps in (37, 120):
                ref = _run_tree(gpu, o, storage, scheme, steps, base)
                got = _run_tree(gpu, o, storage, scheme, steps, runs)
                for k, (x, y) in enumerate(zip(ref, got)):
                    assert np.array_equal(x, y), (o, base, runs, steps, k)


def test_orderings_neighbours_match_oracle(gpu, oracle_mod):
    geo = S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7))
    od = oracle_mod.Domain(geo.xyz, geo.iolets, tau=0.8)
    for scheme in ("ab", "aa"):
        ctx = gpu.Context(storage="f32", scheme=scheme)
        try:
            for o in ORDERS:
                d = ctx.domain(geo.xyz, geo.iolets, tau=0.8, ordering=o)
                assert np.array_equal(d.sites(), od.xyz)
                assert np.array_equal(d.neighbours(), od.nbr), (scheme, o)
        finally:
            ctx.close()


def test_orderings_coupled_alternating(gpu):
    art = S.tree(S.TreeSpec(depth=3, root_radius=5, seed=3), inlet_speed=0.04, period=100.0)
    ven = S.tree(S.TreeSpec(depth=3, root_radius=5, seed=3), venous=True)
    pairs = [(k, k, 0.7) for k in range(1, len(art.iolets))]
    out = {}
    for o in ORDERS:
        ctx = gpu.Context(storage="f32", scheme="aa")
        try:
            da = ctx.domain(art.xyz, art.iolets, ordering=o)
            dv = ctx.domain(ven.xyz, ven.iolets, ordering="morton" if o == "bricks" else o)
            ctx.couple(da, dv, pairs)
            ctx.set_coupling_mode("alternate")
            ctx.step(151)
            out[o] = [da.state(), dv.state(), da.iolet_stats(), dv.iolet_stats(),
                      da.iolet_forces(), dv.boundary_values(), da.mass(), dv.mass()]
        finally:
            ctx.close()
    assert np.abs(out["morton"][4]).max() > 0          # the reverse exchange did force the outlets
    for o in ORDERS[1:]:
        for k, (x, y) in enumerate(zip(out["morton"], out[o])):
            assert np.array_equal(x, y), (o, k)


def test_ordering_argument_checked(gpu):
    geo = S.cylinder(radius=3, length=8)
    ctx = gpu.Context()
    try:
        with pytest.raises(gpu.HgError) as e:
            ctx.domain(geo.xyz, geo.iolets, ordering=7)
        assert e.value.code == gpu.HG_ERR_ARG
    finally:
        ctx.close()
