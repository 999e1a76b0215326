"""Split domains on the GPU (Section 2.2: decomposition with a halo exchange after every
step; Section 2.2.1: balanced cuts), through the C ABI: k partitions of one domain in one
process on one device give the bit-identical state, fields, iolet means, boundary values
and mass of the same domain unsplit, for every storage type, several kernel variants and
cuts (equal counts and boundary-weighted), device orderings of the partitions' sites, both
halo transports (direct and staged), over graph and direct launches.  The
partition sizes and halo counts the device build reports equal the host planner's."""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _geo():
    return S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7), inlet_speed=0.05, period=200.0)


def _unsplit(gpu, geo, storage, launch, steps):
    ctx = gpu.Context(storage=storage, scheme="ab")
    try:
        d = ctx.domain(geo.xyz, geo.iolets)
        if launch:
            ctx.set_launch(*launch)
        out = []
        for k in steps:
            ctx.step(k)
            out.append((d.state(), d.macroscopic(), d.iolet_stats(), d.boundary_values(), d.mass()))
        return out
    finally:
        ctx.close()


@pytest.mark.parametrize("storage,launch", [("f32", None), ("f32", (256, 2, 3)), ("f16", (256, 2, 5)),
                                            ("bf16", (128, 1, 1))])
def test_split_bit_identical_to_unsplit(gpu, storage, launch):
    geo = _geo()
    steps = (1, 36, 83)                  # 83 = five graph replays + three direct steps
    ref = _unsplit(gpu, geo, storage, launch, steps)
    for k, bw, ex in ((1, 1.0, "direct"), (2, 1.0, "direct"), (2, 1.0, "staged"), (3, 1.0, "direct"),
                      (5, 4.0, "direct"), (5, 4.0, "staged")):
        ctx = gpu.Context(storage=storage, scheme="ab")
        try:
            sp = ctx.split(geo.xyz, geo.iolets, k, boundary_weight=bw, exchange=ex)
            if launch:
                ctx.set_launch(*launch)
            for j, n in enumerate(steps):
                sp.step(n)
                got = (sp.state(), sp.macroscopic(), sp.iolet_stats(), sp.boundary_values(), sp.mass())
                for q, (x, y) in enumerate(zip(ref[j], got)):
                    assert np.array_equal(x, y), (k, j, q)
        finally:
            ctx.close()


@pytest.mark.parametrize("storage,launch,ordering", [("f32", (128, 2, 3), "rows"), ("f16", (128, 2, 5), "rows"),
                                                     ("f32", (256, 1, 1), "bricks")])
def test_split_orderings_bit_identical(gpu, storage, launch, ordering):
    """Partitions whose owned sites sit in rows or bricks order on the device: same bits as
    the unsplit Morton-ordered domain (the cut, the slot lists and every sum keep the
    canonical order)."""
    geo = _geo()
    steps = (1, 36, 83)
    ref = _unsplit(gpu, geo, storage, launch, steps)
    for k, bw, ex in ((1, 1.0, "direct"), (3, 1.0, "direct"), (4, 3.0, "staged")):
        ctx = gpu.Context(storage=storage, scheme="ab")
        try:
            sp = ctx.split(geo.xyz, geo.iolets, k, boundary_weight=bw, ordering=ordering, exchange=ex)
            ctx.set_launch(*launch)
            for j, n in enumerate(steps):
                sp.step(n)
                got = (sp.state(), sp.macroscopic(), sp.iolet_stats(), sp.boundary_values(), sp.mass())
                for q, (x, y) in enumerate(zip(ref[j], got)):
                    assert np.array_equal(x, y), (k, j, q)
        finally:
            ctx.close()


def test_split_layout_reported(gpu):
    geo = _geo()
    first, ghosts, halo = gpu.split_layout(geo.xyz, geo.iolets, 4, boundary_weight=3.0)
    ctx = gpu.Context(storage="f32", scheme="ab")
    try:
        sp = ctx.split(geo.xyz, geo.iolets, 4, boundary_weight=3.0)
        for p in range(4):
            info = sp.info(p)
            assert info["first"] == first[p] and info["owned"] == first[p + 1] - first[p]
            assert info["ghosts"] == ghosts[p] and info["halo_in"] == halo[:, p].sum()
        d = ctx.domain(geo.xyz, geo.iolets)          # a split and a domain share a context
        ctx.step(10)
        sp.step(10)
        assert np.array_equal(sp.state(), d.state())
        sp.destroy()
        ctx.step(5)
    finally:
        ctx.close()


def test_split_arguments_checked(gpu):
    geo = S.cylinder(radius=3, length=8)
    ctx = gpu.Context(storage="f32", scheme="aa")
    try:
        with pytest.raises(gpu.HgError) as e:
            ctx.split(geo.xyz, geo.iolets, 2)
        assert e.value.code == gpu.HG_ERR_ARG       # the A/B scheme only
    finally:
        ctx.close()
    ctx = gpu.Context(storage="f32", scheme="ab")
    try:
        with pytest.raises(gpu.HgError):
            ctx.split(geo.xyz, geo.iolets, 0)
        for bad in (dict(exchange=2), dict(ordering=3)):
            with pytest.raises(gpu.HgError) as e:
                ctx.split(geo.xyz, geo.iolets, 2, **bad)
            assert e.value.code == gpu.HG_ERR_ARG
        sp = ctx.split(geo.xyz, geo.iolets, 2)   # the context is still usable
        sp.step(3)
    finally:
        ctx.close()
