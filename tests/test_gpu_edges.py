"""Degenerate and ragged domains through the C ABI (Section 2: the LB step on a sparse
fluid-site list; Section 2.2: the site list and its neighbour table).

  * one-voxel-wide lines of 1, 2, 3, 33 and 129 sites between a pressure inlet and outlet,
    and thin tubes whose site counts leave ragged last tiles (155 and 481 sites): every
    kernel variant, both schemes, Morton and rows ordering (the run-encoded variants take
    their run path where the table compresses, the table path otherwise) gives the same
    bits, and the fields follow the FP64 oracle within the FP32 bar;
  * an empty domain (no sites) steps, reads back and sums to nothing, alone and batched with
    a real domain, whose result stays the bits it has alone;
  * a domain above the site limit is refused before any of its data is read.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S
from test_gpu_parity import TAU, TOL, field_errors

pytestmark = pytest.mark.gpu

STEPS = 40
LAUNCHES = {"ab": [(64, 1, 0), (128, 2, 3), (64, 2, 1), (128, 2, 8), (128, 2, 13), (64, 4, 13)],
            "aa": [(64, 1, 0), (128, 2, 6), (64, 2, 2), (256, 1, 8), (128, 2, 10), (128, 2, 14)]}


def _geoms():
    g = {f"line{n}": S.cylinder(radius=0, length=n, margin=3) for n in (1, 2, 3, 33, 129)}
    g["tube155"] = S.cylinder(radius=1, length=31)
    g["tube481"] = S.cylinder(radius=2, length=37)
    return g


@pytest.mark.parametrize("name", ["line1", "line2", "line3", "line33", "line129", "tube155", "tube481"])
def test_small_and_ragged_domains(gpu, oracle_mod, name):
    geo = _geoms()[name]
    od = oracle_mod.Domain(geo.xyz, geo.iolets, tau=TAU)
    oracle_mod.System([od]).step(STEPS)
    ref = od.moments()
    assert np.abs(ref[:, 1:]).max() > 0            # the inlet drives a flow through every case
    for scheme, launches in LAUNCHES.items():
        first = None
        for ordering in ("morton", "rows"):
            for launch in launches:
                ctx = gpu.Context(storage="f32", scheme=scheme)
                try:
                    d = ctx.domain(geo.xyz, geo.iolets, tau=TAU, ordering=ordering)
                    assert d.n == geo.n
                    ctx.set_launch(*launch)
                    ctx.step(STEPS)
                    got = (d.state(), d.macroscopic(), d.iolet_stats())
                finally:
                    ctx.close()
                if first is None:
                    first = got
                    eu, ep = field_errors(got[1], ref)
                    assert eu < TOL["f32"] and ep < TOL["f32"], (name, scheme, eu, ep)
                for x, y in zip(first, got):
                    assert np.array_equal(x, y), (name, scheme, ordering, launch)


def test_empty_domain(gpu):
    geo = S.cylinder(radius=3, length=20)
    ctx = gpu.Context(storage="f32", scheme="ab")
    try:
        d = ctx.domain(geo.xyz, geo.iolets, tau=TAU)
        ctx.step(25)
        alone = d.state()
    finally:
        ctx.close()
    for scheme in ("ab", "aa"):
        ctx = gpu.Context(storage="f32", scheme=scheme)
        try:
            e = ctx.domain(np.zeros((0, 3), np.int32), [], tau=TAU)
            assert e.n == 0
            ctx.step(5)
            assert e.macroscopic().shape == (0, 4) and e.mass() == 0.0
            assert e.state().size == 0
            if scheme == "ab":
                d = ctx.domain(geo.xyz, geo.iolets, tau=TAU)   # batched with a real domain
                ctx.step(25)
                assert np.array_equal(d.state(), alone)
                assert e.macroscopic().shape == (0, 4)
        finally:
            ctx.close()


def test_site_limit_refused(gpu):
    """The limit is checked before the site array is touched: a one-site array with a site
    count above the limit is refused, and the context stays usable."""
    ctx = gpu.Context(storage="f32", scheme="aa")
    try:
        xyz = np.zeros((1, 3), np.int32)
        h = C.c_void_p()
        rc = gpu.lib().hg_domain_create(ctx.h, xyz.ctypes.data_as(C.c_void_p), (200 << 20) + 1, None, 0,
                                        None, C.byref(h))
        assert rc == gpu.HG_ERR_ARG and not h.value
        assert b"too many sites" in gpu.lib().hg_last_error(ctx.h)
        geo = S.cylinder(radius=2, length=10)
        d = ctx.domain(geo.xyz, geo.iolets, tau=TAU)
        ctx.step(3)
        assert d.step == 3
    finally:
        ctx.close()
