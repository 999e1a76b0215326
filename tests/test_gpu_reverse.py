"""Reverse coupling direction (Section 3) on the GPU against the oracle.

With alternating exchanges the arterial outlets receive a body force from the
venous inflow they feed (Guo forcing on the outlet-adjacent sites), applied by
the body-force pass after stream-collide.  Checked here: fields, iolet forces
and boundary values against the FP64 oracle for both schemes; bit-identity of
every kernel variant with forces on; a checkpoint taken mid-run resumes
bit-identically (forces included); switching back to forward-only clears them.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

from test_gpu_parity import LAUNCHES, TAU, TOL, field_errors

pytestmark = pytest.mark.gpu


def _pair_1toN(gpu):
    art = S.tree(S.TreeSpec(depth=3, root_radius=4.0, seed=21), inlet_speed=0.04, period=300.0)
    ven = S.tree(S.TreeSpec(depth=4, root_radius=3.0, seed=22), venous=True, venous_offset=6.0)
    oa, ov = np.array(art.origin), np.array(ven.origin)
    ac = [tuple(int(c) for c in np.array(io.centre) + 1024 * oa) for io in art.iolets[1:]]
    vc = [tuple(int(c) for c in np.array(io.centre) + 1024 * ov) for io in ven.iolets[1:]]
    aa = [io.area() for io in art.iolets[1:]]
    va = [io.area() for io in ven.iolets[1:]]
    assign, _, _, fac = gpu.hg_coupling_factors(ac, aa, vc, va, S.uniform_draws(5, len(vc)))
    pairs = [(int(assign[v]) + 1, v + 1, float(fac[v])) for v in range(len(vc))]
    return art, ven, pairs


def _setup(gpu, art, ven, pairs, storage="f32", scheme="ab", **kw):
    ctx = gpu.Context(storage=storage, scheme=scheme, **kw)
    da = ctx.domain(art.xyz, art.iolets, tau=TAU)
    dv = ctx.domain(ven.xyz, ven.iolets, tau=TAU)
    ctx.couple(da, dv, pairs)
    ctx.set_coupling_mode("alternate")
    return ctx, da, dv


@pytest.mark.parametrize("storage,scheme", [("f32", "ab"), ("f32", "aa"), ("f16", "aa")])
def test_alternating_exchange_against_oracle(gpu, oracle_mod, storage, scheme):
    art, ven, pairs = _pair_1toN(gpu)
    ctx, da, dv = _setup(gpu, art, ven, pairs, storage, scheme)
    try:
        oa = oracle_mod.Domain(art.xyz, art.iolets, tau=TAU)
        ov = oracle_mod.Domain(ven.xyz, ven.iolets, tau=TAU)
        sysm = oracle_mod.System([oa, ov], [(0, a, 1, v, f) for (a, v, f) in pairs], alternate=True)
        tol = TOL[storage]
        done = 0
        for cp in (151, 300, 463):
            ctx.step(cp - done)
            sysm.step(cp - done)
            done = cp
            for d, od in ((da, oa), (dv, ov)):
                eu, ep = field_errors(d.macroscopic(), od.moments())
                assert eu < tol and ep < tol, (storage, scheme, cp, eu, ep)
            Fg, Fo = da.iolet_forces(), sysm.iolet_force[0]
            assert np.abs(Fo).max() > 0
            bar = {"f32": 1e-4, "f16": 3e-2}[storage]
            np.testing.assert_allclose(Fg, Fo, rtol=0, atol=bar * np.abs(Fo).max())
            assert not np.any(dv.iolet_forces())          # inlets are never forced
            bo = sysm.bc_values(1, cp + 1)
            bg = dv.boundary_values()
            for (_, v, _) in pairs:
                assert abs(bg[v] - bo[v]) <= bar * np.abs(bo).max(), (v, bg[v], bo[v])
    finally:
        ctx.close()


def test_forced_variants_bit_identical(gpu):
    art, ven, pairs = _pair_1toN(gpu)
    ref = {}
    for (scheme, block, spt, var) in LAUNCHES:
        if var in (5, 9):  # 16-bit storage only
            continue
        ctx, da, dv = _setup(gpu, art, ven, pairs, "f32", scheme, block_size=block,
                             sites_per_thread=spt, kernel_variant=var)
        try:
            ctx.step(257)
            got = (da.state(), dv.state(), da.iolet_forces(), da.iolet_stats())
            key = scheme
            if key not in ref:
                ref[key] = got
                assert np.any(got[2])
            for x, y in zip(ref[key], got):
                assert np.array_equal(x, y), (scheme, block, spt, var)
        finally:
            ctx.close()


def test_checkpoint_resume_and_mode_switch(gpu):
    art, ven, pairs = _pair_1toN(gpu)
    ctx, da, dv = _setup(gpu, art, ven, pairs, "f32", "aa")
    try:
        ctx.step(301)
        snap = (da.save_state(), dv.save_state())
        ctx.step(60)
        want = (da.state(), dv.state(), da.iolet_forces())
    finally:
        ctx.close()
    ctx, da, dv = _setup(gpu, art, ven, pairs, "f32", "aa")
    try:
        da.load_state(snap[0])
        dv.load_state(snap[1])
        assert np.any(da.iolet_forces())
        ctx.step(60)
        got = (da.state(), dv.state(), da.iolet_forces())
        for x, y in zip(want, got):
            assert np.array_equal(x, y)
        ctx.set_coupling_mode("forward")
        assert not np.any(da.iolet_forces())
        with pytest.raises(gpu.HgError):
            ctx.set_coupling_mode(7)
    finally:
        ctx.close()
