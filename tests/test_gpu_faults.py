"""Failure detection, host-side only (no GPU fault, trap or hang is made):
  * an allocation that fails (injected: the allocator behaves as if it returned NULL)
    gives HG_ERR_OOM, releases everything the failed call had set up, and leaves the
    context usable -- a later build and run is bit-identical to an undisturbed one;
  * the device error word, set from the host exactly as a bounded device wait that gave
    up sets it, makes hg_sync report HG_ERR_TIMEOUT once, then clears;
  * the NaN/Inf watchdog of the mass pass counts non-finite stored values (a state
    loaded from the host with a NaN in it) and reports HG_ERR_STATE.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _geo():
    return S.tree(S.TreeSpec(depth=3, root_radius=5, seed=3), inlet_speed=0.04, period=100.0)


def _reference(gpu, steps):
    geo = _geo()
    ctx = gpu.Context(storage="f32", scheme="ab")
    try:
        d = ctx.domain(geo.xyz, geo.iolets)
        ctx.step(steps)
        return d.state(), d.iolet_stats()
    finally:
        ctx.close()


def test_injected_allocation_failures(gpu):
    geo = _geo()
    ref = _reference(gpu, 40)
    ctx = gpu.Context(storage="f32", scheme="ab")
    try:
        base = len(ctx._alloc.live)
        failed = 0
        for k in range(1, 40):
            ctx.inject_fault(gpu.FAULT_ALLOC, k)
            try:
                d = ctx.domain(geo.xyz, geo.iolets)
            except gpu.HgError as e:
                assert e.code == gpu.HG_ERR_OOM and "injected" in str(e)
                assert len(ctx._alloc.live) == base          # nothing of the failed build is held
                failed += 1
                continue
            ctx.inject_fault(gpu.FAULT_ALLOC, 0)              # the build needed fewer allocations
            d.destroy()
            assert len(ctx._alloc.live) == base
            break
        assert failed >= 10                                    # every buffer of a build was hit
        d = ctx.domain(geo.xyz, geo.iolets)
        ctx.inject_fault(gpu.FAULT_ALLOC, 1)                   # the first step builds its plan
        with pytest.raises(gpu.HgError) as e:
            ctx.step(40)
        assert e.value.code == gpu.HG_ERR_OOM
        assert d.step == 0
        ctx.step(40)
        got = d.state(), d.iolet_stats()
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)
    finally:
        ctx.close()


def test_device_error_word_reports_timeout(gpu):
    geo = _geo()
    ctx = gpu.Context(storage="f32", scheme="aa")
    try:
        d = ctx.domain(geo.xyz, geo.iolets)
        ctx.step(10)
        ctx.sync()
        ctx.inject_fault(gpu.FAULT_DEVICE_WAIT, 3)
        with pytest.raises(gpu.HgError) as e:
            ctx.sync()
        assert e.value.code == gpu.HG_ERR_TIMEOUT and "not trusted" in str(e.value)
        ctx.sync()                                             # reported once, then cleared
        ctx.step(10)
        ctx.sync()
        assert d.step == 20
    finally:
        ctx.close()


@pytest.mark.parametrize("storage,scheme", [("f32", "ab"), ("f16", "aa")])
def test_nan_watchdog(gpu, storage, scheme):
    geo = S.cylinder(radius=5, length=24)
    ctx = gpu.Context(storage=storage, scheme=scheme)
    try:
        d = ctx.domain(geo.xyz, geo.iolets)
        ctx.step(30)
        m, bad, rc = d.state_check()
        assert rc == gpu.HG_OK and bad == 0 and m == d.mass()
        buf = d.save_state()
        raw = d.state()
        nio = len(geo.iolets)
        off = 40 + 28 * nio                                    # header, boundary values, means
        poisoned = raw.copy()
        poisoned[3, d.n // 2] = np.nan
        buf[off:off + raw.nbytes] = np.frombuffer(poisoned.tobytes(), np.uint8)
        d.load_state(buf)
        m, bad, rc = d.state_check()
        assert rc == gpu.HG_ERR_STATE and bad == 1 and np.isnan(m)
        ctx.step(5)                                            # the NaN spreads to neighbours
        _, bad5, rc = d.state_check()
        assert rc == gpu.HG_ERR_STATE and bad5 > 1
    finally:
        ctx.close()
