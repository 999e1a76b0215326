"""hg_mass_noalloc: the mass reduction for callers that may not allocate device memory.

Some callers cannot call cudaMalloc: an application whose own memory pool
already owns the whole device heap, or a monitoring thread that must not
stall the solver with an allocation.  hg_mass_noalloc keeps its scratch in a
fixed array inside the library; this test checks, through the C ABI, that it
returns what the regular hg_mass returns for the same state, on two calls in
a row (the second call must not be disturbed by what the first left in the
shared scratch array).  The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_mass_noalloc_matches_mass(gpu, storage):
    import torch

    geo = S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7), inlet_speed=0.05, period=200.0)
    ctx = gpu.Context(storage=storage, scheme="aa")
    try:
        d = ctx.domain(geo.xyz, geo.iolets, tau=0.8)
        ctx.step(40)
        raw = d.state()                     # (19, n) raw storage values, canonical order
        ref = d.mass()                      # regular entry point
        dev = torch.from_numpy(raw.view(np.int32 if raw.itemsize == 4 else np.int16).copy()).cuda()
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        code = gpu.STORAGE[storage]
        L = gpu.lib()
        for k in range(2):
            rc = L.hg_mass_noalloc(C.c_void_p(dev.data_ptr()), code, d.n, d.n,
                                   C.c_void_p(out.data_ptr() + 8 * k), None)
            assert rc == gpu.HG_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k in range(2):
            assert abs(got[k] - ref) <= 1e-12 * max(1.0, abs(ref)), (k, got[k], ref)
        assert ref != 0.0
        # sizes beyond the fixed scratch are refused with HG_ERR_ARG
        rc = L.hg_mass_noalloc(C.c_void_p(dev.data_ptr()), code, 16384 * 8192 + 1,
                               16384 * 8192 + 1, C.c_void_p(out.data_ptr()), None)
        assert rc == gpu.HG_ERR_ARG
    finally:
        ctx.close()
