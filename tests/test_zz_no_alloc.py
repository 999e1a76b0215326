"""hg_mass_noalloc: the mass reduction for callers that may not allocate device memory.

Some callers cannot call cudaMalloc: an application whose own memory pool
already owns the whole device heap, or a monitoring thread that must not
stall the solver with an allocation.  hg_mass_noalloc keeps its scratch in a
fixed array inside the library; this test checks, through the C ABI, that it
returns exactly what the regular hg_mass returns for the same state (same
partition, same summation order), on two calls in a row (the second call must
not be disturbed by what the first left in the shared scratch array), for a
dense copy on the legacy stream and for a copy with padded rows (garbage in
the padding) on a caller's stream.  The file name makes pytest collect it last.
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
        assert ref != 0.0
        n = d.n
        bits = raw.view(np.int32 if raw.itemsize == 4 else np.int16)
        dense = torch.from_numpy(bits.copy()).cuda()
        stride = (n + 127) // 128 * 128
        padded_h = np.full((19, stride), -12345, bits.dtype)   # non-zero garbage in the padding
        padded_h[:, :n] = bits
        padded = torch.from_numpy(padded_h).cuda()
        code = gpu.STORAGE[storage]
        L = gpu.lib()
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        for k in range(2):                  # legacy default stream, dense rows
            rc = L.hg_mass_noalloc(C.c_void_p(dense.data_ptr()), code, n, n,
                                   C.c_void_p(out.data_ptr() + 8 * k), None)
            assert rc == gpu.HG_OK
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        for k in range(2, 4):               # a caller's stream, padded rows
            rc = L.hg_mass_noalloc(C.c_void_p(padded.data_ptr()), code, n, stride,
                                   C.c_void_p(out.data_ptr() + 8 * k), C.c_void_p(side.cuda_stream))
            assert rc == gpu.HG_OK
        side.synchronize()
        got = out.cpu().numpy()
        for k in range(4):
            assert got[k] == ref, (k, got[k], ref)
        # sizes beyond the fixed scratch are refused with HG_ERR_ARG
        rc = L.hg_mass_noalloc(C.c_void_p(dense.data_ptr()), code, 16384 * 8192 + 1,
                               16384 * 8192 + 1, C.c_void_p(out.data_ptr()), None)
        assert rc == gpu.HG_ERR_ARG
        rc = L.hg_mass_noalloc(C.c_void_p(dense.data_ptr()), code, n, n - 1,
                               C.c_void_p(out.data_ptr()), None)
        assert rc == gpu.HG_ERR_ARG         # rows shorter than the site count
    finally:
        ctx.close()
