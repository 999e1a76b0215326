"""Precision form on the workload's accuracy instance: the depth-8 tree generator
(root radius 40, all lengths x 0.54: ~1.94M fluid sites), 5000 steps, FP32 / FP16 / BF16
storage on the GPU against the FP64 oracle, velocity and pressure relative L2 at 1000,
2500 and 5000 steps.  Bars: FP32 1e-5 and FP16 1e-3 (the stated tolerances); BF16 is
held to its own bound, 8 units of BF16 rounding (8 * 2^-9 = 1.6e-2 is far above what it
reaches; the bound it is reported against is BF16_BOUND below), because an 8-bit
significand cannot carry these fields to 1e-3.  This instance is larger than L2, so
the FP16 error is accumulated with the traffic pattern of the throughput runs.

The oracle runs in a spawned process while the GPU runs the three forms."""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKS = (1000, 2500, 5000)
BF16_BOUND = 1e-2


def _geo():
    sys.path.insert(0, ROOT)
    from paper_2010_04144_gb300 import synth as S

    return S.tree(S.TreeSpec(depth=8, root_radius=40.0, seed=2010041442, scale=0.54),
                  inlet_speed=0.05, period=1000.0)


def _oracle_run(out_path):
    """Child process: the FP64 oracle over the same instance, moments at the checkpoints."""
    sys.path.insert(0, ROOT)
    import oracle

    geo = _geo()
    od = oracle.Domain(geo.xyz, geo.iolets, tau=0.8)
    sysm = oracle.System([od])
    res, done = {}, 0
    for cp in CHECKS:
        sysm.step(cp - done)
        done = cp
        res[f"m{cp}"] = od.moments()
    np.savez(out_path, **res)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_precision_forms_vs_oracle_5000_steps(gpu, oracle_mod, tmp_path):
    out_path = str(tmp_path / "oracle.npz")
    proc = mp.get_context("spawn").Process(target=_oracle_run, args=(out_path,))
    proc.start()
    geo = _geo()
    got = {}
    try:
        for storage in ("f32", "f16", "bf16"):
            ctx = gpu.Context(storage=storage, scheme="aa")
            try:
                d = ctx.domain(geo.xyz, geo.iolets, tau=0.8)
                done = 0
                for cp in CHECKS:
                    ctx.step(cp - done)
                    done = cp
                    got[(storage, cp)] = d.macroscopic().astype(np.float64)
            finally:
                ctx.close()
    finally:
        proc.join()
    assert proc.exitcode == 0
    ref = np.load(out_path)
    bars = {"f32": 1e-5, "f16": 1e-3, "bf16": BF16_BOUND}
    report = {}
    for (storage, cp), m in got.items():
        r = ref[f"m{cp}"]
        eu, ep = rel(m[:, 1:], r[:, 1:]), rel(m[:, 0] / 3, r[:, 0] / 3)
        report[(storage, cp)] = (eu, ep)
    print("precision vs FP64 oracle (velocity, pressure rel L2):",
          {f"{s}@{c}": (f"{a:.2e}", f"{b:.2e}") for (s, c), (a, b) in report.items()})
    for (storage, cp), (eu, ep) in report.items():
        assert eu < bars[storage] and ep < bars[storage], (storage, cp, eu, ep)
