"""Benchmark: MFLUPS and HBM-roofline fraction of the sparse D3Q19 LBGK hot path.

Workload (default): seeded bifurcating arterial tree, depth 6 (63 segments),
root radius 24 lattice units scaled by 1.71 (~10M fluid sites), child radius
r * 2^(-1/3), branching angles U(30, 70) deg, segment length U(6, 10) radii,
parabolic velocity inlet with peak 0.05 and a (1 - cos) pulse of period 1000
steps, zero-pressure outlets, tau = 0.8.  One step = stream-collide over all
sites + FP64 iolet reduction/update, i.e. the whole hot path.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same workload instead (the reference arm of this build).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# algorithmic bytes per site update of the stream-collide kernel
BYTES_PER_UPDATE = {
    ("f32", "ab"): 19 * 4 * 2 + 18 * 4,        # 224
    ("f32", "aa"): 19 * 4 * 2 + 18 * 4 // 2,   # 188 (neighbour table on odd steps only)
    ("f16", "aa"): 19 * 2 * 2 + 18 * 4 // 2,   # 112
    ("bf16", "aa"): 19 * 2 * 2 + 18 * 4 // 2,  # 112
    ("f16", "ab"): 19 * 2 * 2 + 18 * 4,        # 148
    ("bf16", "ab"): 19 * 2 * 2 + 18 * 4,       # 148
}
DTYPE_NAME = {"f32": "f32", "f16": "f16-stored/f32-compute", "bf16": "bf16-stored/f32-compute"}


def hbm_peak():
    try:
        with open(PEAKS_PATH) as f:
            v = float(json.load(f)["hbm_gbs"])
            return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload(scale=1.71, depth=6, root_radius=24.0, seed=2010041442):
    from paper_2010_04144_gb300 import synth as S

    spec = S.TreeSpec(depth=depth, root_radius=root_radius, seed=seed, scale=scale)
    geo = S.tree(spec, inlet_speed=0.05, period=1000.0, pulse=S.PULSE_COSINE)
    cfg = {"workload": f"arterial tree d={depth} R={root_radius}x{scale} seed={seed}",
           "fluid_sites": geo.n, "steps_per_job": None, "tau": 0.8,
           "inlet": "parabolic velocity, peak 0.05, (1-cos) pulse T=1000",
           "outlets": "pressure drho=0", "l2": "inputs larger than L2 (state >= 1.5 GB)"}
    return geo, cfg


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist

    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    import torch

    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, ws, local, dist


def max_over_ranks(x, dist, device):
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=f"cuda:{device}")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, stream=None):
    import torch

    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
        torch.cuda.synchronize()


def time_variant(H, geo, storage, scheme, steps, warmup, dist, device, sampler=None):
    """Device-timed steps (graphs), per-kernel launch durations, and the e2e job."""
    import torch

    ctx = H.Context(device=device, storage=storage, scheme=scheme)
    try:
        d = ctx.domain(geo.xyz, geo.iolets, tau=0.8)
        n = d.n
        st = ctx.stream
        # warm-up, then the timed region: exactly `steps` steps, barrier + sync on both sides
        ctx.step(warmup)
        barrier(dist)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.__enter__()
        e0.record(st)
        ctx.step(steps)
        e1.record(st)
        barrier(dist)
        if sampler:
            sampler.__exit__()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms, dist, device)
        # per-kernel durations (CUDA events on the context stream, no graph)
        ms_sc, ms_io = ctx.step_profiled(steps)
        # end to end through the C ABI: host state in (pinned), `steps` steps, macroscopic out
        state = d.save_state()
        pinned = torch.empty(state.size, dtype=torch.uint8, pin_memory=True)
        pinned.numpy()[:] = state
        out = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
        barrier(dist)
        t0 = time.perf_counter()
        d.load_state(pinned.numpy())
        ctx.step(steps)
        from paper_2010_04144_gb300 import hemegb as _H
        import ctypes as C

        rc = _H.lib().hg_read_macroscopic(d.h, C.c_void_p(out.data_ptr()), None)
        if rc != 0:
            raise RuntimeError("read-back failed")
        barrier(dist)
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, device)
        launches_timed = steps * (1 + (1 if geo.iolets else 0)) + (steps + 15) // 16
        return dict(n=n, ms=ms, ms_sc=ms_sc, ms_io=ms_io, e2e_s=e2e_s,
                    h2d=int(state.size), d2h=int(n * 16), launches=launches_timed,
                    device_bytes=d.info()["device_bytes"])
    finally:
        ctx.close()


def cpu_baseline(geo, budget_s=20.0):
    """The FP64 oracle as it stands, on the same geometry, for a bounded number of steps."""
    import oracle

    t0 = time.perf_counter()
    od = oracle.Domain(geo.xyz, geo.iolets, tau=0.8)
    build_s = time.perf_counter() - t0
    s = oracle.System([od])
    t0 = time.perf_counter()
    s.step(1)
    one = time.perf_counter() - t0
    k = max(1, min(50, int(budget_s / max(one, 1e-3)) - 1))
    t0 = time.perf_counter()
    s.step(k)
    dt = time.perf_counter() - t0
    steps = k
    return {"value": od.n * steps / dt / 1e6, "unit": "MFLUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} steps over all {od.n} sites of the same tree (after 1 untimed step; "
                      f"table build {build_s:.1f} s untimed)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    geo, cfg = workload(scale=args.scale)
    od = oracle.Domain(geo.xyz, geo.iolets, tau=0.8)
    s = oracle.System([od])
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    v = od.n * args.steps / dt / 1e6
    cfg["steps_per_job"] = args.steps
    line = {"impl": "reference", "metric": "MFLUPS (D3Q19 LBGK site updates per second / 1e6)",
            "value": v, "unit": "MFLUPS", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded tree)", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "MFLUPS", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} steps over all {od.n} sites"},
            "e2e": {"value": v, "unit": "MFLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="hemegb", choices=["hemegb", "reference"])
    ap.add_argument("--scale", type=float, default=1.71)
    ap.add_argument("--variants", default="f32:aa,f32:ab,f16:aa,bf16:aa")
    ap.add_argument("--headline", default="f32:aa")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2010_04144_gb300 import hemegb as H

    H.lib()
    rank, ws, local, dist = dist_setup()
    device = local
    torch.cuda.set_device(device)
    geo, cfg = workload(scale=args.scale)
    cfg["steps_per_job"] = args.steps
    peak, peak_kind = hbm_peak()
    variants = [tuple(v.split(":")) for v in args.variants.split(",")]
    head = tuple(args.headline.split(":"))
    if head not in variants:
        variants.insert(0, head)
    results = {}
    sampler = ClockSampler(device)
    for (storage, scheme) in variants:
        r = time_variant(H, geo, storage, scheme, args.steps, args.warmup, dist, device,
                         sampler if (storage, scheme) == head else None)
        B = BYTES_PER_UPDATE[(storage, scheme)]
        r["mflups"] = r["n"] * args.steps / (r["ms"] / 1e3) / 1e6
        per_launch_ms = r["ms_sc"] / args.steps
        r["achieved_gbs"] = B * r["n"] / (per_launch_ms / 1e3) / 1e9
        r["bytes_per_update"] = B
        results[(storage, scheme)] = r
    h = results[head]
    total_sites = h["n"] * ws
    value = total_sites * args.steps / (h["ms"] / 1e3) / 1e6
    e2e_value = total_sites * args.steps / h["e2e_s"] / 1e6
    line = {
        "metric": "MFLUPS (D3Q19 LBGK site updates per second / 1e6), whole hot path per step",
        "value": value, "unit": "MFLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[head[0]],
        "data": "synthetic (seeded tree geometry, rest initial state)",
        "config": {**cfg, "storage": head[0], "scheme": head[1],
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": h["achieved_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": h["achieved_gbs"] / peak, "traffic": None,
                     "kernel": "k_stream_collide",
                     "bytes_per_update": h["bytes_per_update"],
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
        "e2e": {"value": e2e_value, "unit": "MFLUPS",
                "h2d_bytes_per_step": h["h2d"] / args.steps,
                "d2h_bytes_per_step": h["d2h"] / args.steps,
                "job": "hg_load_state(pinned host) + steps + hg_read_macroscopic(host)"},
        "gpu_launches": h["launches"],
        "clocks": sampler.summary(),
        "variants": {f"{s}:{c}": {"mflups": r["mflups"], "achieved_gbs": r["achieved_gbs"],
                                   "roofline_frac": r["achieved_gbs"] / peak,
                                   "bytes_per_update": r["bytes_per_update"],
                                   "stream_collide_ms": r["ms_sc"] / args.steps,
                                   "iolet_update_ms": r["ms_io"] / args.steps,
                                   "device_bytes": r["device_bytes"]}
                     for (s, c), r in results.items()},
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(geo)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
