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
import math
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
# one metric string for both arms, so the two lines are directly comparable
METRIC = "MFLUPS (D3Q19 LBGK site updates per second / 1e6), whole hot path per step"
# each variant's K-step measurement is repeated until this much device time has passed
# (nvidia-smi samples every 100 ms), and the median repetition is reported
MIN_TIMED_S = 1.0
FALLBACK_HBM_GBS = 6800.0

# device site orderings the autotuner tries (every one gives bit-identical results)
ORDERINGS = ("morton", "rows", "bricks")

def bytes_per_update(storage, scheme, variant=0, n=1, n_runs=0):
    """Algorithmic bytes per site update of the stream-collide kernel: the 19 populations
    read and written once each, plus the neighbour table on pull steps (every A/B step, the
    odd AA steps): its 18 rows (72 bytes), or for the run-encoded variants (8..11, on a
    domain that has runs) the per-site word (4 bytes), the 80-byte offset rows of the runs
    shared by their sites and the per-1024-site chunk word.  With the table: 224 / 188 bytes
    (FP32 A/B / AA), 148 / 112 (16-bit)."""
    eb = 4 if storage == "f32" else 2
    data = 19 * eb * 2
    table = 4 + 80 * n_runs / n + 4 / 1024 if (variant >= 8 and n_runs > 0) else 72
    return data + (table if scheme == "ab" else table / 2)


def domain_bytes(ctx, storage, scheme, doms):
    """Bytes per update averaged over the domains one launch sequence steps."""
    v = ctx.launch[2]
    tot = sum(d.n for d in doms)
    return sum(bytes_per_update(storage, scheme, v, d.n, d.info()["n_runs"]) * d.n for d in doms) / tot
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
    """nvidia-smi clock/throttle sampling; only samples taken inside marked timed regions count."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []
        self.active = False

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def mark(self, on):
        self.active = on

    def _read(self):
        for line in self.proc.stdout:
            if self.active:
                self.lines.append(line.strip())

    def stop(self):
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


def profiled_traffic(variant_key, launch, ordering="morton"):
    """DRAM bytes per launch from the committed ncu summary, if it matches this kernel build,
    launch shape and site ordering."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        entries = t.get(variant_key) or []
        for e in entries if isinstance(entries, list) else [entries]:  # one record per launch shape
            if (e.get("launch") == launch and e.get("kernel_source_sha") == kernel_source_sha()
                    and e.get("ordering", "morton") == ordering):
                return e["bytes_per_launch"], e.get("scaled_from")
    except Exception:
        pass
    return None, None


def kernel_source_sha():
    import hashlib

    h = hashlib.sha256()
    for f in ("hg_device.cuh", "hg_sc_part.cu", "hg_internal.h"):
        with open(os.path.join(ROOT, "paper_2010_04144_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


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
    """Largest value over all ranks (the slowest replica's time)."""
    if dist is None:
        return x
    import torch

    dev = f"cuda:{device}" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    import torch

    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
        if torch.cuda.is_available():
            torch.cuda.synchronize()


def whole_job_mflups(sites_per_rank, world_size, steps, max_ms):
    """Weak scaling: every rank advances its own replica; units of all ranks / slowest time."""
    return sites_per_rank * world_size * steps / (max_ms / 1e3) / 1e6


def time_variant(H, geo, storage, scheme, steps, warmup, dist, device, sampler, launch=None,
                 orderings=ORDERINGS, min_timed_s=MIN_TIMED_S):
    """Autotuned (or given) site ordering and launch shape, device-timed steps (graphs),
    per-kernel times, e2e job."""
    import torch

    from paper_2010_04144_gb300.autotune import autotune, tune_ordering

    nvtx = torch.cuda.nvtx
    tag = f"{storage}:{scheme}"
    order_ms = {}
    if launch is None and len(orderings) > 1:
        def make(o):
            c = H.Context(device=device, storage=storage, scheme=scheme)
            c.domain(geo.xyz, geo.iolets, tau=0.8, ordering=o)
            return c

        nvtx.range_push(f"{tag}-ordering")
        ordering, _, table = tune_ordering(make, orderings)
        order_ms = {o: round(v[1], 4) for o, v in table.items()}
        nvtx.range_pop()
    else:
        ordering = orderings[0]
    ctx = H.Context(device=device, storage=storage, scheme=scheme)
    try:
        d = ctx.domain(geo.xyz, geo.iolets, tau=0.8, ordering=ordering)
        n = d.n
        st = ctx.stream
        nvtx.range_push(f"{tag}-autotune")
        if launch is None:
            best, timing = autotune(ctx)
        else:  # a fixed shape (profiling one kernel form), no tuning
            ctx.set_launch(*launch)
            best, timing = tuple(launch), {}
        nvtx.range_pop()
        # warm-up, then the timed regions: exactly `steps` steps each, barrier + sync on both
        # sides, repeated until MIN_TIMED_S of device time has passed; the median is reported
        ctx.step(warmup)
        reps, total, n_rep = [], 0.0, 1
        nvtx.range_push(f"{tag}-timed")
        while len(reps) < n_rep:
            barrier(dist)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sampler.mark(True)
            e0.record(st)
            ctx.step(steps)
            e1.record(st)
            barrier(dist)
            sampler.mark(False)
            x = e0.elapsed_time(e1)
            reps.append(x)
            total += x
            if len(reps) == 1:  # the repetition count follows from the first measurement,
                # the same on every rank (slowest rank's count)
                n_rep = int(max_over_ranks(float(max(3, min(20000, math.ceil(min_timed_s * 1e3 / x)))),
                                           dist, device))
        nvtx.range_pop()
        ms = max_over_ranks(statistics.median(reps), dist, device)
        # per-kernel durations (CUDA events on the context stream around every launch)
        nvtx.range_push(f"{tag}-profiled")
        ms_sc, ms_io = ctx.step_profiled(steps)
        nvtx.range_pop()
        # end to end through the C ABI: host state in (pinned), `steps` steps, macroscopic out
        import ctypes as C

        state = d.save_state()
        pinned = torch.empty(state.size, dtype=torch.uint8, pin_memory=True)
        pinned.numpy()[:] = state
        out = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
        barrier(dist)
        t0 = time.perf_counter()
        d.load_state(pinned.numpy())
        ctx.step(steps)
        rc = H.lib().hg_read_macroscopic(d.h, C.c_void_p(out.data_ptr()), None)
        if rc != 0:
            raise RuntimeError("read-back failed")
        barrier(dist)
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, device)
        gs = 16
        launches = steps * (1 + (1 if geo.iolets else 0)) + (steps + gs - 1) // gs
        n_runs = d.info()["n_runs"]
        return dict(n=n, ms=ms, reps=len(reps), timed_s=total / 1e3, ms_sc=ms_sc, ms_io=ms_io,
                    n_runs=n_runs, bytes_per_update=bytes_per_update(storage, scheme, best[2], n, n_runs),
                    ordering=ordering, ordering_ms=order_ms, e2e_s=e2e_s, h2d=int(state.size),
                    d2h=int(n * 16), launches=launches, device_bytes=d.info()["device_bytes"],
                    launch={"block": best[0], "sites_per_thread": best[1], "kernel_variant": best[2]},
                    tuning_ms={f"{b}x{t}v{v}": round(x, 4) for (b, t, v), x in timing.items()})
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
    cores = oracle.num_threads()
    # one core: the same update on a seeded sample of 200k sites of the current state
    sample = np.sort(np.random.default_rng(1).choice(od.n, size=min(od.n, 200_000), replace=False))
    bc = s.bc_values(0, s.t + 1)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        od.step_sites(od.F, bc, sample)
        one_core = sample.size / (time.perf_counter() - t0) / 1e6
    finally:
        oracle.set_threads(cores)
    return {"value": od.n * steps / dt / 1e6, "unit": "MFLUPS", "cores": cores,
            "kind": "oracle", "single_core_mflups": one_core,
            "sample": f"{steps} steps over all {od.n} sites of the same tree (after 1 untimed step; "
                      f"table build {build_s:.1f} s untimed); single core: one step of "
                      f"{sample.size} seeded sites"}


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
    line = {"impl": "reference", "metric": METRIC,
            "value": v, "unit": "MFLUPS", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded tree)", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "MFLUPS", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} steps over all {od.n} sites"},
            "e2e": {"value": v, "unit": "MFLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _geo_pool_gen(args):
    """Worker (spawned process): voxelise one request's geometries."""
    from paper_2010_04144_gb300 import synth as S

    spec, coupled = args
    art = S.tree(spec, inlet_speed=0.05, period=1000.0)
    if not coupled:
        return (art,)
    ven = S.tree(spec, venous=True, venous_offset=0.0)
    return (art, ven)


def _large_tree(scale):
    """Worker (spawned process): the precision workload's tree, depth 8, root radius 40."""
    from paper_2010_04144_gb300 import synth as S

    return S.tree(S.TreeSpec(depth=8, root_radius=40.0, seed=2010041442, scale=scale),
                  inlet_speed=0.05, period=1000.0)


def serve_requests(args, pool=None):
    """The seeded request stream and its voxelised geometries (spawned host processes).  With
    a pool given, the voxelisation starts there and a callable returns the result later."""
    import multiprocessing as mp

    from paper_2010_04144_gb300 import synth as S

    reqs = S.request_stream(n_requests=args.requests, rate_per_s=args.rate,
                            sites_range=(args.min_sites, args.max_sites), steps=args.serve_steps)
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    t0 = time.perf_counter()
    pending = pool.map_async(_geo_pool_gen, [(r.spec, r.coupled) for r in reqs], chunksize=1)

    def result():
        geos = pending.get()
        if own:
            pool.close()
        return reqs, geos, time.perf_counter() - t0

    return result if not own else result()


def serve_tuning(args, H, device, reqs, geos):
    """Site ordering and launch shape of the packed (tile-table) launches serving runs: tuned
    on a context that holds the stream's first requests, as a tick would pack them."""
    from paper_2010_04144_gb300 import synth as S
    from paper_2010_04144_gb300.autotune import tune_ordering

    pack = [x for g in geos[:4] for x in g]

    def make(o):
        c = H.Context(device=device, storage=args.serve_storage, scheme=args.serve_scheme)
        for g in pack:
            c.domain(g.xyz, g.iolets, ordering=o)
        return c

    o, shape, table = tune_ordering(make, ORDERINGS if args.serve_ordering == "auto" else (args.serve_ordering,))
    return o, shape, {k: round(v[1], 4) for k, v in table.items()}, int(sum(g.n for g in pack))


def serve_stats(args, H, device, prepared=None):
    """Serving workload: seeded request stream, continuous batching, p50/p99 time-to-result."""
    from paper_2010_04144_gb300 import serve as SV
    from paper_2010_04144_gb300 import synth as S

    reqs, geos, gen_s = prepared if prepared is not None else serve_requests(args)
    ordering, shape, order_ms, tuned_sites = serve_tuning(args, H, device, reqs, geos)
    srv = SV.Server(device=device, storage=args.serve_storage, scheme=args.serve_scheme,
                    budget_bytes=args.budget_gb * 1e9, chunk_steps=100, block_size=shape[0],
                    sites_per_thread=shape[1], kernel_variant=shape[2],
                    build_workers=args.serve_build_workers, policy=args.serve_policy, ordering=ordering,
                    tick_site_steps=args.serve_tick_sites or None)
    try:
        for r, g in zip(reqs, geos):
            if r.coupled:
                job = SV.coupled_job_from_trees(r.rid, r.arrival_s, r.steps, g[0], g[1],
                                                S.uniform_draws(r.rid + 7919, len(g[1].iolets)))
            else:
                job = SV.Job(rid=r.rid, arrival_s=r.arrival_s, steps=r.steps, geoms=[g[0]])
            srv.submit(job)
        srv.run()
        st = srv.stats()
    finally:
        srv.close()
    sites = [sum(x.n for x in g) for g in geos]
    offered = sum(sites) * args.serve_steps / (reqs[-1].arrival_s or 1.0) / 1e6
    # the request rate the measured aggregate throughput sustains (meaningful when the stream
    # saturates the server, i.e. offered > aggregate): throughput / mean work per request
    mean_work = sum(sites) * args.serve_steps / len(sites) / 1e6
    st["max_sustainable_rate_per_s"] = st["aggregate_mflups"] / mean_work
    st["saturated"] = offered > st["aggregate_mflups"]
    cfg = {"workload": f"first {len(reqs)} of the seeded 256-request stream (Poisson {args.rate}/s, "
                       f"sites log-uniform [{args.min_sites:.0e}, {args.max_sites:.0e}], half coupled "
                       f"pairs, {args.serve_steps} steps each)",
           "budget_gb": args.budget_gb, "tick_steps": 100, "tick_site_steps": args.serve_tick_sites or None,
           "scheme": args.serve_scheme,
           "storage": args.serve_storage, "ordering": ordering, "ordering_ms": order_ms,
           "launch": list(shape), "launch_tuned_on_sites": tuned_sites,
           "build_workers": args.serve_build_workers, "policy": args.serve_policy,
           "total_sites": int(sum(sites)), "offered_mflups": offered, "geometry_generation_s": gen_s}
    return st, cfg


def run_serve(args, H, device, prepared=None):
    st, cfg = serve_stats(args, H, device, prepared)
    line = {"metric": "served time-to-result p50/p99 (s) and aggregate MFLUPS", "value": st["p50_s"],
            "unit": "s (p50 time-to-result)", "p99_s": st["p99_s"], "higher_is_better": False,
            "aggregate_mflups": st["aggregate_mflups"], "n_gpus": 1,
            "dtype": args.serve_storage + "-stored/f32-compute", "data": "synthetic (seeded request stream)",
            "config": cfg, "serving": st}
    print(json.dumps(line))


def run_coupled(args, H, device):
    """Coupled pair: arterial tree and its venous twin stepped in the same launches."""
    import torch

    from paper_2010_04144_gb300 import synth as S
    from paper_2010_04144_gb300.autotune import autotune

    from paper_2010_04144_gb300 import serve as SV

    spec = S.TreeSpec(depth=6, root_radius=24.0, seed=2010041442, scale=args.coupled_scale)
    art = S.tree(spec, inlet_speed=0.05, period=1000.0)
    one_to_n = args.coupled_venous_depth > 0
    if one_to_n:  # an independent, deeper venous tree: the greedy 1:N map couples by proximity
        vspec = S.TreeSpec(depth=args.coupled_venous_depth, root_radius=24.0, seed=2010041443,
                           scale=args.coupled_scale)
        ven = S.tree(vspec, venous=True)
    else:
        ven = S.tree(spec, venous=True)
    ctx = H.Context(device=device, storage="f32", scheme=args.coupled_scheme)
    try:
        da = ctx.domain(art.xyz, art.iolets, ordering=args.coupled_ordering)
        dv = ctx.domain(ven.xyz, ven.iolets, ordering=args.coupled_ordering)
        if one_to_n:
            u = S.uniform_draws(2010041444, len(ven.iolets))
            pairs = SV.coupled_job_from_trees(0, 0.0, 0, art, ven, u).pairs
        else:
            pairs = []
            for k in range(1, len(art.iolets)):  # mirrored leaf k feeds venous inlet k (1:1 map)
                _, _, _, f = H.hg_coupling_factors([art.iolets[k].centre], [art.iolets[k].area()],
                                                   [ven.iolets[k].centre], [ven.iolets[k].area()], [0.5])
                pairs.append((k, k, float(f[0])))
        ctx.couple(da, dv, pairs)
        ctx.set_coupling_mode(args.coupled_mode)
        best, _ = autotune(ctx)
        # let the inlet's wave reach every outlet (and the coupled inlets) before timing
        ctx.step(args.coupled_settle)
        ctx.step(args.warmup)
        barrier(None)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        ctx.step(args.steps)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ms_sc, ms_io = ctx.step_profiled(min(args.steps, 200))
        n = da.n + dv.n
        B = domain_bytes(ctx, "f32", args.coupled_scheme, [da, dv])
        per = ms_sc / min(args.steps, 200)
        peak, kind = hbm_peak()
        Mv = dv.iolet_stats()
        Ma = da.iolet_stats()
        # the venous inlets' next boundary values against factor x source outlet mean (exact up to
        # FP32 rounding), and the venous inlet flow they produce against the same product
        bv = dv.boundary_values()
        forces = da.iolet_forces()
        vva = {}
        if args.velocity_area:  # Section 3.3's speed-against-vessel-area plot, per tree level
            from paper_2010_04144_gb300 import analysis as AN

            for name, d, g in (("arterial", da, art), ("venous", dv, ven)):
                fields, sites = d.macroscopic(), d.sites()
                rows = AN.velocity_vs_area(g, fields, sites, arterial_negative=name == "arterial")
                lvl = np.floor(np.log2(rows[:, 0] + 1)).astype(int)
                vva[name] = [[int(L), float(np.median(rows[lvl == L, 1])), float(np.median(rows[lvl == L, 2])),
                              int((lvl == L).sum())] for L in np.unique(lvl)]
                # the paper's own cut: planes at 1/4, 1/2, 3/4 of the domain, one row per vessel
                planes = AN.velocity_vs_area_planes(fields, sites, arterial_negative=name == "arterial")
                vva[name + "_planes"] = [[float(r[0]), float(r[2]), float(r[3])] for r in planes]
        devs = [abs(abs(float(bv[vk])) / abs(f * Ma[ak, 0]) - 1.0) for ak, vk, f in pairs if Ma[ak, 0]]
        bc_dev = max(devs) if devs and args.coupled_mode == "forward" else None  # alternate: may hold
        ratio = [float(abs(Mv[vk, 0]) / abs(f * Ma[ak, 0])) for ak, vk, f in pairs if Ma[ak, 0]]
        fan = np.bincount([ak for ak, _, _ in pairs])
        line = {"metric": "MFLUPS, coupled arterial+venous pair in one launch sequence",
                "value": n * args.steps / (ms / 1e3) / 1e6, "unit": "MFLUPS", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded tree pair)",
                "config": {"workload": (f"arterial tree d=6 R=24x{args.coupled_scale} + "
                                        + (f"independent venous tree d={args.coupled_venous_depth} "
                                           f"(radii x1.2), greedy 1:N map" if one_to_n
                                           else "venous twin (radii x1.2), 1:1 map")),
                           "arterial_sites": da.n, "venous_sites": dv.n, "pairs": len(pairs),
                           "arterial_outlets": len(art.iolets) - 1, "venous_inlets": len(ven.iolets) - 1,
                           "fan_out_max": int(fan.max()), "fan_out_min": int(fan[1:].min()),
                           "factor_range": [min(p[2] for p in pairs), max(p[2] for p in pairs)],
                           "scheme": args.coupled_scheme, "exchange": args.coupled_mode,
                           "ordering": args.coupled_ordering, "n_runs": [da.info()["n_runs"], dv.info()["n_runs"]],
                           "settle_steps": args.coupled_settle,
                           "launch": {"block": best[0], "sites_per_thread": best[1], "kernel_variant": best[2]}},
                "roofline": {"bound": "hbm", "achieved": B * n / (per / 1e3) / 1e9, "peak": peak,
                             "unit": "GB/s", "frac": B * n / (per / 1e3) / 1e9 / peak,
                             "bytes_per_update": B},
                "iolet_update_ms": ms_io / min(args.steps, 200),
                "boundary_value_rel_dev_max": bc_dev,
                "arterial_outlet_force_max": float(np.abs(forces).max()),
                "velocity_vs_area_by_level": vva or None,
                "venous_inlet_flow_over_imposed": ([min(ratio), float(np.median(ratio)), max(ratio)]
                                                   if ratio else None),
                "outlets_with_flow": len(ratio)}
        print(json.dumps(line))
    finally:
        ctx.close()


def run_split(args, H, device):
    """Split domain (Section 2.2 decomposition, halo exchange every step) on one device:
    the whole hot path plus the exchange of the crossing populations (direct, or staged as
    pack / copy / unpack), against the same domain unsplit, every partition's sites in the
    unsplit domain's tuned ordering; results are bit-identical, so only the time differs."""
    import torch

    from paper_2010_04144_gb300.autotune import autotune, autotune_split, tune_ordering

    geo, cfg = workload(scale=args.scale)
    rows = []
    launch = None
    tuned = {}
    ordering = args.split_ordering
    if ordering == "auto":  # the unsplit domain's best ordering, used by every partition too
        def make(o):
            c = H.Context(device=device, storage="f32", scheme="ab")
            c.domain(geo.xyz, geo.iolets, ordering=o)
            return c
        ordering, _, _ = tune_ordering(make, ORDERINGS)
    runs = [(0, None)] + [(int(x), ex) for x in args.parts.split(",") for ex in args.split_exchange.split(",")]
    for k, ex in runs:
        ctx = H.Context(device=device, storage="f32", scheme="ab")
        try:
            if k == 0:
                obj = ctx.domain(geo.xyz, geo.iolets, ordering=ordering)
                if args.split_launch:
                    b, rest = args.split_launch.split("x")
                    launch = (int(b), *[int(x) for x in rest.split("v")])
                    ctx.set_launch(*launch)
                else:
                    launch, _ = autotune(ctx)
            else:
                obj = ctx.split(geo.xyz, geo.iolets, k, boundary_weight=args.boundary_weight, ordering=ordering,
                                exchange=ex)
                if args.split_launch:
                    ctx.set_launch(*launch)
                    split_shape = launch
                elif (k, "shape") in tuned:   # the other transport reuses the shape tuned for k
                    split_shape = tuned[(k, "shape")]
                    ctx.set_launch(*split_shape)
                else:
                    split_shape, _ = autotune_split(ctx, obj)
                    tuned[(k, "shape")] = split_shape
            obj.step(args.warmup) if k else ctx.step(args.warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            obj.step(args.steps) if k else ctx.step(args.steps)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            halo = sum(obj.info(p)["halo_in"] for p in range(k)) if k else 0
            ghosts = sum(obj.info(p)["ghosts"] for p in range(k)) if k else 0
            rows.append({"parts": k, "exchange": ex, "ms_per_step": ms, "mflups": geo.n / (ms / 1e3) / 1e6,
                         "halo_values_per_step": halo, "ghost_sites": ghosts,
                         "launch": list(launch if k == 0 else split_shape)})
        finally:
            ctx.close()
    base = rows[0]["ms_per_step"]
    for r in rows:
        r["time_vs_unsplit"] = r["ms_per_step"] / base
    last = [r for r in rows if r["parts"] == rows[-1]["parts"]]
    line = {"metric": METRIC, "value": max(r["mflups"] for r in last), "unit": "MFLUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (seeded tree geometry, rest initial state)",
            "config": {**cfg, "steps_per_job": args.steps, "storage": "f32", "scheme": "ab",
                       "launch": list(launch), "ordering": ordering,
                       "split": "contiguous Morton ranges, each partition's sites in the device ordering; "
                                "halo exchange every step on one device (direct: one kernel; staged: "
                                "pack, one copy per partition pair, unpack)",
                       "boundary_weight": args.boundary_weight},
            "split": rows}
    print(json.dumps(line))


def time_large(args, H, device, geo, results):
    """The precision workload's ~77M-site tree in the 32- and 16-bit forms, each with the
    ordering and launch shape the ~10M-site tuning chose for it: MFLUPS of the whole step
    and the stream-collide kernel's fraction of its HBM roofline."""
    import torch

    peak, _ = hbm_peak()
    out = {}
    for key in (("f32", "ab"), ("f32", "aa"), ("f16", "ab"), ("f16", "aa")):
        if key not in results:
            continue
        r = results[key]
        storage, scheme = key
        ctx = H.Context(device=device, storage=storage, scheme=scheme)
        try:
            d = ctx.domain(geo.xyz, geo.iolets, ordering=r["ordering"])
            L = r["launch"]
            ctx.set_launch(L["block"], L["sites_per_thread"], L["kernel_variant"])
            ctx.step(args.warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = 64
            e0.record(ctx.stream)
            ctx.step(k)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            ms_sc, _ = ctx.step_profiled(16)
            B = domain_bytes(ctx, storage, scheme, [d])
            out[f"{storage}:{scheme}"] = {"mflups": d.n / (ms / 1e3) / 1e6, "ms_per_step": ms,
                                          "bytes_per_update": B,
                                          "roofline_frac": B * d.n / (ms_sc / 16 / 1e3) / 1e9 / peak,
                                          "ordering": r["ordering"], "launch": L,
                                          "device_gb": d.info()["device_bytes"] / 1e9}
        finally:
            ctx.close()
    return {"workload": f"tree d=8 R=40x{args.large_scale} seed=2010041442", "fluid_sites": geo.n,
            "steps": 64, "forms": out}


def run_precision(args, H, device):
    """FP32 vs FP16 vs BF16 storage: throughput on the large tree, error vs the FP64 oracle."""
    import torch

    from paper_2010_04144_gb300 import synth as S
    from paper_2010_04144_gb300.autotune import autotune

    spec = S.TreeSpec(depth=8, root_radius=40.0, seed=2010041442, scale=args.precision_scale)
    geo = S.tree(spec, inlet_speed=0.05, period=1000.0)
    peak, kind = hbm_peak()
    out = {}
    for storage, scheme in (("f32", "ab"), ("f32", "aa"), ("f16", "aa"), ("bf16", "aa")):
        ctx = H.Context(device=device, storage=storage, scheme=scheme)
        try:
            d = ctx.domain(geo.xyz, geo.iolets, ordering="rows")
            best, _ = autotune(ctx)
            ctx.step(args.warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            ctx.step(args.steps)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ms_sc, _ = ctx.step_profiled(min(args.steps, 100))
            B = domain_bytes(ctx, storage, scheme, [d])
            per = ms_sc / min(args.steps, 100)
            out[f"{storage}:{scheme}"] = {"mflups": d.n * args.steps / (ms / 1e3) / 1e6,
                                          "roofline_frac": B * d.n / (per / 1e3) / 1e9 / peak,
                                          "launch": list(best), "device_gb": d.info()["device_bytes"] / 1e9}
        finally:
            ctx.close()
    err = {}
    if not args.no_cpu_baseline:
        import oracle

        small = S.tree(S.TreeSpec(depth=8, root_radius=40.0, seed=2010041442, scale=args.error_scale),
                       inlet_speed=0.05, period=1000.0)
        od = oracle.Domain(small.xyz, small.iolets, tau=0.8)
        oracle.System([od]).step(args.error_steps)
        ref = od.moments()
        for storage in ("f32", "f16", "bf16"):
            ctx = H.Context(device=device, storage=storage, scheme="aa")
            try:
                d = ctx.domain(small.xyz, small.iolets)
                ctx.step(args.error_steps)
                m = d.macroscopic().astype(np.float64)
                eu = float(np.linalg.norm(m[:, 1:] - ref[:, 1:]) / np.linalg.norm(ref[:, 1:]))
                ep = float(np.linalg.norm(m[:, 0] - ref[:, 0]) / np.linalg.norm(ref[:, 0]))
                err[storage] = {"velocity_rel_l2": eu, "pressure_rel_l2": ep}
            finally:
                ctx.close()
        err["instance"] = f"d=8 R=40x{args.error_scale} ({small.n} sites), {args.error_steps} steps"
    line = {"metric": "MFLUPS and HBM-roofline fraction, FP32 vs FP16/BF16-stored",
            "value": out["f16:aa"]["mflups"], "unit": "MFLUPS (f16:aa)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f16-stored/f32-compute", "data": "synthetic (seeded tree)",
            "config": {"workload": f"tree d=8 R=40x{args.precision_scale}", "fluid_sites": geo.n},
            "variants": out, "error_vs_fp64_oracle": err}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="hemegb", choices=["hemegb", "reference"])
    ap.add_argument("--scale", type=float, default=1.71)
    ap.add_argument("--variants", default="f32:ab,f32:aa,f16:ab,f16:aa,bf16:aa",
                    help="storage:scheme list; append @BLOCKxSPTvVARIANT to fix a launch shape")
    ap.add_argument("--headline", default="f32:best")
    ap.add_argument("--min-timed-s", type=float, default=MIN_TIMED_S,
                    help="device time each variant's repeated K-step measurement covers (0: three)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default="tree", choices=["tree", "coupled", "precision", "serve", "split"])
    ap.add_argument("--parts", default="2,4,8", help="split config: partition counts to time")
    ap.add_argument("--split-ordering", default="auto",
                    help="split config: auto (the unsplit domain's tuned ordering) or morton / rows / bricks")
    ap.add_argument("--split-exchange", default="direct,staged",
                    help="split config: halo transports to time (direct, staged)")
    ap.add_argument("--split-launch", default="", help="split config: fixed launch BLOCKxSPTvVARIANT (no tuning)")
    ap.add_argument("--boundary-weight", type=float, default=1.0,
                    help="split config: load-balancing cost of a site next to an iolet")
    ap.add_argument("--coupled-scale", type=float, default=2.12)
    ap.add_argument("--coupled-scheme", default="ab")
    ap.add_argument("--coupled-ordering", default="rows",
                    help="coupled config: device site ordering of both trees (the ~10M-site tree tunes to rows)")
    ap.add_argument("--coupled-settle", type=int, default=4000,
                    help="untimed steps before the coupled timing, so flow reaches the outlets")
    ap.add_argument("--velocity-area", action="store_true",
                    help="coupled config: add mean speed vs vessel area per tree level (Section 3.3)")
    ap.add_argument("--coupled-mode", default="forward", choices=["forward", "alternate"],
                    help="coupling exchange: forward every step, or alternating forward/reverse (Guo force)")
    ap.add_argument("--coupled-venous-depth", type=int, default=0,
                    help="0: mirrored venous twin, 1:1 pairs; d > 6: independent venous tree of depth d "
                         "coupled by the greedy 1:N map")
    ap.add_argument("--precision-scale", type=float, default=1.84)
    ap.add_argument("--error-scale", type=float, default=0.54)
    ap.add_argument("--error-steps", type=int, default=500)
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--min-sites", type=float, default=5e4)
    ap.add_argument("--max-sites", type=float, default=4e7)
    ap.add_argument("--serve-steps", type=int, default=2000)
    ap.add_argument("--serve-storage", default="f16")
    ap.add_argument("--serve-scheme", default="aa")
    ap.add_argument("--serve-tick-sites", type=float, default=3e8,
                    help="serving: site updates each request advances per tick, in steps of 100 x a power "
                         "of two (0: 100 steps for every request)")
    ap.add_argument("--serve-ordering", default="auto", help="auto (tuned) or morton / rows / bricks")
    ap.add_argument("--serve-policy", default="fifo", choices=["fifo", "backfill"])
    ap.add_argument("--serve-build-workers", type=int, default=4,
                    help="0: build admitted requests inline between ticks; k: on k worker threads")
    ap.add_argument("--budget-gb", type=float, default=180.0)
    ap.add_argument("--large-scale", type=float, default=1.84,
                    help="tree config: scale of the ~77M-site precision tree timed beside the headline "
                         "(0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="tree config: the first k requests of the serving stream, served beside the "
                         "headline (0 skips them)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.config != "tree":
        # single-device workloads: under a multi-rank launch rank 0 runs them on its own
        # device and the other ranks exit without work
        if int(os.environ.get("RANK", "0")) != 0:
            return
        import torch

        from paper_2010_04144_gb300 import hemegb as H

        H.lib()
        device = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(device)
        return {"coupled": run_coupled, "precision": run_precision, "serve": run_serve,
                "split": run_split}[args.config](args, H, device)

    import torch

    from paper_2010_04144_gb300 import hemegb as H

    H.lib()
    rank, ws, local, dist = dist_setup()
    device = local
    torch.cuda.set_device(device)
    extra_pool = large_pending = serve_pending = None
    if rank == 0 and ws == 1 and (args.large_scale > 0 or args.serve_requests > 0):
        # host-side geometry for the large-domain and serving legs, voxelised meanwhile
        import multiprocessing as mp

        extra_pool = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
        if args.large_scale > 0:
            large_pending = extra_pool.apply_async(_large_tree, (args.large_scale,))
        if args.serve_requests > 0:
            sargs = argparse.Namespace(**vars(args))
            sargs.requests = args.serve_requests
            serve_pending = serve_requests(sargs, pool=extra_pool)
    geo, cfg = workload(scale=args.scale)
    cfg["steps_per_job"] = args.steps
    peak, peak_kind = hbm_peak()
    variants = []
    for v in args.variants.split(","):  # "storage:scheme", optionally "@BLOCKxSPTvVARIANT" (no tuning)
        form, _, shape = v.partition("@")  # and "/ORDERING" after the shape (no ordering tuning)
        shape, _, order = shape.partition("/")
        launch = None
        if shape:
            b, rest = shape.split("x")
            spt, var = rest.split("v")
            launch = (int(b), int(spt), int(var))
        variants.append((*form.split(":"), launch, (order,) if order else ORDERINGS))
    results = {}
    sampler = ClockSampler(device).start()
    try:
        for (storage, scheme, launch, orders) in variants:
            r = time_variant(H, geo, storage, scheme, args.steps, args.warmup, dist, device, sampler,
                             launch=launch, orderings=orders if launch is None else (orders[0],),
                             min_timed_s=args.min_timed_s)
            B = r["bytes_per_update"]
            r["mflups"] = r["n"] * ws * args.steps / (r["ms"] / 1e3) / 1e6
            r["achieved_gbs"] = B * r["n"] / (r["ms_sc"] / args.steps / 1e3) / 1e9
            results[(storage, scheme)] = r
    finally:
        sampler.stop()
    if args.headline == "f32:best":
        f32 = [k for k in results if k[0] == "f32"]
        head = max(f32, key=lambda k: results[k]["mflups"]) if f32 else next(iter(results))
    else:
        head = tuple(args.headline.split(":"))
    h = results[head]
    total_sites = h["n"] * ws
    value = whole_job_mflups(h["n"], ws, args.steps, h["ms"])
    e2e_value = total_sites * args.steps / h["e2e_s"] / 1e6
    traffic, scaled_from = profiled_traffic(f"{head[0]}:{head[1]}", h["launch"], h["ordering"])
    line = {
        "metric": METRIC,
        "value": value, "unit": "MFLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[head[0]],
        "data": "synthetic (seeded tree geometry, rest initial state)",
        "config": {**cfg, "storage": head[0], "scheme": head[1], "launch": h["launch"],
                   "ordering": h["ordering"],
                   "timing": f"median of {h['reps']} back-to-back {args.steps}-step measurements "
                             f"({h['timed_s']:.2f} s of device time)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": h["achieved_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": h["achieved_gbs"] / peak, "traffic": traffic,
                     "traffic_note": scaled_from,
                     "kernel": "k_stream_collide_one (single-domain stream-collide)",
                     "bytes_per_update": h["bytes_per_update"],
                     "launch_ms": h["ms_sc"] / args.steps,
                     "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
        "e2e": {"value": e2e_value, "unit": "MFLUPS",
                "h2d_bytes_per_step": h["h2d"] / args.steps,
                "d2h_bytes_per_step": h["d2h"] / args.steps,
                "job": "hg_load_state(pinned host) + steps + hg_read_macroscopic(host)"},
        "gpu_launches": h["launches"] * h["reps"],
        "gpu_launches_per_measurement": h["launches"],
        "clocks": sampler.summary(),
        "variants": {f"{s}:{c}": {"mflups": r["mflups"], "achieved_gbs": r["achieved_gbs"],
                                   "roofline_frac": r["achieved_gbs"] / peak,
                                   "bytes_per_update": r["bytes_per_update"], "n_runs": r["n_runs"],
                                   "stream_collide_ms": r["ms_sc"] / args.steps,
                                   "iolet_update_ms": r["ms_io"] / args.steps,
                                   "launch": r["launch"], "ordering": r["ordering"],
                                   "ordering_ms": r["ordering_ms"], "tuning_ms": r["tuning_ms"],
                                   "device_bytes": r["device_bytes"]}
                     for (s, c), r in results.items()},
    }
    if large_pending is not None:
        line["large_domain"] = time_large(args, H, device, large_pending.get(), results)
    if serve_pending is not None:
        st, scfg = serve_stats(sargs, H, device, prepared=serve_pending())
        line["serving"] = {"p50_s": st.get("p50_s"), "p99_s": st.get("p99_s"),
                           "aggregate_mflups": st["aggregate_mflups"], "requests": st["requests"],
                           "elapsed_s": st["elapsed_s"], "peak_hbm_gb": st["peak_hbm_gb"],
                           "max_sustainable_rate_per_s": st["max_sustainable_rate_per_s"],
                           "saturated": st["saturated"], "config": scfg}
    if extra_pool is not None:
        extra_pool.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(geo)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
