"""Continuous-batching server for LB simulation requests.

A request is one seeded vascular geometry (or a coupled arterial/venous pair)
to be advanced a given number of steps.  The server keeps every admitted
request's distributions resident in HBM and advances all of them together:
each tick is one hg_step_domains call, i.e. one stream-collide launch per step
whose tile table spans every active domain (plus one iolet-update launch),
captured as a CUDA graph per active set.  With tick_site_steps, a tick gives every
request about the same number of site updates instead of the same step count (one
hg_step_domains call per step count), so small requests are not paced by large ones.  Requests that arrive while others
run are admitted, first come first served, as soon as their estimated HBM
footprint fits the budget (policy "fifo"); policy "backfill" also lets a
later request start early when it cannot delay the blocked head (EASY
backfilling on memory, counted in ticks).  Their host-side build (site order, neighbour
table, upload) runs on worker threads while the GPU keeps executing ticks;
a built request joins the active set at the next tick boundary, so builds
never stall the GPU.  Finished requests are read back and retired, freeing
their memory for the queue.

Time-to-result of a request = completion time - arrival time.  Each domain's
arithmetic does not depend on which other domains share its launches, so a
request's result is bit-identical alone and in any mix (tested).
"""
from __future__ import annotations

import math
import time
from concurrent.futures import FIRST_COMPLETED, ThreadPoolExecutor, wait
from dataclasses import dataclass, field

import numpy as np

from . import hemegb as H

# bytes per stored distribution value
_STATE_BYTES = {0: 4, 1: 2, 2: 2}


def adjacent_bound(radius):
    """Upper bound on the fluid sites with a link into one iolet opening of the given radius
    (lattice units).  Such a site lies within sqrt(2) of a point of the opening, which is a
    disc of that radius extended at most 2 units beyond the cut plane: the sites lie in a
    cylinder of radius r + sqrt(2) and length 2 + 2 sqrt(2), and a convex body holds at most
    as many lattice points as the volume of its dilation by sqrt(3)/2."""
    return math.pi * (radius + 3.0) ** 2 * 7.0


def footprint_bytes(n_sites, storage, scheme, n_iolets=2, iolet_radii=None, reordered=False):
    """Upper bound on the HBM bytes of one domain before it is built: distributions,
    neighbour table, iolet mask and prefix per site; the table's run encoding where it is
    built (4 bytes per site plus at most 16 bytes per site of run offsets); moments, link
    codes, link coefficients and site index per boundary slot (164 B) plus one list entry
    per (site, iolet) pair; per-iolet values; the two site permutations of a reordered
    layout; and the 256-byte rounding of each buffer.  With the iolet radii the boundary slots are bounded per iolet
    (adjacent_bound); without them 5% of the sites is assumed."""
    np_ = max(128, (n_sites + 127) // 128 * 128)
    copies = 2 if scheme == H.SCHEME["ab"] else 1
    per_site = 19 * _STATE_BYTES[storage] * copies + 72 + 0.25 + (8 if reordered else 0) + 20 + 4 / 1024
    if iolet_radii is not None:
        pairs = min(18 * n_sites, sum(adjacent_bound(r) for r in iolet_radii))
        adjacent = min(n_sites, pairs)
        n_iolets = len(iolet_radii)
    else:
        adjacent = pairs = 0.05 * n_sites
    return int(per_site * np_ + 164 * adjacent + 4 * pairs + 64 * n_iolets + 20 * 256 + 4 * 4096)


def geometry_footprint(geo, storage, scheme, reordered=False):
    """footprint_bytes of a seeded geometry, with its iolets' radii."""
    return footprint_bytes(geo.n, storage, scheme, iolet_radii=[io.radius / 1024.0 for io in geo.iolets],
                           reordered=reordered)


@dataclass
class Job:
    rid: int
    arrival_s: float
    steps: int
    geoms: list                       # [geometry] or [arterial, venous]
    pairs: list = field(default_factory=list)  # (src_iolet, dst_iolet, factor), art -> ven
    tau: float = 0.8
    want_fields: bool = False
    want_state: bool = False
    # filled by the server
    domains: list = field(default_factory=list)
    admitted_s: float = math.nan
    start_tick: int = -1                # tick count when the request joined the active set
    finished_s: float = math.nan
    done_steps: int = 0
    bytes: int = 0
    result: dict = field(default_factory=dict)
    cancelled: bool = False

    @property
    def sites(self):
        return sum(g.n for g in self.geoms)

    @property
    def time_to_result(self):
        return self.finished_s - self.arrival_s


class Server:
    """FIFO continuous-batching server on one GPU."""

    def __init__(self, device=0, storage="f16", scheme="aa", budget_bytes=180e9, chunk_steps=100,
                 block_size=0, sites_per_thread=0, kernel_variant=None, graph_steps=0,
                 build_workers=1, policy="fifo", ordering="morton", tick_site_steps=None):
        st = H.STORAGE[storage] if isinstance(storage, str) else storage
        sc = H.SCHEME[scheme] if isinstance(scheme, str) else scheme
        if kernel_variant is None:
            kernel_variant = 1 if st != 0 else 0
            if kernel_variant and not sites_per_thread:
                sites_per_thread, block_size = 2, block_size or 128
        self.ctx = H.Context(device=device, storage=st, scheme=sc, block_size=block_size,
                             sites_per_thread=sites_per_thread, kernel_variant=kernel_variant,
                             graph_steps=graph_steps)
        self.storage, self.scheme = st, sc
        self.ordering = ordering          # device site layout of every request's domains
        self.budget = float(budget_bytes)
        self.chunk = int(chunk_steps)
        # None: every active request advances chunk_steps per tick (the same step count);
        # a number: each request advances about tick_site_steps site updates per tick,
        # chunk_steps x a power of two, at least chunk_steps, at most what it has left, so a
        # small request finishes in few ticks instead of pacing at the big ones' rate
        self.tick_site_steps = None if tick_site_steps is None else float(tick_site_steps)
        self.queue: list[Job] = []
        self.building: list[tuple[Job, object]] = []   # (job, future) in admission order
        self.active: list[Job] = []
        self.finished: list[Job] = []
        self.failed: list[Job] = []       # requests whose build failed (result holds the error)
        self.estimate_exceeded = 0        # built domains larger than their footprint estimate
        self.max_overshoot_bytes = 0
        self._now = None
        self.in_use = 0
        self.peak_in_use = 0
        self.admit_order: list[int] = []
        self.site_steps = 0
        self.ticks = 0
        if policy not in ("fifo", "backfill"):
            raise ValueError("policy must be 'fifo' or 'backfill'")
        self.policy = policy
        self.backfilled = 0
        self.build_s = 0.0        # host time spent building domains (worker or inline)
        self.wait_s = 0.0         # main-thread time blocked on the GPU
        self.idle_s = 0.0         # main-thread time with nothing to step
        # build_workers threads: hg_domain_create calls may overlap one another (their
        # serial phases then share the host cores); activation stays in admission order
        self._pool = ThreadPoolExecutor(max_workers=int(build_workers)) if build_workers else None

    # ---- admission -------------------------------------------------------------
    def submit(self, job: Job):
        if job.steps % self.chunk:
            raise ValueError("a request's step count must be a multiple of the tick size")
        need = self._estimate(job)
        if need > self.budget:
            raise ValueError(f"request {job.rid} needs {need / 1e9:.1f} GB, above the budget")
        self.queue.append(job)

    def cancel(self, rid):
        for j in list(self.queue):
            if j.rid == rid:
                j.cancelled = True
                self.queue.remove(j)
                return True
        for j, _ in self.building:
            if j.rid == rid:
                j.cancelled = True    # released when its build completes
                return True
        for j in list(self.active):
            if j.rid == rid:
                j.cancelled = True
                self._retire(j, read=False)
                return True
        return False

    def _estimate(self, job):
        return sum(geometry_footprint(g, self.storage, self.scheme, reordered=self.ordering != "morton")
                   for g in job.geoms)

    def _build(self, job):
        """Host build and upload of a job's domains (worker thread; touches no server state)."""
        t = time.perf_counter()
        doms = []
        try:
            for g in job.geoms:
                doms.append(self.ctx.domain(g.xyz, g.iolets, tau=job.tau, ordering=self.ordering))
        except Exception as e:  # noqa: BLE001 -- handed to the main thread
            return doms, e, time.perf_counter() - t
        return doms, None, time.perf_counter() - t

    def _admit(self, now_s):
        """Reserve memory for arrived queue heads and start their builds; with the backfill
        policy, then let later arrivals that cannot delay the head go ahead of it."""
        while self.queue and self.queue[0].arrival_s <= now_s:
            job = self.queue[0]
            if self.in_use + self._estimate(job) > self.budget:
                break  # the head waits for memory
            self.queue.pop(0)
            self._start(job, now_s)
        if self.policy == "backfill" and self.queue and self.queue[0].arrival_s <= now_s:
            self._backfill(now_s)

    def _ticks_left(self, job):
        left = job.steps - job.done_steps
        return -(-left // self._tick_steps(job)) if left > 0 else 0

    def _tick_steps(self, job):
        """Steps the request advances in its next tick."""
        left = job.steps - job.done_steps
        if self.tick_site_steps is None:
            return min(self.chunk, left)
        n = max(1, sum(g.n for g in job.geoms))
        k = self.chunk
        while k * 2 <= left and 2 * k * n <= self.tick_site_steps:
            k *= 2
        return min(k, left)

    def _backfill(self, now_s):
        """EASY backfilling on memory, counted in ticks: the blocked head's start (its shadow
        tick) is when enough resident requests have retired; a later request may start now if it
        fits and either finishes by the shadow tick or fits in the memory the head leaves spare."""
        head = self.queue[0]
        free = self.budget - self.in_use
        need = self._estimate(head)
        holders = [(self._ticks_left(j), j.bytes) for j in self.active]
        holders += [(self._ticks_left(j) + 1, j.bytes) for j, _ in self.building]  # +1: the build
        holders.sort()
        shadow, extra, freed = None, 0.0, 0.0
        for ticks, b in holders:
            freed += b
            if free + freed >= need:
                shadow, extra = ticks, free + freed - need
                break
        if shadow is None:
            return
        for job in list(self.queue[1:]):
            if job.arrival_s > now_s:
                break
            m = self._estimate(job)
            if self.in_use + m > self.budget:
                continue
            done_by_shadow = self._ticks_left(job) + 1 <= shadow
            if not done_by_shadow and m > extra:
                continue
            if not done_by_shadow:
                extra -= m
            self.queue.remove(job)
            self.backfilled += 1
            self._start(job, now_s)

    def _start(self, job, now_s):
        """Reserve the request's estimated memory and start its build."""
        job.bytes = self._estimate(job)
        self.in_use += job.bytes
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        job.admitted_s = now_s
        self.admit_order.append(job.rid)
        if self._pool is not None:
            self.building.append((job, self._pool.submit(self._build, job)))
        else:
            self.building.append((job, _Done(self._build(job))))

    def _activate(self, block=False, timeout=None):
        """Move completed builds into the active set (with several build workers a later
        admission may be ready first and joins at once); with block, wait for one first."""
        if block and self.building and not any(f.done() for _, f in self.building):
            t = time.perf_counter()
            wait([f for _, f in self.building], timeout=timeout, return_when=FIRST_COMPLETED)
            self.idle_s += time.perf_counter() - t
        joined = []
        while any(f.done() for _, f in self.building):
            i = next(k for k, (_, f) in enumerate(self.building) if f.done())
            job, fut = self.building.pop(i)
            doms, err, secs = fut.result()
            self.build_s += secs
            if err is None and job.pairs and not job.cancelled:
                try:
                    self.ctx.couple(doms[0], doms[1], job.pairs)
                except H.HgError as e:
                    err = e
            if err is not None or job.cancelled:
                for d in doms:
                    d.destroy()
                self.in_use -= job.bytes
                if err is not None:  # this request fails alone; the server keeps serving
                    job.result = {"error": f"{type(err).__name__}: {err}"}
                    job.finished_s = self._now() if self._now else math.nan
                    self.failed.append(job)
                continue
            self.in_use -= job.bytes
            job.domains = doms
            estimate, job.bytes = job.bytes, sum(d.info()["device_bytes"] for d in doms)
            if job.bytes > estimate:  # counted; admissions wait until in_use is back in budget
                self.estimate_exceeded += 1
                self.max_overshoot_bytes = max(self.max_overshoot_bytes, job.bytes - estimate)
            self.in_use += job.bytes
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            job.start_tick = self.ticks
            self.active.append(job)
            joined.append(job)
        return joined

    def _retire(self, job, read=True, now_s=None):
        if read:
            res = {"iolet_stats": [d.iolet_stats() for d in job.domains],
                   "mass": [d.mass() for d in job.domains], "steps": job.done_steps}
            if job.want_fields:
                res["fields"] = [d.macroscopic() for d in job.domains]
            if job.want_state:
                res["state"] = [d.state() for d in job.domains]
            job.result = res
        for d in job.domains:
            d.destroy()
        job.domains = []
        self.in_use -= job.bytes
        self.active.remove(job)
        if read:
            job.finished_s = now_s
            self.finished.append(job)

    # ---- main loop -------------------------------------------------------------
    def run(self, clock=time.perf_counter, sleep=time.sleep, max_ticks=None):
        """Serve every submitted job; returns the finished jobs."""
        t0 = clock()
        self._now = lambda: clock() - t0
        self.queue.sort(key=lambda j: (j.arrival_s, j.rid))
        while self.queue or self.active or self.building:
            self._activate()
            self._admit(clock() - t0)
            if self.active:
                ticking = list(self.active)
                if self.tick_site_steps is None:  # one step count for every request
                    k = min(self.chunk, min(j.steps - j.done_steps for j in ticking))
                    groups = {k: ticking}
                else:
                    groups = {}
                    for j in ticking:
                        groups.setdefault(self._tick_steps(j), []).append(j)
                for k, jobs in sorted(groups.items()):  # asynchronous: builds run meanwhile
                    self.ctx.step_domains([d for j in jobs for d in j.domains], k)
                t = time.perf_counter()
                self.ctx.sync()
                self.wait_s += time.perf_counter() - t
                self.ticks += 1
                for k, jobs in groups.items():
                    self.site_steps += sum(d.n for j in jobs for d in j.domains) * k
                    for j in jobs:
                        if j.cancelled:
                            continue
                        j.done_steps += k
                        if j.done_steps >= j.steps:
                            self._retire(j, read=True, now_s=clock() - t0)
            elif self.building:
                # nothing to step: wait for the oldest build, or for the next arrival if sooner
                gap = self.queue[0].arrival_s - (clock() - t0) if self.queue else 0.0
                self._activate(block=True, timeout=gap if gap > 0 else None)
            elif self.queue:
                gap = self.queue[0].arrival_s - (clock() - t0)
                if gap > 0:
                    sleep(min(gap, 0.05))
            if max_ticks is not None and self.ticks >= max_ticks:
                break
        self.elapsed_s = clock() - t0
        return self.finished

    def stats(self):
        ttr = np.array([j.time_to_result for j in self.finished])
        out = {"requests": len(self.finished), "ticks": self.ticks,
               "elapsed_s": getattr(self, "elapsed_s", float("nan")),
               "aggregate_mflups": self.site_steps / max(getattr(self, "elapsed_s", 1e-9), 1e-9) / 1e6,
               "peak_hbm_gb": self.peak_in_use / 1e9, "build_s": self.build_s,
               "policy": self.policy, "backfilled": self.backfilled, "failed": len(self.failed),
               "estimate_exceeded": self.estimate_exceeded,
               "gpu_wait_s": self.wait_s, "idle_s": self.idle_s}
        if ttr.size:
            out.update(p50_s=float(np.percentile(ttr, 50)), p99_s=float(np.percentile(ttr, 99)),
                       mean_s=float(ttr.mean()), max_s=float(ttr.max()))
        return out

    def close(self):
        if self._pool is not None:
            self._pool.shutdown(wait=True)   # no build may overlap the context's destruction
        self.ctx.close()


class _Done:
    """A completed build in the shape of a future (builds run inline without a worker)."""

    def __init__(self, value):
        self.value = value

    def done(self):
        return True

    def result(self):
        return self.value


def coupled_job_from_trees(rid, arrival_s, steps, art, ven, uniforms, tau=0.8):
    """Coupled arterial/venous request: arterial outlets (iolets 1..) drive venous inlets (1..).

    The map and factors come from hg_coupling_factors (Section 3): greedy nearest map on iolet
    centres in the shared frame, dP/P0 = 0.3 + 0.4 u, velocity factors by area and distance.
    """
    oa, ov = np.array(art.origin), np.array(ven.origin)
    ac = [tuple(int(c) for c in (np.array(io.centre) + 1024 * oa)) for io in art.iolets[1:]]
    vc = [tuple(int(c) for c in (np.array(io.centre) + 1024 * ov)) for io in ven.iolets[1:]]
    aa = [io.area() for io in art.iolets[1:]]
    va = [io.area() for io in ven.iolets[1:]]
    assign, dist, dp, fac = H.hg_coupling_factors(ac, aa, vc, va, uniforms[: len(vc)])
    pairs = [(int(assign[v]) + 1, v + 1, float(fac[v])) for v in range(len(vc))]
    return Job(rid=rid, arrival_s=arrival_s, steps=steps, geoms=[art, ven], pairs=pairs, tau=tau)
