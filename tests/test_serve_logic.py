"""Scheduling logic of the continuous-batching server, on a stub context (CPU only).

FIFO admission by HBM footprint, no starvation, budget never exceeded,
cancellation, exact step counts per request, a failed build that fails its own
request only, a built domain larger than its estimate holding admissions back,
the footprint estimate as an upper bound on the boundary slots of an
iolet-heavy geometry, and ticks that give every request an equal share of site
updates instead of an equal step count.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import serve as SV
from paper_2010_04144_gb300 import synth as S


class _Dom:
    def __init__(self, ctx, n, iolets):
        self.ctx, self.n, self.nio, self.step = ctx, n, len(iolets), 0
        self.radii = [io.radius / 1024.0 for io in iolets]
        self.alive = True

    def info(self):
        b = SV.footprint_bytes(self.n, self.ctx.storage, self.ctx.scheme, iolet_radii=self.radii)
        return {"device_bytes": 2 * b if self.n == 1111 else b}   # 1111 sites: under-estimated

    def iolet_stats(self):
        return np.zeros((self.nio, 3))

    def mass(self):
        return 0.0

    def destroy(self):
        self.alive = False


class _Ctx:
    def __init__(self, **kw):
        self.storage, self.scheme = kw["storage"], kw["scheme"]
        self.calls = []
        self.live = []

    def domain(self, xyz, iolets, tau=0.8, ordering="morton"):
        d = _Dom(self, len(xyz), iolets)
        self.live.append(d)
        return d

    def couple(self, a, b, pairs):
        self.calls.append(("couple", len(pairs)))

    def step_domains(self, doms, k):
        assert all(d.alive for d in doms)
        for d in doms:
            d.step += k
        self.calls.append(("step", len(doms), k))

    def sync(self):
        pass

    def close(self):
        pass


class _Clock:
    def __init__(self, dt=0.01):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t

    def sleep(self, s):
        self.t += s


@pytest.fixture(params=[0, 1], ids=["inline-build", "worker-build"])
def server(monkeypatch, request):
    monkeypatch.setattr(SV.H, "Context", lambda **kw: _Ctx(**kw))
    made = []

    def make(budget):
        srv = SV.Server(storage="f16", scheme="aa", budget_bytes=budget, chunk_steps=50,
                        build_workers=request.param)
        made.append(srv)
        return srv

    yield make
    for srv in made:
        srv.close()


_IO = S.Iolet(kind=S.PRESSURE, centre=(0, 0, 0), axis=(0, 0, 1024), radius=2048)


def _job(rid, t, n=1000, steps=200):
    g = S.Geometry(xyz=np.zeros((n, 3), np.int32), iolets=[_IO, _IO])
    return SV.Job(rid=rid, arrival_s=t, steps=steps, geoms=[g])


def _fp(n):
    return SV.geometry_footprint(_job(0, 0.0, n=n).geoms[0], 1, 1)


def test_fifo_budget_and_exact_steps(server):
    one = _fp(1000)
    srv = server(budget=2.5 * one)           # at most two requests resident
    jobs = [_job(i, 0.02 * i) for i in range(7)]
    for j in jobs:
        srv.submit(j)
    clk = _Clock()
    done = srv.run(clock=clk, sleep=clk.sleep)
    assert [j.rid for j in done] == list(range(7))          # nobody starves or overtakes
    assert srv.admit_order == list(range(7))
    assert srv.peak_in_use <= 2.5 * one
    assert all(j.done_steps == j.steps for j in done)
    for d in srv.ctx.live:
        assert d.step == 200 and not d.alive
    assert all(j.time_to_result > 0 for j in done)
    st = srv.stats()
    assert st["requests"] == 7 and st["p99_s"] >= st["p50_s"] > 0


def test_large_head_blocks_smaller_followers(server):
    small = _fp(1000)
    srv = server(budget=small * 3.2)
    jobs = [_job(0, 0.0), _job(1, 0.0, n=2500), _job(2, 0.001)]
    for j in jobs:
        srv.submit(j)
    clk = _Clock()
    srv.run(clock=clk, sleep=clk.sleep)
    assert srv.admit_order == [0, 1, 2]


def test_oversized_request_rejected(server):
    srv = server(budget=1e6)
    with pytest.raises(ValueError):
        srv.submit(_job(0, 0.0, n=10 ** 6))
    with pytest.raises(ValueError):
        srv.submit(_job(1, 0.0, steps=75))   # not a multiple of the tick


def test_cancel_queued_and_active(server):
    one = _fp(1000)
    srv = server(budget=1.5 * one)
    for i in range(3):
        srv.submit(_job(i, 0.0))
    assert srv.cancel(2)
    srv.run(clock=_Clock(), sleep=lambda s: None, max_ticks=1)
    assert [j.rid for j in srv.active] == [0]
    assert srv.cancel(0)
    assert srv.in_use == 0
    clk = _Clock()
    srv.run(clock=clk, sleep=clk.sleep)
    assert [j.rid for j in srv.finished] == [1]
    assert not srv.cancel(7)


class _SlowCtx(_Ctx):
    """Stub whose domain builds take real time (a large request's host build)."""

    delay = 0.3

    def domain(self, xyz, iolets, tau=0.8, ordering="morton"):
        if len(xyz) >= 2000:
            import time

            time.sleep(self.delay)
        if len(xyz) == 1234:
            raise SV.H.HgError(-1, "build failed")
        return super().domain(xyz, iolets, tau, ordering)

    def sync(self):
        import time

        time.sleep(0.02)   # a tick's GPU time


@pytest.fixture
def slow_server(monkeypatch):
    monkeypatch.setattr(SV.H, "Context", lambda **kw: _SlowCtx(**kw))
    made = []

    def make(budget, workers=1):
        srv = SV.Server(storage="f16", scheme="aa", budget_bytes=budget, chunk_steps=50,
                        build_workers=workers)
        made.append(srv)
        return srv

    yield make
    for srv in made:
        srv.close()


def test_worker_build_overlaps_ticks(slow_server):
    srv = slow_server(budget=1e12)
    srv.submit(_job(0, 0.0, steps=2000))             # 40 ticks of ~20 ms
    srv.submit(_job(1, 0.0, n=2000, steps=100))       # slow build, admitted at once
    clk = _Clock()
    srv.run(clock=clk, sleep=clk.sleep)
    steps = [c for c in srv.ctx.calls if c[0] == "step"]
    # request 0 keeps ticking alone while request 1 builds; then both share launches
    assert steps[0] == ("step", 1, 50)
    assert any(c[1] == 2 for c in steps)
    assert [j.done_steps for j in sorted(srv.finished, key=lambda j: j.rid)] == [2000, 100]
    assert srv.in_use == 0 and srv.stats()["build_s"] >= _SlowCtx.delay


def test_inline_build_blocks_first_tick(slow_server):
    srv = slow_server(budget=1e12, workers=0)
    srv.submit(_job(0, 0.0, steps=400))
    srv.submit(_job(1, 0.0, n=2000, steps=100))
    clk = _Clock()
    srv.run(clock=clk, sleep=clk.sleep)
    steps = [c for c in srv.ctx.calls if c[0] == "step"]
    assert steps[0] == ("step", 2, 50)                # both built before the first tick


def test_cancel_while_building_releases_memory(slow_server):
    srv = slow_server(budget=1e12)
    srv.submit(_job(0, 0.0, n=2000))
    srv._admit(0.0)
    assert srv.building and srv.in_use > 0
    assert srv.cancel(0)
    clk = _Clock()
    srv.run(clock=clk, sleep=clk.sleep)
    assert srv.finished == [] and srv.in_use == 0
    assert all(not d.alive for d in srv.ctx.live)


def test_build_error_fails_only_its_request(slow_server):
    for workers in (0, 1):
        srv = slow_server(budget=1e12, workers=workers)
        srv.submit(_job(0, 0.0, n=1234))              # its build raises
        srv.submit(_job(1, 0.0, steps=100))
        srv.submit(_job(2, 0.01, steps=100))
        clk = _Clock()
        srv.run(clock=clk, sleep=clk.sleep)
        assert [j.rid for j in srv.failed] == [0] and "build failed" in srv.failed[0].result["error"]
        assert sorted(j.rid for j in srv.finished) == [1, 2]
        assert srv.in_use == 0 and not srv.active and srv.stats()["failed"] == 1


def test_underestimated_domain_holds_admissions(server):
    one = _fp(1000)
    srv = server(budget=2.5 * one)
    srv.submit(_job(0, 0.0, n=1111))                  # built at twice its estimate
    srv.submit(_job(1, 0.05))                         # arrives once request 0 is resident
    clk = _Clock()
    srv.run(clock=clk, sleep=clk.sleep)
    j0, j1 = sorted(srv.finished, key=lambda j: j.rid)
    assert srv.estimate_exceeded == 1 and srv.max_overshoot_bytes > 0
    assert j1.admitted_s >= j0.finished_s             # request 1 waited for the memory
    assert srv.in_use == 0


def test_footprint_bounds_iolet_heavy_geometry(hemegb_lib):
    """Many short tubes: nearly every site is next to an iolet, far above the 5% a plain
    tree has.  The per-iolet bound still covers every iolet's adjacent sites."""
    geo = S.parallel_tubes(12, radius=3, length=3)
    _, nbr = hemegb_lib.build_neighbours(geo.xyz, geo.iolets)
    adj_any = (nbr < -1).any(axis=0).sum()
    assert adj_any > 0.5 * geo.n
    for k, io in enumerate(geo.iolets):
        count = (nbr == -(2 + k)).any(axis=0).sum()
        assert count <= SV.adjacent_bound(io.radius / 1024.0)
    slots = 164 * adj_any
    assert SV.geometry_footprint(geo, 1, 1) >= SV.footprint_bytes(geo.n, 1, 1, iolet_radii=[]) + slots


def _run_policy(monkeypatch, policy, jobs, budget):
    monkeypatch.setattr(SV.H, "Context", lambda **kw: _Ctx(**kw))
    srv = SV.Server(storage="f16", scheme="aa", budget_bytes=budget, chunk_steps=50,
                    build_workers=0, policy=policy)
    for j in jobs:
        srv.submit(j)
    clk = _Clock()
    srv.run(clock=clk, sleep=clk.sleep)
    srv.close()
    return srv


def test_backfill_lets_short_requests_pass_without_delaying_the_head(monkeypatch):
    one = _fp(1000)
    big = _fp(2500)
    budget = 2 * one + 0.5 * (big - one)       # two small fit; the big head cannot start while 0 runs
    assert one + big > budget

    def jobs():
        return [_job(0, 0.0, steps=1000), _job(1, 0.001, n=2500, steps=200),
                _job(2, 0.002, steps=100), _job(3, 0.003, steps=5000)]

    fifo = _run_policy(monkeypatch, "fifo", jobs(), budget)
    bf = _run_policy(monkeypatch, "backfill", jobs(), budget)
    assert fifo.admit_order == [0, 1, 2, 3] and fifo.backfilled == 0
    # request 2 (short) passes the blocked head; request 3 (long) may not
    assert bf.admit_order.index(2) < bf.admit_order.index(1) < bf.admit_order.index(3)
    assert bf.backfilled >= 1
    done_f = {j.rid: j for j in fifo.finished}
    done_b = {j.rid: j for j in bf.finished}
    assert all(j.done_steps == j.steps for j in bf.finished) and len(done_b) == 4
    assert done_b[2].finished_s < done_f[2].finished_s
    # the head starts no later (in ticks) than under FIFO
    assert 0 <= done_b[1].start_tick <= done_f[1].start_tick
    assert bf.peak_in_use <= budget


def test_unknown_policy_rejected(monkeypatch):
    monkeypatch.setattr(SV.H, "Context", lambda **kw: _Ctx(**kw))
    with pytest.raises(ValueError):
        SV.Server(policy="lifo")


def test_equal_share_ticks(monkeypatch):
    """With tick_site_steps every request advances about that many site updates per tick:
    a small request takes a multiple of the tick's step count in one call, a large one
    the plain tick; each request still ends at exactly its step count, and the small
    one finishes in fewer ticks than under equal step counts."""
    monkeypatch.setattr(SV.H, "Context", lambda **kw: _Ctx(**kw))
    out = {}
    for share in (None, 4e5):
        srv = SV.Server(storage="f16", scheme="aa", budget_bytes=1e12, chunk_steps=50,
                        build_workers=0, tick_site_steps=share)
        small, large = _job(0, 0.0, n=1000, steps=1000), _job(1, 0.0, n=20000, steps=1000)
        srv.submit(small)
        srv.submit(large)
        clk = _Clock()
        srv.run(clock=clk, sleep=clk.sleep)
        srv.close()
        assert all(j.done_steps == j.steps for j in srv.finished) and len(srv.finished) == 2
        assert all(d.step == 1000 for d in srv.ctx.live)
        steps = [c for c in srv.ctx.calls if c[0] == "step"]
        out[share] = (small.finished_s, large.finished_s, steps, srv.ticks)
    plain, shared = out[None], out[4e5]
    assert all(k == 50 for _, _, k in plain[2])                     # one step count per tick
    assert {k for _, _, k in shared[2]} >= {50, 400}                # 4e5 / 1000 sites -> 400 steps
    assert shared[0] < plain[0]                                     # the small request is done sooner
    assert shared[3] == plain[3] == 20                              # the large one sets the tick count
    with pytest.raises(ValueError):                                 # steps stay multiples of the tick
        SV.Server(storage="f16", scheme="aa", tick_site_steps=4e5).submit(_job(2, 0.0, steps=130))
