"""Scheduling logic of the continuous-batching server, on a stub context (CPU only).

FIFO admission by HBM footprint, no starvation, budget never exceeded,
cancellation, exact step counts per request.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import serve as SV
from paper_2010_04144_gb300 import synth as S


class _Dom:
    def __init__(self, ctx, n, nio):
        self.ctx, self.n, self.nio, self.step = ctx, n, nio, 0
        self.alive = True

    def info(self):
        return {"device_bytes": SV.footprint_bytes(self.n, self.ctx.storage, self.ctx.scheme, self.nio)}

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

    def domain(self, xyz, iolets, tau=0.8):
        d = _Dom(self, len(xyz), len(iolets))
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


@pytest.fixture
def server(monkeypatch):
    monkeypatch.setattr(SV.H, "Context", lambda **kw: _Ctx(**kw))

    def make(budget):
        return SV.Server(storage="f16", scheme="aa", budget_bytes=budget, chunk_steps=50)

    return make


def _job(rid, t, n=1000, steps=200):
    g = S.Geometry(xyz=np.zeros((n, 3), np.int32), iolets=[None, None])
    return SV.Job(rid=rid, arrival_s=t, steps=steps, geoms=[g])


def test_fifo_budget_and_exact_steps(server):
    one = SV.footprint_bytes(1000, 1, 1, 2)
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
    small = SV.footprint_bytes(1000, 1, 1, 2)
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
    one = SV.footprint_bytes(1000, 1, 1, 2)
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
