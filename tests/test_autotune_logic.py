"""Launch-shape autotuner logic on a stub context (CPU only).

Which candidates each storage/scheme may try, that the fastest is chosen and
applied, that the domains' state is restored afterwards, and that the cache
key separates different candidate sets.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import autotune as AT


class _Dom:
    def __init__(self, n):
        self.n = n
        self.state = np.arange(4, dtype=np.uint8)
        self.loads = 0

    def save_state(self):
        return self.state.copy()

    def load_state(self, buf):
        self.loads += 1
        self.state = buf.copy()


class _Ctx:
    def __init__(self, storage, scheme, cost):
        self.device, self.storage, self.scheme = 0, storage, scheme
        self.domains = [_Dom(1000)]
        self.tried, self.launch, self.cost = [], None, cost

    def set_launch(self, b, spt, var):
        self.launch = (b, spt, var)
        self.tried.append(self.launch)

    def step(self, n):
        self.domains[0].state = self.domains[0].state + 1   # stepping changes the state

    def step_profiled(self, n):
        self.step(n)
        return self.cost(self.launch) * n, 0.0


@pytest.mark.parametrize("storage,scheme,allowed", [
    (0, 0, {0, 1, 3, 8, 13}), (1, 0, {0, 1, 3, 5, 8, 9, 13}), (2, 0, {0, 1, 3, 5, 8, 9, 13}),
    (0, 1, {0, 1, 2, 3, 6, 7, 8, 10, 11, 12, 13, 14}), (1, 1, {0, 1, 2, 3, 6, 7, 8, 10, 11, 12, 13, 14}),
])
def test_candidates_per_form(storage, scheme, allowed):
    ctx = _Ctx(storage, scheme, cost=lambda L: 1.0 + L[0] / 1e4 + L[1] / 1e3 + L[2] / 1e2)
    best, timing = AT.autotune(ctx, use_cache=False)
    variants = {t[2] for t in timing}
    assert variants == allowed
    assert best == min(timing, key=timing.get) and ctx.launch == best
    assert best == (128, 1, 0)                       # the cheapest under this cost model
    assert np.array_equal(ctx.domains[0].state, np.arange(4, dtype=np.uint8))  # state restored


def test_picks_the_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("HEMEGB_TUNE_CACHE", str(tmp_path / "tune.json"))
    ctx = _Ctx(1, 0, cost=lambda L: 0.5 if L == (256, 2, 5) else 1.0)
    best, _ = AT.autotune(ctx)
    assert best == (256, 2, 5)
    again = _Ctx(1, 0, cost=lambda L: 1.0)           # a cache hit does not re-time
    best2, timing2 = AT.autotune(again)
    assert best2 == (256, 2, 5) and again.tried == [(256, 2, 5)]
    assert timing2[(256, 2, 5)] == 0.5
    other = _Ctx(1, 0, cost=lambda L: 0.5 if L == (128, 1, 0) else 1.0)
    best3, _ = AT.autotune(other, candidates=[(128, 1, 0), (256, 1, 0)])   # other set: new key
    assert best3 == (128, 1, 0)


def test_needs_a_domain():
    ctx = _Ctx(0, 0, cost=lambda L: 1.0)
    ctx.domains = []
    with pytest.raises(ValueError):
        AT.autotune(ctx, use_cache=False)
