"""Host logic of the continuous-batching server, with a fake engine (no GPU):
admission against the HBM budget, LRU eviction of idle hierarchies, reuse,
grouping of queued requests, and failure isolation."""
import threading
import time
import types

import pytest

from paper_2206_11294_gb300.serve import HierarchyCache, Server, poisson_arrivals, run_stream


class FakeEngine:
    def __init__(self, fail_name=None, delay=0.002):
        self.fail_name = fail_name
        self.delay = delay
        self.live = 0
        self.max_live = 0
        self.lock = threading.Lock()
        self.groups = []
        self.streams = []

    def new_stream(self, high=False):
        return ("high" if high else "normal", object())

    def key(self, p):
        return (p.grid.n,)

    def size(self, p):
        return p.bytes

    def make(self, p, stream):
        with self.lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)
        return types.SimpleNamespace(n=p.grid.n)

    def free(self, obj):
        with self.lock:
            self.live -= 1

    def run(self, solvers, problems, stream):
        self.groups.append(len(problems))
        self.streams.append((stream[0], max(p.grid.N for p in problems)))
        time.sleep(self.delay)
        if any(p.name == self.fail_name for p in problems):
            raise RuntimeError("bad coefficients")
        return [(p.name, {"cycles": 1}) for p in problems]


def prob(name, n, nbytes, dim=2):
    return types.SimpleNamespace(name=name, grid=types.SimpleNamespace(n=n, dim=dim, N=n), bytes=nbytes)


def test_cache_budget_eviction_and_reuse():
    freed = []
    c = HierarchyCache(100, make=lambda k: object(), free=freed.append)
    a = c.acquire(("a",), 60)
    assert c.acquire(("b",), 60) is None          # does not fit while a is busy
    c.release(a)
    b = c.acquire(("b",), 60)                      # evicts idle a
    assert b is not None and len(freed) == 1 and c.used == 60
    c.release(b)
    assert c.acquire(("b",), 60) is b              # reused, not re-created
    assert c.created == 2 and c.reused == 1
    with pytest.raises(MemoryError):
        c.acquire(("c",), 500)


def test_server_respects_budget_and_completes_everything():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget=250, slots=3, max_batch=4)
    probs = [prob(f"p{q}", 10 + q % 5, 50 + 10 * (q % 5)) for q in range(40)]
    futs = [srv.submit(p) for p in probs]
    names = [f.result(timeout=30)[0] for f in futs]
    srv.close()
    assert names == [p.name for p in probs]
    assert srv.cache.peak <= 250
    st = srv.stats()
    assert st["requests"] == 40 and st["p99_ms"] >= st["p50_ms"] > 0
    assert max(eng.groups) > 1                     # queued requests were grouped


def test_failure_is_isolated():
    eng = FakeEngine(fail_name="bad")
    srv = Server(eng, hbm_budget=1000, slots=2, max_batch=1)
    good = [srv.submit(prob(f"g{q}", 8, 10)) for q in range(5)]
    bad = srv.submit(prob("bad", 8, 10))
    more = [srv.submit(prob(f"h{q}", 8, 10)) for q in range(5)]
    with pytest.raises(RuntimeError):
        bad.result(timeout=10)
    assert all(f.result(timeout=10)[0].startswith(("g", "h")) for f in good + more)
    srv.close()
    assert eng.live == 0                           # every hierarchy released


def test_oversized_request_fails_alone():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget=100, slots=1)
    big = srv.submit(prob("big", 99, 1000))
    ok = srv.submit(prob("ok", 4, 10))
    with pytest.raises(MemoryError):
        big.result(timeout=10)
    assert ok.result(timeout=10)[0] == "ok"
    srv.close()


def test_poisson_stream_rate():
    offs = poisson_arrivals(100.0, 2000, seed=3)
    assert abs(offs[-1] / 2000 - 0.01) < 0.001     # mean gap 1/rate
    eng = FakeEngine(delay=0.0)
    srv = Server(eng, hbm_budget=10_000, slots=2, max_batch=8)
    st = run_stream(srv, [prob("a", 4, 10), prob("b", 6, 20)], rate=2000.0, count=200)
    srv.close()
    assert st["requests"] == 200 and st["throughput_rps"] > 0


def test_prewarm_builds_resident_hierarchies_within_budget():
    """prewarm builds per_shape hierarchies per distinct grid without evicting
    any, stops at the budget, runs one solve on each, and later requests reuse
    them instead of creating new ones."""
    eng = FakeEngine()
    srv = Server(eng, hbm_budget=250, slots=2, max_batch=1)
    pool = [prob("a", 8, 50), prob("a2", 8, 50), prob("b", 16, 60), prob("c", 32, 100)]
    built = srv.prewarm(pool, per_shape=2)
    # a: 2 x 50, b: 2 x 60 -> 220 used; c (100) does not fit without evicting
    assert built == 4 and srv.cache.used == 220 and srv.cache.evictions == 0
    assert eng.groups == [1, 1, 1, 1]
    created = srv.cache.created
    futs = [srv.submit(p) for p in pool[:3] * 3]
    for f in futs:
        f.result(timeout=10)
    assert srv.cache.created == created          # every request found a resident hierarchy
    srv.close()


def test_small_groups_run_on_the_high_priority_stream():
    eng = FakeEngine(delay=0.0)
    srv = Server(eng, hbm_budget=10_000, slots=2, max_batch=1, small_cells=100)
    futs = [srv.submit(prob(f"p{i}", n, 10)) for i, n in enumerate([50, 100, 101, 4000])]
    for f in futs:
        f.result(timeout=10)
    srv.close()
    assert sorted(eng.streams, key=lambda t: t[1]) == [("high", 50), ("high", 100), ("normal", 101),
                                                        ("normal", 4000)]
