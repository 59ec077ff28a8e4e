"""Host logic of the continuous-batching scheduler (no GPU): admission by HBM budget, LRU eviction,
per-geometry batching of requests that arrive while a batch is in flight, result routing."""
import numpy as np
import pytest

from paper_2203_15461_gb300.serve import Request, Scheduler, latency_stats, run_stream


class FakeBackend:
    def __init__(self, latency_pumps=2):
        self.created, self.released, self.launches = [], [], []
        self.latency = latency_pumps
        self.pending = {}
        self.t = 0.0

    def now(self):
        return self.t

    def create(self, key, geom):
        self.created.append(key)

    def release(self, key):
        self.released.append(key)

    def launch(self, key, batch):
        self.launches.append((key, [r.rid for r in batch]))
        # q of each replica: its total electrolyte charge repeated, so routing is checkable
        self.pending[key] = [self.latency, np.array([[r.Q.sum()] * 3 for r in batch]), np.array([r.rid for r in batch])]

    def ready(self, key):
        self.t += 1.0
        self.pending[key][0] -= 1
        return self.pending[key][0] <= 0

    def collect(self, key):
        _, q, rid = self.pending.pop(key)
        return q, rid.astype(float)


def _req(rid, key, nq=4):
    rng = np.random.default_rng(rid)
    return Request(rid=rid, key=key, xyz=rng.normal(size=(nq, 3)), Q=rng.normal(size=nq), psi=np.zeros(2))


def test_results_are_routed_to_their_requests():
    be = FakeBackend()
    sch = Scheduler(be, hbm_budget=100, max_batch=3)
    sch.add_geometry("a", None, 10)
    sch.add_geometry("b", None, 10)
    reqs = [_req(i, "a" if i % 3 else "b") for i in range(11)]
    for r in reqs:
        sch.submit(r)
    while not sch.idle():
        sch.pump()
    assert sorted(r.rid for r in sch.finished) == list(range(11))
    for r in sch.finished:
        assert np.allclose(r.q, r.Q.sum()) and r.qtot == r.rid
    assert all(len(ids) <= 3 for _, ids in be.launches)


def test_requests_arriving_during_a_batch_join_the_next_one():
    be = FakeBackend(latency_pumps=10)
    sch = Scheduler(be, hbm_budget=100, max_batch=8)
    sch.add_geometry("a", None, 10)
    sch.submit(_req(0, "a"))
    sch.pump()                                   # batch [0] in flight
    for i in range(1, 6):
        sch.submit(_req(i, "a"))
        sch.pump()
    while not sch.idle():
        sch.pump()
    assert be.launches[0] == ("a", [0])
    assert be.launches[1][1] == [1, 2, 3, 4, 5]  # everything that queued up went in one batch


def test_budget_admission_and_lru_eviction():
    be = FakeBackend()
    sch = Scheduler(be, hbm_budget=25, max_batch=4)
    for k in "abc":
        sch.add_geometry(k, None, 10)
    for i, k in enumerate("aabbccab"):
        sch.submit(_req(i, k))
        sch.pump()
        assert sum(sch.resident.values()) <= 25
    while not sch.idle():
        sch.pump()
        assert sum(sch.resident.values()) <= 25
    assert len(sch.finished) == 8
    assert sch.evictions >= 1 and be.released


def test_geometry_larger_than_the_budget_is_rejected():
    sch = Scheduler(FakeBackend(), hbm_budget=5)
    sch.add_geometry("big", None, 10)
    sch.submit(_req(0, "big"))
    with pytest.raises(ValueError):
        sch.pump()


def test_run_stream_and_latency_stats():
    be = FakeBackend()
    sch = Scheduler(be, hbm_budget=100, max_batch=4)
    sch.add_geometry("a", None, 10)
    reqs = [_req(i, "a") for i in range(9)]
    run_stream(reqs, sch, arrivals=np.zeros(9))
    st = latency_stats(sch.finished)
    assert st["n"] == 9 and st["p99_ms"] >= st["p50_ms"]
