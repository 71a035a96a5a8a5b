"""Serving loop: the seeded request stream (CPU) and, on the GPU, continuous admission
against a memory budget with overlapping solves whose results equal each request run alone
(bit for bit: a mesh's kernels touch only its own pools)."""
import math

import numpy as np
import pytest

from paper_2607_19277_gb300 import serving


def test_request_stream_is_seeded_poisson():
    reqs = serving.request_stream(4000, rate=50.0)
    assert reqs == serving.request_stream(4000, rate=50.0) or all(
        a.arrival == b.arrival for a, b in zip(reqs, serving.request_stream(4000, rate=50.0)))
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 50.0) < 0.05 / 50.0 * 4
    # exponential gaps: std equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08
    assert {r.physics for r in reqs} == {"hd", "mhd", "srhd"}
    assert {r.side for r in reqs} == {32, 64, 128, 256}
    assert min(r.steps for r in reqs) >= 50 and max(r.steps for r in reqs) <= 500


def test_pool_bytes_cover_the_pools():
    r = serving.Request(rid=0, physics="mhd", side=64, steps=10, seed=1, arrival=0.0)
    assert serving.pool_bytes(r, 4) >= 3 * 64 * 9 * 4096 * 4


@pytest.mark.gpu
def test_serving_admits_within_budget_overlaps_and_matches_alone():
    reqs = [serving.Request(rid=i, physics=("hd", "mhd", "srhd")[i % 3], side=(32, 48)[i % 2],
                            steps=3 + (i % 4), seed=500 + i, arrival=0.002 * i) for i in range(7)]
    sizes = sorted(serving.pool_bytes(r, 4) for r in reqs)
    budget = sizes[-1] + sizes[-2] + sizes[-3]       # room for about three at once
    srv = serving.Server(budget, real_bytes=4, steps_per_poll=1, keep_results=True)
    rep = srv.run(reqs, max_wall_s=120.0)
    s = rep.summary()
    assert rep.max_resident_bytes <= budget
    assert rep.max_concurrent >= 2
    assert s["latency_p99_s"] >= s["latency_p50_s"] > 0
    for r in reqs:
        assert r.finished > 0 and r.admitted >= r.arrival - 1e-9
        alone = serving.run_alone(r, real_bytes=4)
        assert np.array_equal(r.result, alone), r.rid


class FakeEvent:
    """A CUDA event stand-in that completes after `lag` queries (0: at once)."""
    lag = 0
    recorded = []

    def __init__(self):
        self.left = FakeEvent.lag

    def record(self, stream):
        FakeEvent.recorded.append(self)

    def query(self):
        if self.left > 0:
            self.left -= 1
            return False
        return True


class FakeTorch:
    class cuda:
        Event = FakeEvent

        @staticmethod
        def Stream():
            return None

        class stream:
            def __init__(self, s):
                pass

            def __enter__(self):
                return self

            def __exit__(self, *a):
                return False


def test_server_loop_terminates_without_gpu_work(monkeypatch):
    """The scheduling loop ends when every request is retired (host logic, fake meshes)."""
    class FakeMesh:
        def __init__(self, cfg, stream=None):
            self.steps = 0

        def set_state(self, ic):
            pass

        def set_state_prims(self, prim):
            pass

        def step(self, dt=0.0):
            self.steps += 1

        def sync(self):
            pass

        def get_state(self):
            return None, None, np.zeros(1)

        def close(self):
            pass

    monkeypatch.setattr(FakeEvent, "lag", 0)
    monkeypatch.setattr(serving.agile, "Mesh", FakeMesh)
    monkeypatch.setattr(serving, "prepare", lambda r, rb: np.zeros(1))
    reqs = serving.request_stream(20, rate=5000.0, sides=(32, 64), steps=(2, 5))
    srv = serving.Server.__new__(serving.Server)
    srv.torch = FakeTorch
    srv.budget = 3 * max(serving.pool_bytes(r, 4) for r in reqs)
    srv.rb = 4
    srv.steps_per_poll = 2
    srv.keep = False
    srv.workers = 2
    srv.max_prepared = 3
    rep = srv.run(reqs, max_wall_s=30.0)
    assert all(r.finished >= 0 for r in reqs)
    assert rep.max_resident_bytes <= srv.budget and rep.max_concurrent >= 1


@pytest.mark.gpu
def test_batched_serving_matches_alone():
    """Requests attach to per-physics batches as they are admitted and detach when done (the
    other solves stay in place); every result equals the request run alone, bit for bit."""
    reqs = [serving.Request(rid=i, physics=("hd", "mhd", "srhd")[i % 3], side=(32, 48)[i % 2],
                            steps=3 + (i % 5), seed=700 + i, arrival=0.001 * i) for i in range(9)]
    sizes = sorted(serving.pool_bytes(r, 4) for r in reqs)
    budget = sum(sizes[-4:])                         # room for about four at once
    srv = serving.BatchedServer(budget, real_bytes=4, keep_results=True)
    rep = srv.run(reqs, max_wall_s=120.0)
    assert rep.max_resident_bytes <= budget
    assert rep.max_concurrent >= 2
    st = rep.summary()["membership"]
    assert st["joins"] == 9 and st["leaves"] == 9
    for r in reqs:
        assert r.finished > 0 and r.admitted >= r.arrival - 1e-9
        assert np.array_equal(r.result, serving.run_alone(r, real_bytes=4)), r.rid


@pytest.mark.parametrize("lag", [0, 3])
def test_batched_server_reads_each_solve_at_its_step_count(monkeypatch, lag):
    """Host logic of the batched loop with a fake batch that counts steps per attached solve
    and reuses detached indices like the library, and fake step events that complete at once
    or only after a few polls: every request is read out after exactly its requested steps,
    no batch has more steps enqueued ahead than the server allows, the budget is respected,
    every join has its leave and every batch is closed."""
    class FakeBatch:
        live = []

        def __init__(self, cfgs, stream=None):
            self.n = [0] * len(cfgs)
            self.on = [True] * len(cfgs)
            FakeBatch.live.append(self)

        def attach(self, cfg):
            for i, on in enumerate(self.on):
                if not on:
                    self.on[i], self.n[i] = True, 0
                    return i
            self.on.append(True)
            self.n.append(0)
            return len(self.n) - 1

        def detach(self, i):
            assert self.on[i]
            self.on[i] = False

        def set_state_prims(self, i, prim):
            assert self.on[i]
            self.n[i] = 0

        def step(self):
            pending = sum(1 for e in FakeEvent.recorded if e.left > 0)
            FakeBatch.max_pending = max(FakeBatch.max_pending, pending)
            self.n = [v + 1 if on else v for v, on in zip(self.n, self.on)]

        def get_state(self, i):
            assert self.on[i]
            return None, None, np.array([self.n[i]])

        def close(self):
            FakeBatch.live.remove(self)

    FakeBatch.max_pending = 0
    monkeypatch.setattr(FakeEvent, "lag", lag)
    monkeypatch.setattr(FakeEvent, "recorded", [])
    monkeypatch.setattr(serving.agile, "Batch", FakeBatch)
    monkeypatch.setattr(serving, "initial_condition", lambda r: None)
    monkeypatch.setattr(serving, "prepare", lambda r, rb: np.zeros(1))
    reqs = serving.request_stream(30, rate=3000.0, sides=(32, 64), steps=(2, 9))
    budget = 4 * max(serving.pool_bytes(r, 4) for r in reqs)
    srv = serving.BatchedServer.__new__(serving.BatchedServer)
    srv.__dict__.update(torch=FakeTorch, budget=budget, rb=4, keep=True, workers=2, max_prepared=3, depth=3)
    rep = srv.run(reqs, max_wall_s=30.0)
    assert all(r.finished > 0 and int(r.result[0]) == r.steps for r in reqs)
    # three physics batches, each with at most `depth` uncompleted step events
    assert FakeBatch.max_pending <= 3 * srv.depth
    assert rep.max_resident_bytes <= budget
    st = rep.summary()["membership"]
    assert st["joins"] == 30 and st["leaves"] == 30
    assert not FakeBatch.live                          # every batch closed


def test_preparer_bounds_outstanding_work(monkeypatch):
    """Initial conditions are prepared for the earliest waiting requests only, at most `limit`
    held at once; a taken preparation frees its slot."""
    import threading
    gate = threading.Event()
    started = []

    def slow_prepare(r, rb):
        started.append(r.rid)
        gate.wait(5.0)
        return np.full(1, r.rid)
    monkeypatch.setattr(serving, "prepare", slow_prepare)
    reqs = [serving.Request(rid=i, physics="hd", side=32, steps=1, seed=i, arrival=0.0) for i in range(6)]
    p = serving._Preparer(workers=2, limit=3, real_bytes=4)
    try:
        p.feed(reqs)
        assert sorted(p.futs) == [0, 1, 2]
        assert not p.ready(reqs[0])
        gate.set()
        p.futs[0].result(5.0)
        assert p.ready(reqs[0]) and int(p.take(reqs[0])[0]) == 0
        p.feed(reqs[1:])
        assert sorted(p.futs) == [1, 2, 3]
        assert not p.ready(reqs[5])
    finally:
        gate.set()
        p.close()


def test_command_line_rejects_bad_ranges():
    with pytest.raises(SystemExit):
        serving.main(["--sides", "32,40"])
    with pytest.raises(SystemExit):
        serving.main(["--steps", "10"])
