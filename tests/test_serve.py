"""Serving loop: admission, continuous batching and results (CPU logic with a fake executor; GPU
results identical alone and in the mix)."""
import itertools
import time

import numpy as np
import pytest

from paper_2006_06775_gb300 import serve, synth


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor(serve.Executor):
    """Each enqueue of k steps keeps the simulation busy for k * cost seconds of fake time; every
    ready() poll advances the clock a little, so the loop makes progress without sleeping."""

    def __init__(self, clock, cost=1e-4):
        self.clock, self.cost = clock, cost
        self.live, self.peak_bytes, self.peak_active = {}, 0, 0
        self.started = []
        self.ids = itertools.count()

    def start(self, req, pl):
        h = next(self.ids)
        self.live[h] = (serve.estimate_bytes(req.kind, req.n), self.clock())
        self.started.append(req.rid)
        self.peak_bytes = max(self.peak_bytes, sum(b for b, _ in self.live.values()))
        self.peak_active = max(self.peak_active, len(self.live))
        return {"h": h, "busy": self.clock()}

    def enqueue(self, h, steps):
        h["busy"] = max(h["busy"], self.clock()) + steps * self.cost

    def ready(self, h):
        self.clock.t += 1e-5
        return self.clock() >= h["busy"]

    def result(self, h):
        return {}

    def close(self, h):
        del self.live[h["h"]]


class FakePoolExecutor(FakeExecutor):
    """Adds a pool of `slots` places for mechanics requests up to `cap` agents: each tick on an idle
    pool retires the simulations that reached their step count and advances all the others by one
    chunk, which keeps the pool busy for chunk * step_cost seconds whatever their number."""

    def __init__(self, clock, slots=4, cap=5000, chunk=25, step_cost=5e-5):
        super().__init__(clock)
        self.slots, self.cap, self.chunk, self.step_cost = slots, cap, chunk, step_cost
        self.in_pool, self.busy_until, self.peak_pool, self.chunks = [], 0.0, 0, 0

    def pooled(self, req):
        return req.kind == "mechanics" and req.n <= self.cap

    def pool_free(self):
        return len(self.in_pool) < self.slots

    def start(self, req, pl):
        if not self.pooled(req):
            return super().start(req, pl)
        assert self.pool_free()
        self.started.append(req.rid)
        h = {"pooled": True, "left": req.steps, "done": False}
        self.in_pool.append(h)
        self.peak_pool = max(self.peak_pool, len(self.in_pool))
        return h

    def tick(self):
        if self.clock() < self.busy_until:
            return
        for h in list(self.in_pool):
            if h["left"] <= 0:
                h["done"] = True
                self.in_pool.remove(h)
        if self.in_pool:
            for h in self.in_pool:
                h["left"] -= self.chunk
            self.busy_until = self.clock() + self.chunk * self.step_cost
            self.chunks += 1

    def ready(self, h):
        if not h.get("pooled"):
            return super().ready(h)
        self.clock.t += 1e-5
        return h["done"]

    def result(self, h):
        return {}

    def close(self, h):
        if not h.get("pooled"):
            super().close(h)


def trace(count=200, rate=200.0):
    return synth.request_stream(count=count, rate=rate, seed=4)


def test_fifo_admission_budget_and_slots(monkeypatch):
    clock = FakeClock()
    monkeypatch.setattr(serve.time, "sleep", lambda s: setattr(clock, "t", clock.t + s))
    reqs = trace()
    ex = FakeExecutor(clock)
    budget = 3e9
    srv = serve.Server(ex, budget_bytes=budget, max_active=16, chunk=25, clock=clock)
    done = srv.run(reqs, lambda r: None)
    assert len(done) == len(reqs)
    assert ex.started == sorted(ex.started)          # admitted strictly in arrival order
    assert ex.peak_bytes <= budget
    assert ex.peak_active <= 16
    for j in done:
        assert j.done >= j.admitted >= j.req.arrival
        assert j.steps_left == 0


def test_requests_join_while_others_run(monkeypatch):
    """Continuous batching: later arrivals are admitted while earlier simulations are still
    running (not after the queue drains)."""
    clock = FakeClock()
    monkeypatch.setattr(serve.time, "sleep", lambda s: setattr(clock, "t", clock.t + s))
    reqs = trace(count=60)
    ex = FakeExecutor(clock, cost=2e-3)
    done = serve.Server(ex, budget_bytes=150e9, max_active=64, clock=clock).run(reqs, lambda r: None)
    by_id = {j.req.rid: j for j in done}
    overlaps = sum(1 for a, b in itertools.combinations(sorted(by_id), 2)
                   if by_id[b].admitted < by_id[a].done)
    assert overlaps > len(reqs)


def test_request_larger_than_budget_is_refused(monkeypatch):
    clock = FakeClock()
    monkeypatch.setattr(serve.time, "sleep", lambda s: setattr(clock, "t", clock.t + s))
    r = synth.Request(0, 0.0, "mechanics", 10 ** 6, 10, 1)
    with pytest.raises(RuntimeError):
        serve.Server(FakeExecutor(clock), budget_bytes=1e6, clock=clock).run([r], lambda r: None)


def test_pool_takes_small_mechanics_in_order(monkeypatch):
    """Small mechanics requests go to the pool, the rest get handles of their own: admission stays
    in arrival order across both, the pool never holds more than its slots, pooled simulations hold
    no budget, and one pool chunk advances many simulations at once."""
    clock = FakeClock()
    monkeypatch.setattr(serve.time, "sleep", lambda s: setattr(clock, "t", clock.t + s))
    reqs = trace(count=300)
    ex = FakePoolExecutor(clock, slots=6, cap=5000, step_cost=4e-4)
    budget = 3e9
    done = serve.Server(ex, budget_bytes=budget, max_active=8, chunk=25, clock=clock).run(
        reqs, lambda r: None)
    assert len(done) == len(reqs)
    assert ex.started == sorted(ex.started)
    pooled = [j for j in done if j.pooled]
    assert {j.req.rid for j in pooled} == {r.rid for r in reqs if ex.pooled(r)}
    assert len(pooled) > 30
    assert all(j.bytes == 0 for j in pooled)
    assert ex.peak_pool <= 6 and ex.peak_active <= 8 and ex.peak_bytes <= budget
    per_sim_chunks = sum(-(-j.req.steps // 25) for j in pooled)
    assert ex.chunks < per_sim_chunks / 2
    for j in done:
        assert j.done >= j.admitted >= j.req.arrival


def test_summary_statistics():
    jobs = []
    for k in range(100):
        j = serve.Job(synth.Request(k, 0.0, "sir", 1000, 10, k), 0, 0)
        j.done = (k + 1) * 0.01
        jobs.append(j)
    s = serve.summarize(jobs)
    assert s["requests"] == 100 and abs(s["makespan_s"] - 1.0) < 1e-12
    assert abs(s["p50_s"] - np.percentile([(k + 1) * 0.01 for k in range(100)], 50)) < 1e-12
    assert abs(s["agent_steps_per_s"] - 100 * 1000 * 10 / 1.0) < 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("skin,pool", [(0.0, 0), (2.5, 0), (0.0, 3)])
def test_served_results_equal_results_alone(skin, pool):
    """A small mixed trace served concurrently gives, for every request, exactly the result of
    the same simulation run alone (with the grid rebuilt every step, with neighbour lists, and with
    the small mechanics requests in a three-slot pool next to own handles)."""
    g = synth.rng(4, 77)
    reqs = [synth.Request(k, 0.002 * k, "mechanics" if k % 3 else "sir",
                          int(g.integers(1000, 20000)), int(g.integers(20, 60)), 900 + k)
            for k in range(12)]
    payloads = {r.rid: serve.payload(r) for r in reqs}
    ex = serve.GpuExecutor(streams=4, mechanics_skin=skin, pool_slots=pool, pool_capacity=12000,
                           pool_chunk=9)
    mixed = serve.Server(ex, budget_bytes=150e9, max_active=8, chunk=7).run(
        reqs, lambda r: payloads[r.rid])
    alone = serve.run_one_at_a_time(serve.GpuExecutor(streams=1, mechanics_skin=skin), reqs,
                                    lambda r: payloads[r.rid])
    ex.shutdown()
    A = {j.req.rid: j.result for j in alone}
    assert len(mixed) == len(reqs)
    assert sum(j.pooled for j in mixed) == (sum(1 for r in reqs if r.kind == "mechanics" and
                                                r.n <= 12000) if pool else 0)
    for j in mixed:
        for f, v in j.result.items():
            if isinstance(v, np.ndarray):
                assert np.array_equal(v, A[j.req.rid][f]), (j.req.rid, f)
