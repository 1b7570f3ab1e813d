"""Serving: a request loop over the simulation library with continuous batching.

Requests (mechanics or SIR simulations of different sizes and step counts) arrive over time.  The
server admits them in arrival order while the estimated device memory of the admitted set stays
inside a budget and a slot is free; admitted simulations keep their state resident on the device,
each on one of several CUDA streams, and every pass of the loop enqueues the next chunk of steps
(one CUDA-graph replay) for every active simulation, so work of different requests overlaps on the
GPU.  A simulation whose last chunk has completed (checked with events, without blocking) has its
state read back to the host; its memory returns to the pool and the next waiting request is
admitted.  Latency = time from arrival to the result on the host.

The scheduling logic only talks to "executors" (create / add agents / enqueue steps / poll /
result / close), so it is tested on the CPU with a fake executor; `GpuExecutor` drives libbdm.
"""
import heapq
import time
from dataclasses import dataclass, field

import numpy as np

from . import synth

# agent arrays + ~3 boxes per agent (count/start, capacity) + the neighbour-list mode's lists (32
# entries), second position set, list length and move
MECH_BYTES_PER_AGENT = 124 + 8 * 3 + 128 + 40 + 8
SIR_BYTES_PER_AGENT = 13 + 5 * 4 + 8 + 8   # state, 5 words per agent, list entry, ~1 box each
MIN_BYTES = 4 << 20


def estimate_bytes(kind: str, n: int) -> int:
    """Device memory a request will hold (upper estimate used for admission)."""
    per = MECH_BYTES_PER_AGENT if kind == "mechanics" else SIR_BYTES_PER_AGENT
    return max(MIN_BYTES, int(n * per * 1.25))


@dataclass
class Job:
    req: "synth.Request"
    bytes: int
    steps_left: int
    handle: object = None
    admitted: float = 0.0
    done: float = 0.0
    result: dict = field(default_factory=dict)


class Server:
    """Continuous-batching loop.  `executor` provides:
        start(req, payload) -> handle          (allocates, uploads the agents)
        enqueue(handle, steps)                 (asynchronous)
        ready(handle) -> bool                  (all enqueued work finished)
        result(handle) -> dict                 (reads the state back; may block briefly)
        close(handle)
    """

    def __init__(self, executor, budget_bytes=150e9, max_active=64, chunk=25, clock=time.perf_counter):
        self.ex = executor
        self.budget = budget_bytes
        self.max_active = max_active
        self.chunk = chunk
        self.clock = clock

    def run(self, requests, payload_of, time_scale=1.0):
        """Serve `requests` (sorted by arrival) in real time.  Returns the finished jobs."""
        t0 = self.clock()
        pending = list(requests)
        pending.sort(key=lambda r: r.arrival)
        waiting, active, finished = [], [], []
        used = 0
        i = 0
        while i < len(pending) or waiting or active:
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival * time_scale <= now:
                r = pending[i]
                waiting.append(Job(r, estimate_bytes(r.kind, r.n), r.steps))
                i += 1
            # admit in arrival order while memory and slots allow (no overtaking)
            while waiting and len(active) < self.max_active and used + waiting[0].bytes <= self.budget:
                job = waiting.pop(0)
                job.admitted = self.clock() - t0
                job.handle = self.ex.start(job.req, payload_of(job.req))
                used += job.bytes
                active.append(job)
            if waiting and not active and waiting[0].bytes > self.budget:
                raise RuntimeError("request %d needs more memory than the budget" % waiting[0].req.rid)
            # keep every active simulation's stream busy with its next chunk
            progressed = False
            for job in list(active):
                if self.ex.ready(job.handle):
                    if job.steps_left > 0:
                        k = min(self.chunk, job.steps_left)
                        self.ex.enqueue(job.handle, k)
                        job.steps_left -= k
                        progressed = True
                    else:
                        job.result = self.ex.result(job.handle)
                        job.done = self.clock() - t0
                        self.ex.close(job.handle)
                        used -= job.bytes
                        active.remove(job)
                        finished.append(job)
                        progressed = True
            if not progressed:
                if active:
                    time.sleep(0.0002)
                elif i < len(pending):
                    wait = pending[i].arrival * time_scale - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
        return finished


def run_one_at_a_time(executor, requests, payload_of, clock=time.perf_counter, time_scale=1.0):
    """Baseline: the same trace, FIFO, one simulation at a time, all its steps at once."""
    t0 = clock()
    finished = []
    for r in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if r.arrival * time_scale > now:
            time.sleep(r.arrival * time_scale - now)
        job = Job(r, estimate_bytes(r.kind, r.n), 0)
        job.admitted = clock() - t0
        h = executor.start(r, payload_of(r))
        executor.enqueue(h, r.steps)
        job.result = executor.result(h)
        job.done = clock() - t0
        executor.close(h)
        finished.append(job)
    return finished


def summarize(jobs, time_scale=1.0):
    lat = np.array([j.done - j.req.arrival * time_scale for j in jobs])
    makespan = max(j.done for j in jobs) if jobs else 0.0
    agent_steps = float(sum(j.req.n * j.req.steps for j in jobs))
    return {"requests": len(jobs), "sims_per_s": len(jobs) / makespan if makespan else 0.0,
            "agent_steps_per_s": agent_steps / makespan if makespan else 0.0,
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "makespan_s": makespan}


# ------------------------------------------------------------------------------------------------
# GPU executor over libbdm
# ------------------------------------------------------------------------------------------------
def payload(req):
    """The request's synthetic population (mechanics at the plain-mechanics density, SIR at the
    ensemble's density), seeded by the request."""
    if req.kind == "mechanics":
        params, inp = synth.served_mechanics(req.n, req.seed)
    else:
        params, inp = synth.served_sir(req.n, req.seed)
    return params, inp


class GpuExecutor:
    """Each simulation gets a libbdm handle on one of `streams` CUDA streams (round robin).
    `mechanics_skin` > 0 runs mechanics requests with neighbour lists of that skin (um; the
    interaction radius is then the request's largest diameter)."""

    def __init__(self, streams=8, mechanics_skin=0.0):
        import torch
        from . import bdm
        self.torch = torch
        self.bdm = bdm
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.next = 0
        self.skin = float(mechanics_skin)

    def start(self, req, pl):
        params, inp = pl
        if params["kind"] != "sir" and self.skin > 0.0:
            params = dict(params, interaction_radius=float(np.max(inp["diameter"])), skin=self.skin)
        s = self.streams[self.next % len(self.streams)]
        self.next += 1
        sim = self.bdm.Sim(params, stream=s)
        if params["kind"] == "sir":
            sim.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        else:
            sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
        ev = self.torch.cuda.Event()
        ev.record(s)
        return {"sim": sim, "stream": s, "event": ev, "kind": params["kind"]}

    def enqueue(self, h, steps):
        h["sim"].step(steps)
        h["event"].record(h["stream"])

    def ready(self, h):
        return h["event"].query()

    def result(self, h):
        fields = ("sir_state",) if h["kind"] == "sir" else ("x", "y", "z")
        st = h["sim"].get_state(fields=fields)
        return st

    def close(self, h):
        h["sim"].close()
