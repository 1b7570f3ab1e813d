"""Serving: a request loop over the simulation library with continuous batching.

Requests (mechanics or SIR simulations of different sizes and step counts) arrive over time.  The
server admits them in arrival order while the estimated device memory of the admitted set stays
inside a budget and a place is free; admitted simulations keep their state resident on the device.
Two kinds of place:
  - a handle of its own on one of several CUDA streams: every pass of the loop enqueues the next
    chunk of steps (one CUDA-graph replay) for every such simulation, so work of different requests
    overlaps on the GPU;
  - a slot of the mechanics pool (bdm_mbatch), for mechanics requests up to the slot capacity: the
    pool advances all its simulations together, one launch sequence per step whatever their number,
    so small requests stop paying a dozen launches each per step.
A simulation whose last chunk has completed (checked with events, without blocking) has its state
read back to the host; its memory or slot returns to the pool and the next waiting request is
admitted.  Latency = time from arrival to the result on the host.

The scheduling logic only talks to "executors" (the `Executor` interface), so it is tested on the
CPU with fake executors; `GpuExecutor` drives libbdm.
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
    pooled: bool = False
    result: dict = field(default_factory=dict)


class Executor:
    """What the server needs from the library.  Own-handle simulations:
        start(req, payload) -> handle          (allocates, uploads the agents)
        enqueue(handle, steps)                 (asynchronous)
        ready(handle) -> bool                  (all enqueued work finished)
        result(handle) -> dict                 (reads the state back; may block briefly)
        close(handle)
    Pooled simulations (an executor with a pool overrides the last three): `pooled(req)` says the
    request runs in the pool, `pool_free()` that a slot is free; `start` then returns a handle that
    the pool steps by itself to the request's step count, `ready` turns true when its result is on
    the host, and `tick()`, called once per pass of the loop, drives the pool."""

    def pooled(self, req) -> bool:
        return False

    def pool_free(self) -> bool:
        return False

    def tick(self) -> None:
        pass


class Server:
    """Continuous-batching loop over an `Executor`.  `max_active` bounds the own-handle simulations;
    pooled ones are bounded by the pool's slots and hold no budget (the pool is allocated once)."""

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
        own = 0  # active simulations with a handle of their own
        i = 0
        while i < len(pending) or waiting or active:
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival * time_scale <= now:
                r = pending[i]
                waiting.append(Job(r, estimate_bytes(r.kind, r.n), r.steps))
                i += 1
            # admit in arrival order while memory and places allow (no overtaking)
            while waiting:
                job = waiting[0]
                job.pooled = self.ex.pooled(job.req)
                if job.pooled:
                    if not self.ex.pool_free():
                        break
                    job.bytes = 0
                    job.steps_left = 0
                elif own >= self.max_active or used + job.bytes > self.budget:
                    break
                waiting.pop(0)
                job.admitted = self.clock() - t0
                job.handle = self.ex.start(job.req, payload_of(job.req))
                used += job.bytes
                own += 0 if job.pooled else 1
                active.append(job)
            if waiting and not active and waiting[0].bytes > self.budget:
                raise RuntimeError("request %d needs more memory than the budget" % waiting[0].req.rid)
            self.ex.tick()
            # keep every own-handle simulation's stream busy with its next chunk
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
                        own -= 0 if job.pooled else 1
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


class GpuExecutor(Executor):
    """Each own-handle simulation gets a libbdm handle on one of `streams` CUDA streams (round
    robin).  `mechanics_skin` > 0 runs those mechanics requests with neighbour lists of that skin
    (um; the interaction radius is then the request's largest diameter).  `pool_slots` > 0 adds a
    mechanics pool (bdm_mbatch, mixed precision, grid rebuilt every step) of that many slots of
    `pool_capacity` agents on a stream of its own; mechanics requests up to the capacity run there,
    the pool advancing all of them `pool_chunk` steps per graph replay."""

    def __init__(self, streams=8, mechanics_skin=0.0, pool_slots=0, pool_capacity=32768,
                 pool_chunk=25):
        import torch
        from . import bdm
        self.torch = torch
        self.bdm = bdm
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.next = 0
        self.skin = float(mechanics_skin)
        self.pool = None
        if pool_slots > 0:
            self.pool_stream = torch.cuda.Stream()
            self.pool = bdm.MechBatch("mixed", slots=pool_slots, slot_capacity=pool_capacity,
                                      stream=self.pool_stream)
            self.pool_capacity = int(pool_capacity)
            self.pool_chunk = int(pool_chunk)
            self.free = list(range(pool_slots))[::-1]
            self.to_load, self.in_pool = [], []
            self.pool_event = torch.cuda.Event()
            self.pool_busy = False

    # ---- pool -------------------------------------------------------------------------------
    def pooled(self, req):
        return self.pool is not None and req.kind == "mechanics" and req.n <= self.pool_capacity

    def pool_free(self):
        return bool(self.free)

    def tick(self):
        """When the pool's last chunk has finished: read out and release the simulations that
        reached their step count, load the admitted ones, and enqueue the next chunk."""
        if self.pool is None or (self.pool_busy and not self.pool_event.query()):
            return
        self.pool_busy = False
        if self.in_pool:
            done = self.pool.poll()  # the pool's stream is idle: no wait
            for h in list(self.in_pool):
                if done[h["slot"]] >= h["steps"]:
                    h["result"] = self.pool.get_state(h["slot"], fields=("x", "y", "z"))
                    self.pool.release(h["slot"])
                    self.free.append(h["slot"])
                    self.in_pool.remove(h)
        for h in self.to_load:
            params, inp = h.pop("payload")
            self.pool.load_sim(h["slot"], params, inp["x"], inp["y"], inp["z"], inp["diameter"],
                               h["steps"])
            self.in_pool.append(h)
        self.to_load = []
        if self.in_pool:
            self.pool.step(self.pool_chunk)
            self.pool_event.record(self.pool_stream)
            self.pool_busy = True

    def warm_pool(self, payload, steps):
        """Capture the pool's graphs before a timed run (one small simulation, run to its end)."""
        params, inp = payload
        slot = self.free.pop()
        self.pool.load_sim(slot, params, inp["x"], inp["y"], inp["z"], inp["diameter"], steps)
        for _ in range(-(-steps // self.pool_chunk) + 1):
            self.pool.step(self.pool_chunk)
        self.pool.poll()
        self.pool.release(slot)
        self.free.append(slot)

    # ---- own handles and pooled handles -------------------------------------------------------
    def start(self, req, pl):
        params, inp = pl
        if self.pooled(req):
            h = {"pooled": True, "slot": self.free.pop(), "steps": req.steps, "payload": pl,
                 "result": None}
            self.to_load.append(h)
            return h
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
        return {"pooled": False, "sim": sim, "stream": s, "event": ev, "kind": params["kind"]}

    def enqueue(self, h, steps):
        h["sim"].step(steps)
        h["event"].record(h["stream"])

    def ready(self, h):
        if h["pooled"]:
            return h["result"] is not None
        return h["event"].query()

    def result(self, h):
        if h["pooled"]:
            return h["result"]
        fields = ("sir_state",) if h["kind"] == "sir" else ("x", "y", "z")
        st = h["sim"].get_state(fields=fields)
        return st

    def close(self, h):
        if not h["pooled"]:
            h["sim"].close()

    def shutdown(self):
        if self.pool is not None:
            self.pool.close()
            self.pool = None
