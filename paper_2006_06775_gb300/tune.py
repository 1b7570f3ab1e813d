"""Autotuner for the tunable knobs of a workload, measured on the GPU.

Knobs (none changes a result beyond FP32 summation order; neighbour counts, grid membership tests
and SIR states are exact for every choice):
  mechanics   box_factor    grid box = factor x interaction radius (>= 1: the 27-box search stays
                            exact; bigger boxes mean fewer boxes but more candidates per agent)
              force_variant 0 = one thread per agent, 1 = warp-shared (agent, candidate) pairs
              skin          sort cadence: 0 = grid rebuilt every step; s > 0 = neighbour lists of
                            radius R + s, the grid rebuilt only when an agent may have moved more
                            than s / 2 (the grid box is then R + s)
  SIR         sir_boxes     boxes per axis (a divisor of the lattice side with box >= r)

The FP64 check path keeps the canonical (box, id) order of every step (it fixes the summation order
that makes it bit-exact), so it always rebuilds every step.

`tune_*` time each candidate for a few steps (CUDA events on the simulation's stream) and return
the fastest; `TuneCache` keeps choices per (workload signature, GPU) in a small JSON file.
"""
import json
import math
import os

import numpy as np

MECH_CANDIDATES = ([dict(box_factor=1.0, force_variant=0, skin=0.0),
                    dict(box_factor=1.15, force_variant=0, skin=0.0),
                    dict(box_factor=1.0, force_variant=1, skin=0.0)] +
                   [dict(box_factor=1.0, force_variant=0, skin=s) for s in (1.0, 1.5, 2.0, 2.5, 3.0, 3.5)])


def workload_signature(params, n, volume):
    """Kind, precision, size bucket (powers of 2) and density bucket (quarter decades)."""
    dens = n / max(volume, 1e-30)
    return "%s/%s/n2^%d/rho10^%.2f" % (params.get("kind", "mechanics"),
                                       params.get("precision", "mixed"),
                                       int(round(math.log2(max(n, 1)))),
                                       round(4 * math.log10(max(dens, 1e-30))) / 4)


def gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


class TuneCache:
    def __init__(self, path):
        self.path = path
        self.data = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)

    def get(self, sig, gpu):
        return self.data.get(gpu, {}).get(sig)

    def put(self, sig, gpu, choice):
        self.data.setdefault(gpu, {})[sig] = choice
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def choose(candidates, measure):
    """Measure every candidate (ms per step) and return (best, table)."""
    table = []
    for cand in candidates:
        ms = float(measure(cand))
        table.append(dict(cand, ms_per_step=ms))
    best = min(table, key=lambda r: r["ms_per_step"])
    return best, table


def mechanics_params(params, inputs, cand):
    p = dict(params)
    R = params.get("interaction_radius") or float(np.max(inputs["diameter"]))
    p["box_length"] = cand["box_factor"] * R if cand["box_factor"] != 1.0 else 0.0
    p["force_variant"] = cand["force_variant"]
    p["skin"] = cand.get("skin", 0.0)  # with a skin, box_length 0 means R + skin
    return p


def gpu_measure_mechanics(params, inputs, steps=10, warmup=3):
    """Measurement function for `choose`: ms per step of one candidate on the GPU."""
    import torch
    from . import bdm

    def measure(cand):
        p = mechanics_params(params, inputs, cand)
        p.pop("diffusion_enabled", None)
        sim = bdm.Sim(p)
        sim.add_agents(inputs["x"], inputs["y"], inputs["z"], inputs["diameter"])
        sim.step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        sim.close()
        return e0.elapsed_time(e1) / steps
    return measure


def tune_mechanics(params, inputs, volume, cache=None, measure=None, candidates=None):
    sig = workload_signature(params, len(inputs["x"]), volume)
    gpu = gpu_name()
    if cache is not None:
        hit = cache.get(sig, gpu)
        if hit is not None:
            return hit
    best, table = choose(candidates or MECH_CANDIDATES,
                         measure or gpu_measure_mechanics(params, inputs))
    choice = {"box_factor": best["box_factor"], "force_variant": best["force_variant"],
              "skin": best.get("skin", 0.0), "ms_per_step": best["ms_per_step"], "table": table,
              "signature": sig}
    if cache is not None:
        cache.put(sig, gpu, choice)
    return choice


def sir_box_candidates(params, n):
    """Divisors of the lattice side near (0.5 .. 2) x n^(1/3) with box side >= r."""
    L = int(round(params["sir_domain"] * 1024))
    r = int(round(params["sir_radius"] * 1024))
    hi = L // r if r > 0 else L
    out = set()
    base = max(1.0, n ** (1.0 / 3.0))
    for f in (0.5, 0.7, 1.0, 1.25, 1.5, 2.0):
        t = min(hi, max(1, int(base * f)))
        for nb in range(t, 0, -1):
            if L % nb == 0:
                out.add(nb)
                break
    return sorted(out)


def gpu_measure_sir_batch(param_list, inputs, steps=20, warmup=3):
    import time
    from . import bdm

    def measure(cand):
        ps = [dict(p, sir_boxes=cand["sir_boxes"]) for p in param_list]
        b = bdm.Batch(ps)
        for k, inp in enumerate(inputs):
            b.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
        b.step(warmup)
        b.sync()
        t0 = time.perf_counter()
        b.step(steps)
        b.sync()
        dt = time.perf_counter() - t0
        b.close()
        return 1e3 * dt / steps
    return measure


def tune_sir_batch(param_list, inputs, cache=None, measure=None):
    n = len(inputs[0]["x"])
    L = param_list[0]["sir_domain"]
    sig = "sir-batch/%d-runs/" % len(param_list) + workload_signature(param_list[0], n, L ** 3)
    gpu = gpu_name()
    if cache is not None:
        hit = cache.get(sig, gpu)
        if hit is not None:
            return hit
    cands = [dict(sir_boxes=nb) for nb in sir_box_candidates(param_list[0], n)]
    best, table = choose(cands, measure or gpu_measure_sir_batch(param_list, inputs))
    choice = {"sir_boxes": best["sir_boxes"], "ms_per_step": best["ms_per_step"], "table": table,
              "signature": sig}
    if cache is not None:
        cache.put(sig, gpu, choice)
    return choice
