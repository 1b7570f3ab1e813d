"""Handles built on device memory that still holds old data: every buffer a step reads before
writing must be initialised by the library.  The stream's cached blocks in PyTorch's allocator are
filled with 0xFF and freed first, so the handle's allocations come back holding all-ones bytes;
results must still equal the oracle (SIR) or a handle built on fresh memory (mechanics, growth,
diffusion) bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu

SIR_FIELDS = ("x", "y", "z", "sir_state", "neighbour_count", "box_id", "sir_counts")


def poisoned_stream():
    """A new stream whose allocator cache holds small and large blocks filled with 0xFF."""
    import torch
    s = torch.cuda.Stream()
    sizes = [4 << 10] * 256 + [64 << 10] * 64 + [512 << 10] * 32 + [1 << 20] * 16 + \
            [24 << 20] * 8 + [256 << 20] * 4
    with torch.cuda.stream(s):
        blocks = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in sizes]
        for b in blocks:
            b.fill_(0xFF)
    s.synchronize()
    del blocks
    return s


def sir_runs():
    specs = [(5000, 400.0, 16, 0.05), (3000, 150.0, 3, 0.05), (20000, 1000.0, 25, 0.05),
             (2500, 90.0, 6, 0.6)]
    out = []
    for k, (n, dom, nb, frac) in enumerate(specs):
        p = dict(kind="sir", seed=5, run_id=k, sir_domain=dom, sir_radius=6.0, sir_step=5.0,
                 sir_boxes=nb, p_infect=0.3, p_recover=0.02)
        x, y, z, st = synth.sir_run(n, 5, k, dom, infected_frac=frac)
        out.append((p, dict(x=x, y=y, z=z, sir_state=st)))
    return out


@pytest.mark.parametrize("steps", [1, 6])
def test_batch_on_stale_memory_matches_oracle(steps):
    runs = sir_runs()
    batch = bdm.Batch([p for p, _ in runs], stream=poisoned_stream())
    for k, (_, inp) in enumerate(runs):
        batch.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
    batch.step(steps)
    for k, (p, inp) in enumerate(runs):
        ref = oracle.OracleSim(p)
        ref.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        ref.step(steps)
        want, got = ref.get_state(), batch.get_state(k)
        for f in SIR_FIELDS:
            assert np.array_equal(got[f], want[f]), (k, f)
    batch.close()


def test_sir_handle_on_stale_memory_matches_oracle():
    p, inp = sir_runs()[0]
    sim = bdm.Sim(p, stream=poisoned_stream())
    ref = oracle.OracleSim(p)
    for s in (sim, ref):
        s.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
    for k in range(3):
        sim.step(1)
        ref.step(1)
        got, want = sim.get_state(), ref.get_state()
        for f in SIR_FIELDS:
            assert np.array_equal(got[f], want[f]), (k, f)
    sim.close()


def mech_cases():
    params, inp = synth.large_mechanics(n=200_000, seed=41, with_grid=False)
    yield "mixed", params, inp, 4
    yield "fp64", dict(params, precision="fp64"), inp, 2
    yield "skin", dict(params, interaction_radius=12.0, box_length=14.5, skin=2.5), inp, 6
    sp, si = synth.spheroid(grid_n=64)
    yield "spheroid", dict(sp, capacity=1 << 15, grid_origin=(-320.0, -320.0, -320.0)), si, 20


@pytest.mark.parametrize("name", ["mixed", "fp64", "skin", "spheroid"])
def test_mechanics_on_stale_memory_equals_fresh(name):
    import torch
    (params, inp, steps), = [(p, i, s) for n, p, i, s in mech_cases() if n == name]
    states = []
    for stream in (torch.cuda.Stream(), poisoned_stream()):
        sim = bdm.Sim(params, stream=stream)
        sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
        sim.step(steps)
        states.append(sim.get_state())
        sim.close()
    fresh, stale = states
    assert fresh["n"] == stale["n"]
    for f, v in fresh.items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, stale[f]), f
        else:
            assert v == stale[f], f
