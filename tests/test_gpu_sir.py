"""GPU parity of the SIR model (one run per handle): states, positions, infected-neighbour counts,
box ids and S/I/R counts bit-exact against the oracle every step."""
import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu


def sir_params(domain, boxes, seed=3, run=0, p_inf=0.3, p_rec=0.02, radius=6.0, step=5.0):
    return dict(kind="sir", seed=seed, run_id=run, sir_domain=domain, sir_radius=radius,
                sir_step=step, sir_boxes=boxes, p_infect=p_inf, p_recover=p_rec)


@pytest.mark.parametrize("n,domain,boxes,steps", [(5000, 400.0, 16, 30), (2000, 100.0, 1, 10),
                                                  (2000, 100.0, 2, 10), (3000, 150.0, 3, 10),
                                                  (20000, 1000.0, 40, 20), (1, 50.0, 2, 3)])
def test_sir_run_matches_oracle(n, domain, boxes, steps):
    params = sir_params(domain, boxes)
    x, y, z, st = synth.sir_run(n, 3, 0, domain, infected_frac=0.05)
    if n == 1:
        st[:] = 1
    sim = bdm.Sim(params)
    ref = oracle.OracleSim(params)
    for s in (sim, ref):
        s.add_agents(x, y, z, sir_state=st)
    for k in range(steps):
        sim.step(1)
        ref.step(1)
        got, want = sim.get_state(), ref.get_state()
        for f in ("x", "y", "z", "sir_state", "neighbour_count", "box_id", "sir_counts"):
            assert np.array_equal(got[f], want[f]), (k, f)


def test_sir_graph_replay_and_large_step_size():
    params = sir_params(300.0, 10, p_inf=0.4, step=140.0)
    x, y, z, st = synth.sir_run(4000, 5, 0, 300.0, infected_frac=0.02)
    sim = bdm.Sim(params)
    ref = oracle.OracleSim(params)
    for s in (sim, ref):
        s.add_agents(x, y, z, sir_state=st)
    sim.step(25)
    ref.step(25)
    got, want = sim.get_state(), ref.get_state()
    for f in ("x", "y", "z", "sir_state", "sir_counts"):
        assert np.array_equal(got[f], want[f]), f


def compare_all(sim, ref, tag):
    got, want = sim.get_state(), ref.get_state()
    for f in ("x", "y", "z", "sir_state", "neighbour_count", "box_id", "sir_counts"):
        assert np.array_equal(got[f], want[f]), (tag, f)


def test_sir_dense_infection_matches_oracle():
    """Most agents infected at a density of several agents per box: almost every agent pushes
    into its neighbours' counts, many of them into the same counters."""
    params = sir_params(120.0, 10, p_inf=0.5, p_rec=0.05)
    x, y, z, st = synth.sir_run(4000, 9, 0, 120.0, infected_frac=0.7)
    sim = bdm.Sim(params)
    ref = oracle.OracleSim(params)
    for s in (sim, ref):
        s.add_agents(x, y, z, sir_state=st)
    for k in range(12):
        sim.step(1)
        ref.step(1)
        compare_all(sim, ref, k)
    assert ref.get_state()["neighbour_count"].max() >= 3


def test_sir_agents_added_between_steps_and_after_reset():
    """Agents appended after steps join the grid index with the next ids; a reset empties the
    handle, and a new population then runs as on a fresh handle."""
    params = dict(sir_params(200.0, 8), capacity=3000)
    x, y, z, st = synth.sir_run(3000, 11, 0, 200.0, infected_frac=0.05)
    sim = bdm.Sim(params)
    ref = oracle.OracleSim(params)
    for s in (sim, ref):
        s.add_agents(x[:2000], y[:2000], z[:2000], sir_state=st[:2000])
        s.step(5)
        s.add_agents(x[2000:], y[2000:], z[2000:], sir_state=st[2000:])
        s.step(5)
    compare_all(sim, ref, "appended")
    sim.reset()
    ref = oracle.OracleSim(params)
    x2, y2, z2, st2 = synth.sir_run(1500, 12, 0, 200.0, infected_frac=0.1)
    for s in (sim, ref):
        s.add_agents(x2, y2, z2, sir_state=st2)
        s.step(4)
    compare_all(sim, ref, "after reset")

