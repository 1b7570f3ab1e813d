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
