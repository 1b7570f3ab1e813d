"""GPU parity of the oncology behaviours (readings R13, R14) inside the growing spheroid: apoptosis at
step start and Brownian migration after the mechanical update.  Every step, from the GPU's own state,
one oracle step must give the same agents (count, ids, diameters, volumes: exact), the same neighbour
counts and grid assignment (exact) and the same positions within the path's tolerance."""
import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu


def oncology_params(precision, p_apo=0.02, sigma=0.5):
    params, inp = synth.spheroid(seed=4)
    params = dict(params, precision=precision, capacity=1 << 16, diffusion_enabled=0,
                  p_apoptosis=p_apo, brownian_sigma=sigma, run_id=3)
    return params, inp


@pytest.mark.parametrize("precision,tol", [("mixed", 2e-4), ("fp64", 1e-8)])
def test_spheroid_with_apoptosis_and_brownian_teacher_forced(precision, tol):
    params, inp = oncology_params(precision)
    sim = bdm.Sim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    prev = sim.get_state()
    for k in range(16):
        sim.step(1)
        got = sim.get_state()
        ref = oracle.OracleSim(dict(params, first_step=k))
        ref.add_agents(prev["x"], prev["y"], prev["z"], prev["diameter"], prev["volume"])
        ref.step(1)
        want = ref.get_state()
        assert got["n"] == want["n"], k
        for f in ("diameter", "volume", "neighbour_count", "box_id"):
            assert np.array_equal(got[f], want[f]), (k, f)
        for a in ("x", "y", "z"):
            assert np.max(np.abs(got[a] - want[a])) < tol, (k, a)
        prev = got
    assert prev["n"] > 512  # the spheroid still grows
    sim.close()


def test_apoptosis_alone_matches_the_oracle_count_and_order():
    """10^5 agents on a settled lattice, apoptosis only: the survivors and their order are exact."""
    params, inp = synth.settled_mechanics(100_000, 0.0, seed=13)
    params = dict(params, p_apoptosis=0.1, seed=21, run_id=1)
    sim = bdm.Sim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    ref = oracle.OracleSim(params)
    ref.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    for k in range(3):
        sim.step(1)
        ref.step(1)
        got, want = sim.get_state(), ref.get_state()
        assert got["n"] == want["n"], k
        for a in ("x", "y", "z"):
            assert np.array_equal(got[a], want[a]), (k, a)  # no contacts: positions only move by removal
        assert np.array_equal(got["diameter"], want["diameter"]), k
    assert abs(got["n"] / 100_000 - 0.9 ** 3) < 0.01
    sim.close()


def test_oncology_parameters_are_checked():
    params, inp = oncology_params("mixed")
    for bad in (dict(p_apoptosis=1.5), dict(brownian_sigma=-1.0),
                dict(growth_enabled=0, skin=2.0, interaction_radius=14.0)):
        with pytest.raises(bdm.BdmError):
            bdm.Sim(dict(params, **bad))


@pytest.mark.parametrize("precision,tol", [("mixed", 2e-4), ("fp64", 1e-8)])
def test_chemotaxis_teacher_forced(precision, tol):
    """Secreting spheroid on the co-stepped grid, agents following the gradient (reading R15): from
    the GPU's state and grid, one oracle step gives the same agents, counts and grid assignment, and
    positions within the path's tolerance."""
    params, inp = synth.spheroid(seed=5, grid_n=64)
    params = dict(params, precision=precision, capacity=1 << 15, chemotaxis=50.0,
                  grid_origin=(-320.0, -320.0, -320.0))
    sim = bdm.Sim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(3)  # some substance first
    prev = sim.get_state()
    moved = 0.0
    for k in range(3, 11):
        sim.step(1)
        got = sim.get_state()
        ref = oracle.OracleSim(dict(params, first_step=k))
        ref.add_agents(prev["x"], prev["y"], prev["z"], prev["diameter"], prev["volume"])
        ref.set_grid(prev["grid"])
        ref.step(1)
        want = ref.get_state()
        assert got["n"] == want["n"], k
        for f in ("diameter", "volume", "neighbour_count", "box_id"):
            assert np.array_equal(got[f], want[f]), (k, f)
        for a in ("x", "y", "z"):
            assert np.max(np.abs(got[a] - want[a])) < tol, (k, a)
        no_chemo = oracle.OracleSim(dict(params, first_step=k, chemotaxis=0.0))
        no_chemo.add_agents(prev["x"], prev["y"], prev["z"], prev["diameter"], prev["volume"])
        no_chemo.set_grid(prev["grid"])
        no_chemo.step(1)
        moved = max(moved, float(np.max(np.abs(want["x"] - no_chemo.get_state()["x"]))))
        prev = got
    assert moved > 1e-3  # the gradient term is not negligible in this test
    sim.close()
