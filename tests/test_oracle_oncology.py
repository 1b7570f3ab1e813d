"""Oracle pins for the oncology behaviours: Brownian migration (reading R13) and apoptosis (reading
R14).  The deviates must be standard normal and independent across axes; apoptosis must remove the
expected binomial fraction, keep the survivors' order, and reduce to the identity at p = 0 and to an
empty population at p = 1."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2006_06775_gb300 import synth


def test_brownian_deviates_are_standard_normal():
    n, sigma = 200_000, 0.7
    zero = np.zeros(n)
    x, y, z = oracle.brownian(zero, zero, zero, sigma, 11, 3, 5)
    g = np.stack([x, y, z], 1) / sigma
    tol_mean = 5.0 / math.sqrt(n)
    tol_var = 5.0 * math.sqrt(2.0 / n)
    assert np.all(np.abs(g.mean(0)) < tol_mean)
    assert np.all(np.abs(g.var(0) - 1.0) < tol_var)
    c = np.corrcoef(g.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < tol_mean)
    for a in range(3):
        assert stats.kstest(g[:, a], "norm").pvalue > 1e-3
    # a different step draws different deviates
    x2, _, _ = oracle.brownian(zero, zero, zero, sigma, 11, 3, 6)
    assert abs(np.corrcoef(x, x2)[0, 1]) < tol_mean


def test_apoptosis_removes_a_binomial_fraction_in_order():
    n, p = 100_000, 0.2
    g = synth.rng(12)
    x, y, z = g.uniform(0, 100, n), g.uniform(0, 100, n), g.uniform(0, 100, n)
    d = np.full(n, 10.0, np.float32)
    v = np.arange(n, dtype=np.float64)  # tags the agents
    r = oracle.apoptosis(x, y, z, d, v, p, 4, 1, 7)
    m = len(r["x"])
    assert abs(m / n - (1.0 - p)) < 5.0 * math.sqrt(p * (1.0 - p) / n)
    kept = r["volume"].astype(np.int64)
    assert np.all(np.diff(kept) > 0)  # survivors keep their relative order
    assert np.array_equal(r["x"], x[kept]) and np.array_equal(r["z"], z[kept])
    assert len(oracle.apoptosis(x, y, z, d, v, 0.0, 4, 1, 7)["x"]) == n
    assert len(oracle.apoptosis(x, y, z, d, v, 1.0, 4, 1, 7)["x"]) == 0


def test_settled_lattice_moves_by_the_brownian_deviates_only():
    """On a lattice without contacts an oracle step is the Brownian move alone."""
    params, inp = synth.settled_mechanics(2000, 0.0, seed=8)
    params = dict(params, brownian_sigma=0.5, seed=9, run_id=2)
    sim = oracle.OracleSim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(1)
    got = sim.get_state()
    want = oracle.brownian(inp["x"], inp["y"], inp["z"], 0.5, 9, 2, 0)
    for a, w in zip(("x", "y", "z"), want):
        assert np.array_equal(got[a], w)


def test_apoptosis_in_the_step_survival_follows_the_power_law():
    params, inp = synth.settled_mechanics(20_000, 0.0, seed=10)
    p = 0.05
    params = dict(params, p_apoptosis=p, seed=1, run_id=0)
    sim = oracle.OracleSim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(6)
    m = sim.get_state()["n"]
    q = (1.0 - p) ** 6
    assert abs(m / 20_000 - q) < 5.0 * math.sqrt(q * (1.0 - q) / 20_000)
