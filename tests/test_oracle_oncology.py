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


def _voxel_centres(n, h, o):
    return o + h * (np.arange(n) + 0.5)


def test_chemotaxis_follows_a_linear_field_exactly():
    """On c = a.x + b the central and one-sided differences are exact: every agent, inside or at a
    wall, moves by chi * a; a constant field moves nobody."""
    nx, ny, nz, h, o = 7, 5, 4, 2.0, (-3.0, 1.0, 0.5)
    a = np.array([0.25, -0.5, 1.5])
    zc, yc, xc = np.meshgrid(_voxel_centres(nz, h, o[2]), _voxel_centres(ny, h, o[1]),
                             _voxel_centres(nx, h, o[0]), indexing="ij")
    grid = a[0] * xc + a[1] * yc + a[2] * zc + 3.0
    g = synth.rng(14)
    n = 500
    sx = g.uniform(o[0] - 1.0, o[0] + nx * h + 1.0, n)  # some outside: clamped to the wall voxels
    sy = g.uniform(o[1], o[1] + ny * h, n)
    sz = g.uniform(o[2], o[2] + nz * h, n)
    chi = 0.7
    x, y, z = oracle.chemotaxis(sx, sy, sz, sx, sy, sz, grid, o, h, chi)
    for got, start, ak in ((x, sx, a[0]), (y, sy, a[1]), (z, sz, a[2])):
        assert np.allclose(got - start, chi * ak, rtol=0, atol=1e-12)
    x, y, z = oracle.chemotaxis(sx, sy, sz, sx, sy, sz, np.full_like(grid, 2.0), o, h, chi)
    assert np.array_equal(x, sx) and np.array_equal(y, sy) and np.array_equal(z, sz)


def test_chemotaxis_moves_up_a_parabola():
    """c = x^2 along x: inside, the central difference equals the derivative 2 x at the voxel
    centre, and agents move towards higher concentration."""
    nx, h, o = 9, 1.0, (0.0, 0.0, 0.0)
    xc = _voxel_centres(nx, h, 0.0)
    grid = np.broadcast_to((xc - 4.5) ** 2, (1, 1, nx)).copy()
    sx = xc[1:-1].copy()
    zero = np.zeros_like(sx)
    x, _, _ = oracle.chemotaxis(sx, zero, zero, sx, zero, zero, grid, o, h, 1.0)
    assert np.allclose(x - sx, 2.0 * (sx - 4.5), atol=1e-12)
    assert np.all(np.sign(x - sx) == np.sign(sx - 4.5))
