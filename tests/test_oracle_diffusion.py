"""Pins of the oracle's FTCS diffusion and secretion (CPU only): mass conservation with closed walls,
the exact decay recurrence, the exact discrete second moment of a point source (variance 2 D t per
axis) and the approach to the Gaussian profile."""
import math

import numpy as np

import oracle
from paper_2006_06775_gb300 import synth


def test_mass_conserved_with_closed_walls():
    u = synth.rng(21).uniform(0, 2, (20, 24, 28))
    m0 = u.sum()
    lam = 0.4 / 100.0
    for _ in range(50):
        u, m = oracle.ftcs(u, lam, 0.0)
    assert abs(m - m0) <= 1e-12 * m0
    assert abs(u.sum() - m) <= 1e-12 * m0


def test_decay_recurrence():
    u = synth.rng(22).uniform(0, 2, (16, 16, 16))
    m = u.sum()
    lam, mu_dt = oracle.ftcs_coefficients(0.4, 1.0, 10.0, 0.01)
    for _ in range(30):
        u, mass = oracle.ftcs(u, lam, mu_dt)
        m = (1.0 - mu_dt) * m
        assert abs(mass - m) <= 1e-12 * m


def test_secretion_then_decay_recurrence():
    params, inp = synth.spheroid()
    n = 64
    g = np.zeros((128, 128, 128))
    lam, mu_dt = oracle.ftcs_coefficients(0.4, 1.0, 10.0, 0.01)
    m = 0.0
    for _ in range(3):
        oracle.secrete(inp["x"][:n], inp["y"][:n], inp["z"][:n], g, params["grid_origin"], 10.0, 1.0)
        g, mass = oracle.ftcs(g, lam, mu_dt)
        m = (1.0 - mu_dt) * (m + n * 1.0)
        assert abs(mass - m) <= 1e-12 * m


def test_secretion_voxel_and_clamp():
    g = np.zeros((4, 4, 4))
    # inside, on a face, and far outside (clamped to the corner voxels)
    x = np.array([5.0, 10.0, -100.0, 100.0]); y = np.array([5.0, 5.0, -100.0, 100.0])
    z = np.array([5.0, 15.0, -100.0, 100.0])
    oracle.secrete(x, y, z, g, (0.0, 0.0, 0.0), 10.0, 2.0)
    assert g[0, 0, 0] == 4.0 and g[1, 0, 1] == 2.0 and g[3, 3, 3] == 2.0 and g.sum() == 8.0


def test_point_source_second_moment_is_2_lambda_n():
    n = 72
    u = np.zeros((n, n, n))
    c = n // 2
    u[c, c, c] = 1.0
    lam = 0.15
    steps = 30
    for _ in range(steps):
        u, mass = oracle.ftcs(u, lam, 0.0)
    idx = np.arange(n) - c
    for axis in range(3):
        marginal = u.sum(axis=tuple(a for a in range(3) if a != axis))
        mean = (marginal * idx).sum()
        var = (marginal * idx * idx).sum() - mean * mean
        assert abs(mean) < 1e-12
        assert abs(var - 2 * lam * steps) < 1e-10


def test_point_source_approaches_gaussian():
    n = 96
    u = np.zeros((n, n, n))
    c = n // 2
    u[c, c, c] = 1.0
    D, dt, h = 0.1, 1.0, 1.0  # lambda = 0.1 <= 1/6: stable
    lam, _ = oracle.ftcs_coefficients(D, dt, h, 0.0)
    steps = 100
    for _ in range(steps):
        u, _m = oracle.ftcs(u, lam, 0.0)
    sigma2 = 2 * D * dt * steps
    marginal = u.sum(axis=(0, 1))
    xs = np.arange(n) - c
    gauss = np.exp(-xs ** 2 / (2 * sigma2)) / math.sqrt(2 * math.pi * sigma2)
    core = np.abs(xs) <= 2 * math.sqrt(sigma2)
    rel = np.abs(marginal[core] - gauss[core]) / gauss[core]
    assert rel.max() < 0.03
