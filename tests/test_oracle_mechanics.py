"""Pins of the FP64 oracle's grid, neighbour search, force law and update (CPU only).

Each test checks the oracle against something other than itself: an O(N^2) brute force with no
grid, a closed form, an invariant of the pair law, or an equivalent problem.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import synth


def brute_neighbour_counts(x, y, z, R):
    """All-pairs count of j != i with (dx*dx + dy*dy) + dz*dz < R*R, no grid."""
    dx = x[:, None] - x[None, :]
    dy = y[:, None] - y[None, :]
    dz = z[:, None] - z[None, :]
    d2 = dx * dx + dy * dy
    d2 = d2 + dz * dz
    hit = d2 < R * R
    np.fill_diagonal(hit, False)
    return hit.sum(axis=1).astype(np.uint32)


def step(x, y, z, d, **kw):
    p = dict(dt=0.01, repulsion=2.0, attraction=1.0, max_displacement=3.0)
    p.update(kw)
    return oracle.mech_step(x, y, z, d, p["dt"], p["repulsion"], p["attraction"],
                            p["max_displacement"], p.get("interaction_radius", 0.0),
                            p.get("box_length", 0.0), want_force=True)


@pytest.mark.parametrize("n,side,seed", [(512, 60.0, 11), (512, 200.0, 12), (300, 20.0, 13)])
def test_neighbour_counts_equal_brute_force(n, side, seed):
    x, y, z, d = synth.uniform_spheres(n, side, seed)
    r = step(x, y, z, d)
    R = float(d.astype(np.float64).max())
    assert np.array_equal(r["neighbour_count"], brute_neighbour_counts(x, y, z, R))


def test_neighbour_counts_plain_mechanics_population():
    params, inp = synth.plain_mechanics()
    r = step(inp["x"], inp["y"], inp["z"], inp["diameter"])
    R = float(inp["diameter"].astype(np.float64).max())
    assert np.array_equal(r["neighbour_count"],
                          brute_neighbour_counts(inp["x"], inp["y"], inp["z"], R))
    assert r["neighbour_count"].mean() > 3  # heavily overlapping population


def test_agents_on_box_faces_and_lattice():
    # Centres exactly on box faces of a 12 um box (lattice spacing = box length) and at half steps.
    g = np.arange(6, dtype=np.float64) * 12.0
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = xx.ravel(), yy.ravel(), zz.ravel()
    x = np.concatenate([x, x[:50] + 6.0])
    y = np.concatenate([y, y[:50]])
    z = np.concatenate([z, z[:50] + 12.0])
    d = np.full(len(x), 12.0, np.float32)
    r = step(x, y, z, d)
    assert np.array_equal(r["neighbour_count"], brute_neighbour_counts(x, y, z, 12.0))


def test_two_sphere_closed_form():
    # r = 5 and 5 at distance 8: delta = 2, reduced radius 2.5, F = 2*2 - 1*sqrt(5).
    x = np.array([0.0, 8.0]); y = np.zeros(2); z = np.zeros(2)
    d = np.array([10.0, 10.0], np.float32)
    r = step(x, y, z, d)
    F = 4.0 - math.sqrt(5.0)
    assert abs(r["force"][0, 0] + F) < 1e-14 and abs(r["force"][1, 0] - F) < 1e-14
    assert abs(r["x"][0] - (0.0 - 0.01 * F)) < 1e-15
    assert abs(r["x"][1] - (8.0 + 0.01 * F)) < 1e-15
    assert np.array_equal(r["neighbour_count"], [1, 1])


def test_two_sphere_attraction_and_unequal_radii():
    # r = 5 and 5 at distance 9.9: delta = 0.1, F = 0.2 - sqrt(0.25) = -0.3 (net attraction).
    x = np.array([0.0, 9.9]); y = np.zeros(2); z = np.zeros(2)
    r = step(x, y, z, np.array([10.0, 10.0], np.float32))
    delta = 10.0 - 9.9
    F = 2.0 * delta - math.sqrt(2.5 * delta)
    assert F < 0
    assert abs(r["force"][1, 0] - F) < 1e-13
    # r = 3 and 6 along a diagonal at distance 7: delta = 2, reduced radius 2.
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    x = np.array([1.0, 1.0 + 7 * u[0]]); y = np.array([2.0, 2.0 + 7 * u[1]])
    z = np.array([3.0, 3.0 + 7 * u[2]])
    r = step(x, y, z, np.array([6.0, 12.0], np.float32), repulsion=1.5, attraction=0.5)
    F = 1.5 * 2.0 - 0.5 * math.sqrt(2.0 * 2.0)
    np.testing.assert_allclose(r["force"][1], F * u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["force"][0], -F * u, rtol=0, atol=1e-13)


def test_no_force_without_contact_and_single_agent():
    x = np.array([0.0, 10.5]); y = np.zeros(2); z = np.zeros(2)
    r = step(x, y, z, np.array([10.0, 11.0], np.float32))
    assert np.all(r["force"] == 0) and np.array_equal(r["x"], x)
    assert np.array_equal(r["neighbour_count"], [1, 1])  # within R = 11 but not touching
    r = step(np.array([3.0]), np.array([4.0]), np.array([5.0]), np.array([9.0], np.float32))
    assert r["x"][0] == 3.0 and r["neighbour_count"][0] == 0
    r = step(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0, np.float32))
    assert len(r["x"]) == 0


def test_coincident_centres_count_but_do_not_push():
    x = np.array([1.0, 1.0, 30.0]); y = np.array([2.0, 2.0, 2.0]); z = np.array([3.0, 3.0, 3.0])
    r = step(x, y, z, np.array([10.0, 10.0, 10.0], np.float32))
    assert np.array_equal(r["neighbour_count"], [1, 1, 0])
    assert np.array_equal(r["x"], x)


def test_net_force_vanishes():
    params, inp = synth.plain_mechanics()
    r = step(inp["x"], inp["y"], inp["z"], inp["diameter"])
    F = r["force"]
    total = F.sum(axis=0)
    scale = np.abs(F).sum()
    assert scale > 0
    assert np.all(np.abs(total) <= 1e-12 * scale)


def test_displacement_cap():
    # Deep overlap: F = 2*9.5 - sqrt(2.5*9.5) ~ 14.1 with dt = 1 -> capped to 3 along the axis.
    u = np.array([2.0, -3.0, 6.0]) / 7.0
    x = np.array([0.0, 0.5 * u[0]]); y = np.array([0.0, 0.5 * u[1]]); z = np.array([0.0, 0.5 * u[2]])
    r = step(x, y, z, np.array([10.0, 10.0], np.float32), dt=1.0)
    dvec = np.array([r["x"][1] - x[1], r["y"][1] - y[1], r["z"][1] - z[1]])
    assert abs(np.linalg.norm(dvec) - 3.0) < 1e-14
    np.testing.assert_allclose(dvec / 3.0, u, atol=1e-14)
    # Below the cap the displacement is dt * F exactly along the line.
    r = step(x, y, z, np.array([10.0, 10.0], np.float32), dt=0.1)
    dvec = np.array([r["x"][1] - x[1], r["y"][1] - y[1], r["z"][1] - z[1]])
    F = 2.0 * 9.5 - math.sqrt(2.5 * 9.5)
    np.testing.assert_allclose(dvec, 0.1 * F * u, atol=1e-13)


def test_larger_box_same_neighbours_and_forces():
    params, inp = synth.plain_mechanics()
    a = step(inp["x"], inp["y"], inp["z"], inp["diameter"])
    b = step(inp["x"], inp["y"], inp["z"], inp["diameter"], box_length=24.5)
    assert np.array_equal(a["neighbour_count"], b["neighbour_count"])
    assert b["grid"]["nbox"] < a["grid"]["nbox"]
    np.testing.assert_allclose(a["force"], b["force"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a["x"], b["x"], rtol=1e-14, atol=1e-13)


def test_grid_lattice_quantisation_and_faces():
    # Box length 1 um, Q = 20: a centre exactly on a face belongs to the upper box.
    x = np.array([0.0, 1.0, 2.0, 2.999999, 3.0]); y = np.zeros(5); z = np.zeros(5)
    g, box = oracle.grid(x, y, z, np.ones(5, np.float32))
    assert g["Lq"] == 1 << 20 and list(g["dims"]) == [4, 1, 1]
    assert list(box) == [0, 1, 2, 2, 3]
    # Interaction radius larger than the box is rejected.
    with pytest.raises(ValueError):
        oracle.grid(x, y, z, np.ones(5, np.float32), interaction_radius=2.0, box_length=1.0)


def test_all_agents_in_one_box():
    g = synth.rng(5)
    x, y, z = (g.uniform(0, 3.0, 64) for _ in range(3))
    d = np.full(64, 11.0, np.float32)
    r = step(x, y, z, d)
    assert r["grid"]["nbox"] == 1
    assert np.all(r["neighbour_count"] == 63)
    F = r["force"]
    assert np.all(np.abs(F.sum(axis=0)) <= 1e-12 * np.abs(F).sum())


def test_settled_lattice_agents_do_not_move():
    """The settled workload's premise: lattice agents (no contact within the largest diameter) get
    exactly zero displacement from the oracle, while the packed ball moves."""
    params, inp = synth.settled_mechanics(3000, 0.2, seed=7)
    x, y, z, d = inp["x"], inp["y"], inp["z"], inp["diameter"]
    out = oracle.mech_step(x, y, z, d, params["dt"], params["repulsion"], params["attraction"],
                           params["max_displacement"], 12.0, 0.0)
    moved = (out["x"] != x) | (out["y"] != y) | (out["z"] != z)
    na = inp["n_active"]
    r = np.sqrt(x ** 2 + y ** 2 + z ** 2)
    far = np.arange(len(x)) >= na
    far &= r > inp["ball_radius"] + 2 * 14.0
    assert far.sum() > 1000
    assert not moved[far].any()
    assert moved[:na].mean() > 0.5
