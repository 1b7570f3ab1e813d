"""GPU parity of the mechanics hot path (grid rebuild, 27-box neighbour search, sphere-sphere force,
capped update) against the FP64 oracle, through the C ABI.

Bar: grid assignment and neighbour counts bit-exact; FP64 positions within 1e-9 relative after 10
steps; mixed precision (FP32 forces, FP64 positions) teacher-forced per step with bit-exact integer
state, and its position deviation bounded and reported.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu

FP64_REL = 1e-9


def make_pair(params, inp):
    sim = bdm.Sim(params)
    ref = oracle.OracleSim(params)
    for s in (sim, ref):
        s.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"], inp.get("volume"))
    return sim, ref


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))) if len(b) else 0.0


def assert_step_equal(got, want, rel=FP64_REL):
    assert got["n"] == want["n"]
    assert np.array_equal(got["box_id"], want["box_id"])
    assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
    for a in ("x", "y", "z"):
        assert rel_err(got[a], want[a]) <= rel, a


def test_fp64_plain_mechanics_ten_steps():
    params, inp = synth.plain_mechanics()
    sim, ref = make_pair(params, inp)
    bitexact = True
    for _ in range(10):
        sim.step(1)
        ref.step(1)
        got, want = sim.get_state(), ref.get_state()
        assert_step_equal(got, want)
        bitexact &= all(np.array_equal(got[a], want[a]) for a in ("x", "y", "z"))
    assert got["step"] == 10
    g = ref.last_grid
    assert list(got["grid_origin_q"]) == list(g["origin_q"]) and got["grid_box_q"] == g["Lq"]
    assert list(got["grid_dims"]) == list(g["dims"])
    # the FP64 path follows the oracle's rounded operations in the same order
    assert bitexact
    sim.close()


def test_graph_replay_equals_single_steps():
    params, inp = synth.plain_mechanics(n=2000, side=120.0, seed=7)
    a = bdm.Sim(params)
    b = bdm.Sim(params)
    for s in (a, b):
        s.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    a.step(6)
    for _ in range(6):
        b.step(1)
    ga, gb = a.get_state(), b.get_state()
    for f in ("x", "y", "z", "neighbour_count", "box_id"):
        assert np.array_equal(ga[f], gb[f])
    a.step(6)  # replay of the cached 6-step graph
    for _ in range(6):
        b.step(1)
    ga, gb = a.get_state(), b.get_state()
    for f in ("x", "y", "z", "neighbour_count", "box_id"):
        assert np.array_equal(ga[f], gb[f])


def lattice_on_faces():
    g = np.arange(6, dtype=np.float64) * 12.0
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = xx.ravel(), yy.ravel(), zz.ravel()
    return dict(x=np.concatenate([x, x[:50] + 6.0]), y=np.concatenate([y, y[:50]]),
                z=np.concatenate([z, z[:50] + 12.0]), diameter=np.full(266, 12.0, np.float32))


def one_box():
    g = synth.rng(5)
    return dict(x=g.uniform(0, 3.0, 64), y=g.uniform(0, 3.0, 64), z=g.uniform(0, 3.0, 64),
                diameter=np.full(64, 11.0, np.float32))


def coincident():
    return dict(x=np.array([1.0, 1.0, 30.0]), y=np.array([2.0, 2.0, 2.0]),
                z=np.array([3.0, 3.0, 3.0]), diameter=np.full(3, 10.0, np.float32))


def single():
    return dict(x=np.array([3.0]), y=np.array([4.0]), z=np.array([5.0]),
                diameter=np.array([9.0], np.float32))


def ragged(n, side, seed):
    x, y, z, d = synth.uniform_spheres(n, side, seed)
    return dict(x=x, y=y, z=z, diameter=d)


CASES = {
    "single": (single, {}),
    "coincident": (coincident, {}),
    "one_box": (one_box, {}),
    "faces": (lattice_on_faces, {}),
    "bigger_box": (lambda: ragged(3000, 150.0, 3), {"box_length": 24.5}),
    "fixed_radius": (lambda: ragged(3000, 150.0, 4), {"interaction_radius": 13.0}),
    "multi_tile": (lambda: ragged(20000, 300.0, 5), {}),
    "negative_coords": (lambda: {k: (v - 77.7 if k != "diameter" else v)
                                 for k, v in ragged(5000, 170.0, 6).items()}, {}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_edge_cases(case):
    make, extra = CASES[case]
    inp = make()
    params = dict(synth.MECH_DEFAULTS, precision="fp64", **extra)
    sim, ref = make_pair(params, inp)
    for _ in range(3):
        sim.step(1)
        ref.step(1)
        assert_step_equal(sim.get_state(), ref.get_state())


def test_empty_simulation_steps():
    params = dict(synth.MECH_DEFAULTS, precision="fp64", capacity=16, box_capacity=64)
    sim = bdm.Sim(params)
    sim.step(3)
    st = sim.get_state()
    assert st["n"] == 0 and st["step"] == 3


def test_capacity_is_enforced():
    params = dict(synth.MECH_DEFAULTS, precision="fp64", capacity=4)
    sim = bdm.Sim(params)
    inp = ragged(5, 50.0, 1)
    with pytest.raises(bdm.BdmError) as e:
        sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    assert e.value.code == bdm.BDM_ENOMEM


def test_grid_overflow_is_reported_not_faulted():
    params = dict(synth.MECH_DEFAULTS, precision="fp64", capacity=8, box_capacity=8)
    sim = bdm.Sim(params)
    inp = ragged(8, 500.0, 2)  # needs ~40^3 boxes
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(1)
    with pytest.raises(bdm.BdmError) as e:
        sim.get_state()
    assert e.value.code == bdm.BDM_ENOMEM and "box_capacity" in str(e.value)


def test_mixed_teacher_forced_integer_state_exact():
    """Population at the large workload's density (0.3 volume fraction), ~300k agents over many
    scan tiles: from the same state, one mixed step reproduces grid assignment and neighbour counts
    exactly, and positions to within FP32 force error."""
    n = 300_000
    params, inp = synth.large_mechanics(n=n, seed=12, with_grid=False)
    x, y, z, d = inp["x"], inp["y"], inp["z"], inp["diameter"]
    sim = bdm.Sim(params)
    worst = 0.0
    for k in range(3):
        sim.reset()
        sim.add_agents(x, y, z, d)
        sim.step(1)
        got = sim.get_state()
        want = oracle.mech_step(x, y, z, d, params["dt"], params["repulsion"], params["attraction"],
                                params["max_displacement"])
        assert np.array_equal(got["box_id"], want["box_id"])
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
        dev = max(float(np.max(np.abs(got[a] - want[a]))) for a in ("x", "y", "z"))
        worst = max(worst, dev)
        x, y, z = want["x"], want["y"], want["z"]
    assert worst < 2e-5, worst


def test_dense_spheroid_teacher_forced():
    """A densely packed state (the tumour spheroid after 52 steps of growth and division: tens of
    agents per box, hundreds of neighbours and contacts per agent): from the same state, mixed
    mechanics steps reproduce grid assignment and neighbour counts exactly.  Exercises the
    collective contact flush of dense rows and the band queue under heavy load."""
    params, inp = synth.spheroid()
    grow = bdm.Sim(dict(params, capacity=1 << 17, diffusion_enabled=0))
    grow.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    grow.step(52)
    s = grow.get_state()
    assert s["n"] >= 32768
    mech = dict(params, growth_enabled=0, diffusion_enabled=0)
    x, y, z, d = s["x"], s["y"], s["z"], s["diameter"]
    sim = bdm.Sim(mech)
    worst = 0.0
    for k in range(3):
        sim.reset()
        sim.add_agents(x, y, z, d)
        sim.step(1)
        got = sim.get_state()
        want = oracle.mech_step(x, y, z, d, mech["dt"], mech["repulsion"], mech["attraction"],
                                mech["max_displacement"], mech["interaction_radius"])
        assert np.array_equal(got["box_id"], want["box_id"]), k
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"]), k
        worst = max(worst, max(float(np.max(np.abs(got[a] - want[a]))) for a in ("x", "y", "z")))
        x, y, z = want["x"], want["y"], want["z"]
    assert want["neighbour_count"].mean() > 100
    assert worst < 2e-4, worst


def test_band_queue_overflow_is_recounted_exactly():
    """An agent with 40 others at distance R (1 +- 2e-8): all fall in the FP32 band around R^2, more
    than the per-thread band queue holds, so its count comes from the exact second pass; the FP64
    decisions must split the shell exactly as the oracle does."""
    R = 12.0
    g = np.random.default_rng(5)
    m = 40
    k = np.arange(m) + 0.5
    theta = np.arccos(1 - 2 * k / m)
    phi = np.pi * (1 + 5 ** 0.5) * k
    dirs = np.stack([np.cos(phi) * np.sin(theta), np.sin(phi) * np.sin(theta), np.cos(theta)], 1)
    sign = np.where(np.arange(m) % 2 == 0, 1.0, -1.0)
    centre = np.array([300.0, 300.0, 300.0]) + g.uniform(0, 1, 3)
    pts = centre + dirs * (R * (1 + sign * 2e-8))[:, None]
    x = np.concatenate([[centre[0]], pts[:, 0]])
    y = np.concatenate([[centre[1]], pts[:, 1]])
    z = np.concatenate([[centre[2]], pts[:, 2]])
    d = np.full(m + 1, 6.0, np.float32)
    params = dict(synth.MECH_DEFAULTS, precision="mixed", interaction_radius=R)
    sim = bdm.Sim(params)
    sim.add_agents(x, y, z, d)
    sim.step(1)
    got = sim.get_state()
    want = oracle.mech_step(x, y, z, d, params["dt"], params["repulsion"], params["attraction"],
                            params["max_displacement"], R)
    assert want["neighbour_count"][0] == m // 2
    assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
    assert np.array_equal(got["box_id"], want["box_id"])


def test_mixed_ten_step_deviation_from_fp64():
    """End to end, mixed vs FP64 oracle after 10 steps (stated, and bounded)."""
    params, inp = synth.large_mechanics(n=50_000, seed=13, with_grid=False)
    sim, ref = make_pair(params, inp)
    sim.step(10)
    ref.step(10)
    got, want = sim.get_state(), ref.get_state()
    dev = max(float(np.max(np.abs(got[a] - want[a]))) for a in ("x", "y", "z"))
    print("mixed vs FP64 after 10 steps: max |dx| = %.3g um" % dev)
    assert dev < 1e-3


def test_full_size_sampled():
    """10^8 agents, the benchmark's launch configuration: every agent's box id against the reported
    grid, and sampled agents' neighbour counts and displacements against the oracle run on
    sub-cubes that contain their whole neighbourhood."""
    params, inp = synth.large_mechanics(n=100_000_000, seed=2, with_grid=False)
    x, y, z, d = inp["x"], inp["y"], inp["z"], inp["diameter"]
    sim = bdm.Sim(params)
    sim.add_agents(x, y, z, d)
    sim.step(1)
    st = sim.get_state(fields=("x", "y", "z", "neighbour_count", "box_id"))
    # grid assignment of every agent
    Lq = st["grid_box_q"]
    dims = st["grid_dims"]
    box = np.zeros(len(x), np.int64)
    mult = 1
    for a, c in enumerate((x, y, z)):
        q = np.rint(c * 1048576.0).astype(np.int64)
        assert q.min() == st["grid_origin_q"][a]
        b = (q - q.min()) // Lq
        assert b.max() == dims[a] - 1
        box += b * mult
        mult *= int(dims[a])
        del q, b
    assert np.array_equal(box, st["box_id"].astype(np.int64))
    del box
    # sampled neighbourhoods
    g = synth.rng(99)
    R = float(d.max())
    side = inp["side"]
    checked = 0
    H = 60.0
    for _ in range(8):
        c = g.uniform(H + 10.0, side - H - 10.0, 3)
        outer = (np.abs(x - c[0]) < H) & (np.abs(y - c[1]) < H) & (np.abs(z - c[2]) < H)
        idx = np.nonzero(outer)[0]
        sub = oracle.mech_step(x[idx], y[idx], z[idx], d[idx], params["dt"], params["repulsion"],
                               params["attraction"], params["max_displacement"],
                               interaction_radius=R)
        inner = ((np.abs(x[idx] - c[0]) < H - 2 * R) & (np.abs(y[idx] - c[1]) < H - 2 * R) &
                 (np.abs(z[idx] - c[2]) < H - 2 * R))
        ii = idx[inner]
        assert np.array_equal(st["neighbour_count"][ii], sub["neighbour_count"][inner])
        for a, c0 in (("x", x), ("y", y), ("z", z)):
            np.testing.assert_allclose(st[a][ii] - c0[ii], sub[a][inner] - c0[ii], atol=2e-5)
        checked += len(ii)
    assert checked > 1000


def test_growth_division_matches_oracle():
    """Tumour-spheroid growth: division ids and volumes exact every step; teacher-forced steps
    reproduce grid assignment, neighbour counts and new agents exactly."""
    params, inp = synth.spheroid()
    params = dict(params, capacity=1 << 17, diffusion_enabled=0)
    sim, ref = make_pair(params, inp)
    for k in range(30):
        sim.step(1)
        ref.step(1)
        got, want = sim.get_state(), ref.get_state()
        assert got["n"] == want["n"], k
        np.testing.assert_array_equal(got["volume"], want["volume"])
        np.testing.assert_allclose(got["diameter"], want["diameter"], rtol=2e-7)
    assert got["n"] > 4 * 512
    # teacher-forced: start both from the oracle's state
    for k in (30, 31, 32):
        s = ref.get_state()
        t = bdm.Sim(params)
        t.add_agents(s["x"], s["y"], s["z"], s["diameter"], s["volume"])
        t.set_step(k)
        ref.step(1)
        t.step(1)
        got, want = t.get_state(), ref.get_state()
        assert got["n"] == want["n"]
        np.testing.assert_array_equal(got["volume"], want["volume"])
        assert np.array_equal(got["box_id"], want["box_id"])
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
        dev = max(float(np.max(np.abs(got[a] - want[a]))) for a in ("x", "y", "z"))
        assert dev < 1e-4, dev
        t.close()


def test_growth_with_secretion_and_diffusion_mass():
    params, inp = synth.spheroid()
    params = dict(params, capacity=1 << 16)
    sim, ref = make_pair(params, inp)
    for _ in range(12):
        sim.step(1)
        ref.step(1)
    got, want = sim.get_state(), ref.get_state()
    assert got["n"] == want["n"]
    assert abs(got["mass_total"] - want["mass_total"]) <= 1e-6 * want["mass_total"]
    g = got["grid"].reshape(want["grid"].shape)
    assert np.max(np.abs(g - want["grid"])) <= 1e-4 * max(1.0, np.max(want["grid"]))


def test_resume_is_bit_exact():
    """10 steps == 5 steps + read-out + new handle + 5 steps (Philox keyed by step)."""
    params, inp = synth.spheroid(seed=3)
    params = dict(params, capacity=1 << 15, diffusion_enabled=0)
    a = bdm.Sim(params)
    a.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    a.step(10)
    full = a.get_state()
    b = bdm.Sim(params)
    b.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    b.step(5)
    half = b.get_state()
    c = bdm.Sim(params)
    c.add_agents(half["x"], half["y"], half["z"], half["diameter"], half["volume"])
    c.set_step(half["step"])
    c.step(5)
    res = c.get_state()
    for f in ("x", "y", "z", "diameter", "volume", "neighbour_count", "box_id"):
        assert np.array_equal(full[f], res[f]), f


def test_invalid_agents_are_rejected_and_handle_stays_usable():
    params = dict(synth.MECH_DEFAULTS, precision="fp64", capacity=64)
    sim = bdm.Sim(params)
    bad = ragged(10, 50.0, 3)
    bad["diameter"][4] = 0.0
    with pytest.raises(bdm.BdmError) as e:
        sim.add_agents(bad["x"], bad["y"], bad["z"], bad["diameter"])
    assert e.value.code == bdm.BDM_EINVAL and "agent 4" in str(e.value)
    nan = ragged(10, 50.0, 4)
    nan["y"][7] = float("nan")
    with pytest.raises(bdm.BdmError):
        sim.add_agents(nan["x"], nan["y"], nan["z"], nan["diameter"])
    good = ragged(20, 50.0, 5)
    ref = oracle.OracleSim(params)
    for s in (sim, ref):
        s.add_agents(good["x"], good["y"], good["z"], good["diameter"])
    sim.step(2)
    ref.step(2)
    assert_step_equal(sim.get_state(), ref.get_state())


def test_mixed_radius_below_a_diameter_is_refused():
    """Mixed precision finds contacts among the pairs within R: an interaction radius below the
    largest diameter is reported (BDM_ESTATE) instead of silently dropping contacts."""
    params, inp = synth.plain_mechanics()
    sim = bdm.Sim(dict(params, precision="mixed", interaction_radius=9.0))
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(1)
    with pytest.raises(bdm.BdmError) as e:
        sim.get_state()
    assert e.value.code == bdm.BDM_ESTATE
    sim.close()
    ok = bdm.Sim(dict(params, precision="mixed", interaction_radius=12.0))
    ok.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    ok.step(1)
    assert ok.get_state(fields=())["n"] == len(inp["x"])
