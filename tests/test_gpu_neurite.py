"""GPU parity of neurite mechanics (readings R16-R20) through the C ABI of include/bdm_neurite.h.

Every step is checked against the FP64 oracle from the GPU's own state (teacher forcing): the
neighbour counts and the radius L exactly, positions within 1e-9 um on the FP64 path and 1e-5 um on
the mixed path (FP32 contact geometry from box-relative offsets; an FP32 force of magnitude F carries
about 1e-6 F of error, moved by dt = 0.01).  At the benchmark's full size (5000 neurons, 9e6
agents) sampled agents are checked against the oracle one by one."""
import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-5}
# The neighbour-list path bins on boxes of L + skin, so its FP32 box-relative contact geometry rounds
# differently.  Contacts of nearly parallel elements are ill-conditioned (reading R18: the contact
# point moves by about eps / sin^2 theta for an input error eps); on the 9001-agent forest the same
# three elements deviate by up to 1.2e-5 um (3-D) on the per-step-rebuild path and by up to 1.7e-5
# um with skins of 0.5-2 um.  The list path is held to twice the mixed limit.
TOL_SKIN = 2e-5
NEURITE_BENCH_SKIN = 1.0  # the neighbour-list skin (um) of bench.py's neuron forest


def oracle_step(params, inp):
    return oracle.neurite_step(inp["x"], inp["y"], inp["z"], inp["diameter"], inp["rest"],
                               inp["mother"], inp["ox"], inp["oy"], inp["oz"], params["dt"],
                               params["repulsion"], params["attraction"],
                               params["max_displacement"], params["spring"],
                               params.get("interaction_radius", 0.0))


def make(params, precision, capacity=None, **kw):
    p = dict(params, precision=precision, capacity=capacity or (1 << 16), **kw)
    return bdm.Neurite(p)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("seed,neurons,agents,side", [(1, 16, 2500, 60.0), (2, 40, 9001, 70.0),
                                                      (3, 3, 700, 25.0)])
def test_forest_teacher_forced(precision, seed, neurons, agents, side):
    params, inp = synth.neuron_forest(neurons, agents, side=side, seed=seed)
    sim = make(params, precision)
    sim.set_agents(inp)
    cur = dict(inp)
    contacts_seen = 0.0
    for k in range(4):
        sim.step(1)
        got = sim.get_state()
        want = oracle_step(params, cur)
        assert got["n"] == agents
        assert got["L"] == want["L"], k
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"]), k
        for a in "xyz":
            err = np.max(np.abs(got[a] - want[a]))
            assert err < TOL[precision], (k, a, err)
        contacts_seen = max(contacts_seen, float(np.abs(want["force"]).max()))
        cur = dict(cur, x=got["x"], y=got["y"], z=got["z"])
    assert contacts_seen > 0.0
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_many_steps_stay_close_to_the_oracle(precision):
    """20 free-running steps on both sides (no teacher forcing)."""
    params, inp = synth.neuron_forest(10, 1500, side=40.0, seed=7)
    sim = make(params, precision)
    sim.set_agents(inp)
    sim.step(20)
    got = sim.get_state()
    cur = dict(inp)
    for _ in range(20):
        r = oracle_step(params, cur)
        cur = dict(cur, x=r["x"], y=r["y"], z=r["z"])
    for a in "xyz":
        assert np.max(np.abs(got[a] - cur[a])) < 20 * TOL[precision]
    assert np.array_equal(got["neighbour_count"], r["neighbour_count"])
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_somata_only_and_single_agents(precision):
    params, _ = synth.neuron_forest(1, 1, seed=0)
    x, y, z, d = synth.uniform_spheres(3000, 100.0, seed=8)
    n = len(x)
    inp = dict(x=x, y=y, z=z, diameter=d.astype(np.float64), rest=np.zeros(n),
               mother=-np.ones(n, np.int32), ox=np.zeros(n), oy=np.zeros(n), oz=np.zeros(n))
    sim = make(params, precision)
    sim.set_agents(inp)
    sim.step(1)
    got = sim.get_state()
    want = oracle_step(params, inp)
    assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
    for a in "xyz":
        assert np.max(np.abs(got[a] - want[a])) < TOL[precision]
    # one soma and one element: only the spring acts
    one = {k: v[:1].copy() for k, v in inp.items()}
    two = {k: np.concatenate([one[k], np.asarray([v], one[k].dtype)]) for k, v in
           dict(x=x[0] + 7.5, y=y[0], z=z[0], diameter=1.0, rest=2.0, mother=0, ox=5.0, oy=0.0,
                oz=0.0).items()}
    for case in (one, two):
        sim.set_agents(case)
        sim.step(1)
        got = sim.get_state()
        want = oracle_step(params, case)
        for a in "xyz":
            assert np.max(np.abs(got[a] - want[a])) < TOL[precision]
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
    # no agents: steps are a no-op
    sim.set_agents({k: v[:0] for k, v in inp.items()})
    sim.step(3)
    assert sim.get_state()["n"] == 0
    sim.close()


def test_errors_are_reported_without_a_fault():
    params, inp = synth.neuron_forest(8, 800, side=40.0, seed=9)
    sim = make(params, "mixed", box_capacity=8)
    sim.set_agents(inp)
    sim.step(1)
    with pytest.raises(bdm.BdmError) as e:
        sim.get_state()
    assert e.value.code == bdm.BDM_ENOMEM
    sim.close()
    sim = make(params, "mixed", capacity=100)
    with pytest.raises(bdm.BdmError) as e:
        sim.set_agents(inp)
    assert e.value.code == bdm.BDM_ENOMEM
    sim.close()
    sim = make(params, "fp64")
    bad = dict(inp, mother=inp["mother"].copy())
    bad["mother"][20] = 25
    with pytest.raises(bdm.BdmError) as e:
        sim.set_agents(bad)
    assert e.value.code == bdm.BDM_EINVAL and "agent 20" in str(e.value)
    sim.close()


@pytest.mark.parametrize("skin", [0.0, NEURITE_BENCH_SKIN])
def test_full_size_forest_sampled_against_the_oracle(skin):
    """The benchmark workload (5000 neurons, 9e6 agents, mixed precision, the bench's launch
    configuration, with and without the bench's neighbour-list skin): 48 sampled agents against
    the oracle one by one, exact neighbour counts; and the total displacement of all agents is zero
    up to rounding when no cap is hit (every force comes in equal and opposite pairs, and the split
    and the springs only move force around).  With the skin, a few list steps run first and the
    checked step is a list step."""
    params, inp = synth.neuron_forest()
    n = len(inp["x"])
    sim = make(params, "mixed", capacity=n, skin=skin)
    sim.set_agents(inp)
    if skin > 0.0:
        # step until a step evaluates the lists (no rebuild), and check that step
        for _ in range(16):
            start = sim.get_state()
            rebuilds = sim.list_info()[0]
            sim.step(1)
            if sim.list_info()[0] == rebuilds:
                break
        assert sim.list_info()[0] == rebuilds, "no list step in 16 steps"
        inp = dict(inp, **{a: start[a] for a in "xyz"})
    else:
        sim.step(1)
    got = sim.get_state()
    g = synth.rng(77)
    idx = np.unique(np.concatenate([g.integers(0, n, 40), g.integers(0, 5000, 8)]))
    want = oracle.neurite_sample(inp["x"], inp["y"], inp["z"], inp["diameter"], inp["rest"],
                                 inp["mother"], inp["ox"], inp["oy"], inp["oz"], params["dt"],
                                 params["repulsion"], params["attraction"],
                                 params["max_displacement"], params["spring"], idx)
    assert got["L"] == want["L"]
    assert np.array_equal(got["neighbour_count"][idx], want["neighbour_count"])
    for a in "xyz":
        assert np.max(np.abs(got[a][idx] - want[a])) < TOL["mixed"]
    d = np.stack([got[a] - inp[a] for a in "xyz"], 1)
    assert np.abs(d).max() < params["max_displacement"]
    assert np.abs(d.sum(0)).max() < 1e-6 * np.abs(d).sum()
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("change", [{"interaction_radius": 14.0}, {"max_displacement": 0.002},
                                    {"spring": 0.0, "attraction": 0.0}])
def test_radius_cap_and_law_variants(precision, change):
    """A fixed radius above the largest extent (L = 14 um: more neighbours, same contacts), a cap
    that most moving agents hit, and pure repulsion without springs."""
    params, inp = synth.neuron_forest(12, 2000, side=45.0, seed=11)
    params = dict(params, **change)
    sim = make(params, precision)
    sim.set_agents(inp)
    cur = dict(inp)
    for k in range(3):
        sim.step(1)
        got = sim.get_state()
        want = oracle_step(params, cur)
        assert got["L"] == want["L"], k
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"]), k
        for a in "xyz":
            assert np.max(np.abs(got[a] - want[a])) < TOL[precision], (k, a)
        prev = cur
        cur = dict(cur, x=got["x"], y=got["y"], z=got["z"])
    if "interaction_radius" in change:
        assert got["L"] == 14.0
    if "max_displacement" in change:
        # the last oracle step started from `prev`; every displacement respects the cap, and many
        # agents sit on it
        moved = np.sqrt(sum((want[a] - prev[a]) ** 2 for a in "xyz"))
        assert np.all(moved <= 0.002 * (1 + 1e-9))
        assert np.mean(moved > 0.002 * (1 - 1e-6)) > 0.05
    sim.close()


def _rows(rows):
    a = np.array(rows, dtype=np.float64)
    inp = {k: np.ascontiguousarray(a[:, i]) for i, k in
           enumerate(("x", "y", "z", "diameter", "rest", "mother", "ox", "oy", "oz"))}
    inp["mother"] = inp["mother"].astype(np.int32)
    return inp


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_degenerate_geometry_one_step(precision):
    """Coincident somata (counted, no force), a zero-length element (a point on its mother's distal
    end), and two exactly parallel elements of different trees 0.8 um apart (closest points not
    unique: both sides take the proximal end, s = 0)."""
    params, _ = synth.neuron_forest(1, 1, seed=0)
    inp = _rows([(0, 0, 0, 10, 0, -1, 0, 0, 0),          # soma A
                 (0, 0, 0, 8, 0, -1, 0, 0, 0),           # soma B, coincident with A
                 (30, 0, 0, 10, 0, -1, 0, 0, 0),         # soma C
                 (39, 0, 0, 1.0, 4.0, 2, 5, 0, 0),       # element E1 on C: (35,0,0)-(39,0,0)
                 (39, 0, 0, 1.0, 1.0, 3, 0, 0, 0),       # element E2 on E1: zero length at (39,0,0)
                 (30, 0.8, 0, 10, 0, -1, 0, 0, 0),       # soma D overlapping C
                 (39, 0.8, 0, 1.0, 4.0, 5, 5, 0, 0)])    # element F1 on D, parallel to E1
    want = oracle_step(params, inp)
    assert want["neighbour_count"][0] >= 1 and np.abs(want["force"]).max() > 0.0
    sim = make(params, precision)
    sim.set_agents(inp)
    sim.step(1)
    got = sim.get_state()
    assert got["L"] == want["L"]
    assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
    for a in "xyz":
        assert np.max(np.abs(got[a] - want[a])) < TOL[precision], a
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parallel_elements_tie_rule_one_step(precision):
    """Two exactly parallel elements of different trees, 0.8 um apart and overlapping along half
    their length: E1 spans x in [35, 39], F1 x in [37, 41].  Their closest pair is not unique;
    reading R18 takes the first edge minimiser that attains the distance: for E1 against F1 the
    s = 1 edge (E1's distal end, F1 at t = 0.5), for F1 against E1 the s = 0 edge.  E1 therefore
    keeps the whole contact force at its distal point and F1 passes all of it to its soma."""
    params, _ = synth.neuron_forest(1, 1, seed=0)
    inp = _rows([(30, 0, 0, 10, 0, -1, 0, 0, 0),         # soma C
                 (39, 0, 0, 1.0, 4.0, 0, 5, 0, 0),       # element E1 on C: (35,0,0)-(39,0,0)
                 (32, 0.8, 0, 10, 0, -1, 0, 0, 0),       # soma D
                 (41, 0.8, 0, 1.0, 4.0, 2, 5, 0, 0)])    # element F1 on D: (37,0.8,0)-(41,0.8,0)
    s, t = oracle.segment_closest([35, 0, 0], [4, 0, 0], [37, 0.8, 0], [4, 0, 0])
    assert (s, t) == (1.0, 0.5)
    want = oracle_step(params, inp)
    assert np.abs(want["force"][3]).max() == 0.0  # F1 passed its whole share on (s = 0)
    assert np.abs(want["force"][1]).max() > 0.0
    sim = make(params, precision)
    sim.set_agents(inp)
    sim.step(1)
    got = sim.get_state()
    assert got["L"] == want["L"]
    assert np.array_equal(got["neighbour_count"], want["neighbour_count"])
    for a in "xyz":
        assert np.max(np.abs(got[a] - want[a])) < TOL[precision], a
    sim.close()


@pytest.mark.parametrize("skin", [0.5, 2.0])
@pytest.mark.parametrize("seed,neurons,agents,side", [(1, 16, 2500, 60.0), (2, 40, 9001, 70.0)])
def test_forest_with_skin_teacher_forced(skin, seed, neurons, agents, side):
    """Neighbour lists (mixed precision): every step, rebuild steps and list steps alike, matches
    the oracle's step from the GPU's own state -- counts and L exactly, positions within TOL_SKIN --
    and the lists do carry steps between rebuilds."""
    params, inp = synth.neuron_forest(neurons, agents, side=side, seed=seed)
    sim = make(params, "mixed", skin=skin)
    sim.set_agents(inp)
    cur = dict(inp)
    steps = 12
    for k in range(steps):
        sim.step(1)
        got = sim.get_state()
        want = oracle_step(params, cur)
        assert got["L"] == want["L"], k
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"]), k
        for a in "xyz":
            err = np.max(np.abs(got[a] - want[a]))
            assert err < TOL_SKIN, (k, a, err)
        cur = dict(cur, x=got["x"], y=got["y"], z=got["z"])
    rebuilds, entries = sim.list_info()
    assert 1 <= rebuilds < steps
    assert entries > 0
    sim.close()


def test_skin_list_overflow_falls_back_to_the_sweep():
    """600 somata in a 30 um cube with a 4 um skin: somata with more than 128 agents within L + skin
    overflow their lists and sweep their 27 boxes instead, next to slots that use their lists; the
    results match the oracle."""
    params, _ = synth.neuron_forest(1, 1, seed=0)
    x, y, z, d = synth.uniform_spheres(600, 30.0, seed=12)
    n = len(x)
    inp = dict(x=x, y=y, z=z, diameter=d.astype(np.float64), rest=np.zeros(n),
               mother=-np.ones(n, np.int32), ox=np.zeros(n), oy=np.zeros(n), oz=np.zeros(n))
    sim = make(params, "mixed", skin=4.0)
    sim.set_agents(inp)
    cur = dict(inp)
    for k in range(3):
        sim.step(1)
        got = sim.get_state()
        want = oracle_step(params, cur)
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"]), k
        assert int(want["neighbour_count"].max()) > 128
        for a in "xyz":
            assert np.max(np.abs(got[a] - want[a])) < TOL_SKIN, (k, a)
        cur = dict(cur, x=got["x"], y=got["y"], z=got["z"])
    sim.close()


@pytest.mark.parametrize("bad", [dict(skin=-1.0), dict(skin=float("nan")),
                                 dict(skin=1.0, precision="fp64")])
def test_skin_parameter_checks(bad):
    params, _ = synth.neuron_forest(1, 1, seed=0)
    p = dict(params, precision="mixed", capacity=64)
    p.update(bad)
    with pytest.raises(bdm.BdmError) as e:
        bdm.Neurite(p)
    assert e.value.code == bdm.BDM_EINVAL
