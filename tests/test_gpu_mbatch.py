"""Batched mechanics (bdm_mbatch_*): a pool of simulation slots advanced together, every step one
launch sequence covering all active slots.  Each slot must compute exactly what a single handle
computes for the same simulation (grid rebuilt every step): positions, neighbour counts and box ids
bit for bit, on the FP64 path and on the mixed path (the same FP32 operations in the same order),
including simulations admitted while others run and slots reused after release."""
import numpy as np
import pytest

from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "neighbour_count", "box_id")


def sims(precision, count, seed0=100):
    """Served-mechanics simulations of different sizes and constants."""
    g = np.random.default_rng(seed0)
    out = []
    for k in range(count):
        n = int(g.choice([64, 500, 1200, 3000, 7000]))
        params, inp = synth.served_mechanics(n, seed0 + k)
        params = dict(params, precision=precision, dt=float(g.uniform(0.005, 0.02)),
                      repulsion=float(g.uniform(1.0, 3.0)), attraction=float(g.uniform(0.5, 1.5)),
                      max_displacement=float(g.choice([0.05, 3.0])))
        out.append((params, inp, int(g.integers(1, 9))))
    return out


def single(params, inp, steps):
    sim = bdm.Sim(dict(params, skin=0.0))
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(steps)
    st = sim.get_state(fields=FIELDS)
    sim.close()
    return st


def check_equal(got, want, tag):
    for f in FIELDS:
        assert np.array_equal(got[f], want[f]), (tag, f)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pool_slots_equal_single_handles(precision):
    cases = sims(precision, 7)
    pool = bdm.MechBatch(precision, slots=8, slot_capacity=8192)
    for s, (params, inp, steps) in enumerate(cases):
        pool.load_sim(s, params, inp["x"], inp["y"], inp["z"], inp["diameter"], steps)
    for _ in range(10):
        pool.step(1)
    done = pool.poll()
    assert list(done[:7]) == [c[2] for c in cases] and done[7] == -1
    for s, (params, inp, steps) in enumerate(cases):
        got = pool.get_state(s)
        assert got["step"] == steps
        check_equal(got, single(params, inp, steps), s)
    pool.close()


def test_pool_admits_while_running_and_reuses_slots():
    """Slots loaded after others have stepped, finished slots released and reused, steps in
    chunks: every simulation still equals its single handle."""
    cases = sims("mixed", 6, seed0=200)
    targets = [steps + 4 if k < 3 else steps for k, (_, _, steps) in enumerate(cases)]
    pool = bdm.MechBatch("mixed", slots=3, slot_capacity=8192)
    owner = {}
    for s in range(3):
        params, inp, _ = cases[s]
        pool.load_sim(s, params, inp["x"], inp["y"], inp["z"], inp["diameter"], targets[s])
        owner[s] = s
    pool.step(3)
    nxt, results = 3, {}
    for _ in range(40):
        done = pool.poll()
        for s in range(3):
            case = owner.get(s)
            if case is None or done[s] != targets[case]:
                continue
            results[case] = pool.get_state(s)
            pool.release(s)
            del owner[s]
            if nxt < len(cases):
                params, inp, _ = cases[nxt]
                pool.load_sim(s, params, inp["x"], inp["y"], inp["z"], inp["diameter"], targets[nxt])
                owner[s] = nxt
                nxt += 1
        if len(results) == len(cases):
            break
        pool.step(2)
    assert len(results) == len(cases)
    for case, (params, inp, _) in enumerate(cases):
        assert results[case]["step"] == targets[case]
        check_equal(results[case], single(params, inp, targets[case]), case)
    pool.close()


def test_pool_rejects_bad_loads():
    pool = bdm.MechBatch("mixed", slots=2, slot_capacity=1000)
    params, inp = synth.served_mechanics(500, 3)
    pool.load_sim(0, params, inp["x"], inp["y"], inp["z"], inp["diameter"], 2)
    with pytest.raises(bdm.BdmError):  # occupied
        pool.load_sim(0, params, inp["x"], inp["y"], inp["z"], inp["diameter"], 2)
    with pytest.raises(bdm.BdmError):  # a neighbour-list skin is not a plain simulation
        pool.load_sim(1, dict(params, skin=2.0), inp["x"], inp["y"], inp["z"], inp["diameter"], 2)
    with pytest.raises(bdm.BdmError):  # another precision than the pool's
        pool.load_sim(1, dict(params, precision="fp64"), inp["x"], inp["y"], inp["z"],
                      inp["diameter"], 2)
    big = synth.served_mechanics(1001, 4)[1]
    with pytest.raises(bdm.BdmError):  # beyond the slot capacity
        pool.load_sim(1, params, big["x"], big["y"], big["z"], big["diameter"], 2)
    bad = dict(inp, diameter=np.where(np.arange(500) == 7, -1.0, inp["diameter"]).astype(np.float32))
    with pytest.raises(bdm.BdmError):  # a negative diameter
        pool.load_sim(1, params, bad["x"], bad["y"], bad["z"], bad["diameter"], 2)
    # the pool still works after the refused loads
    pool.load_sim(1, params, inp["x"], inp["y"], inp["z"], inp["diameter"], 1)
    pool.step(2)
    check_equal(pool.get_state(1), single(params, inp, 1), 1)
    check_equal(pool.get_state(0), single(params, inp, 2), 0)
    pool.close()


def test_pool_edge_sizes_and_idle_steps():
    """A one-agent simulation and one at exactly the slot capacity; steps with no active slot are
    no-ops; a slot keeps its state after reaching its target while others still step."""
    pool = bdm.MechBatch("mixed", slots=3, slot_capacity=2000)
    pool.step(3)  # nothing loaded: nothing happens
    assert list(pool.poll()) == [-1, -1, -1]
    params, inp = synth.served_mechanics(2000, 11)
    one = {k: v[:1].copy() for k, v in inp.items() if hasattr(v, "__len__")}
    pool.load_sim(0, params, one["x"], one["y"], one["z"], one["diameter"], 4)
    pool.load_sim(2, params, inp["x"], inp["y"], inp["z"], inp["diameter"], 9)
    pool.step(6)
    assert list(pool.poll()) == [4, -1, 6]
    check_equal(pool.get_state(0), single(params, one, 4), "one agent")
    pool.step(5)
    assert list(pool.poll()) == [4, -1, 9]
    check_equal(pool.get_state(2), single(params, inp, 9), "full slot")
    check_equal(pool.get_state(0), single(params, one, 4), "one agent, after others stepped")
    pool.release(0)
    pool.release(2)
    pool.step(2)
    assert list(pool.poll()) == [-1, -1, -1]
    pool.close()
