"""Autotuner: choice logic and cache on CPU; on the GPU, every tuned knob leaves the integer results
unchanged (neighbour counts, SIR states) and the positions within FP32 summation tolerance."""
import numpy as np
import pytest

from paper_2006_06775_gb300 import synth, tune


def test_choose_picks_fastest_and_keeps_table():
    cands = [dict(box_factor=f, force_variant=v) for v in (0, 1) for f in (1.0, 1.3)]
    cost = {(1.0, 0): 3.0, (1.3, 0): 2.5, (1.0, 1): 4.0, (1.3, 1): 2.7}
    best, table = tune.choose(cands, lambda c: cost[(c["box_factor"], c["force_variant"])])
    assert (best["box_factor"], best["force_variant"]) == (1.3, 0)
    assert len(table) == 4 and all("ms_per_step" in r for r in table)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tuned.json")
    c = tune.TuneCache(path)
    params, inp = synth.large_mechanics(n=5000, seed=1, with_grid=False)
    calls = []

    def measure(cand):
        calls.append(cand)
        return 1.0 + cand["box_factor"] + cand["force_variant"]
    ch = tune.tune_mechanics(params, inp, inp["side"] ** 3, cache=c, measure=measure)
    assert ch["box_factor"] == 1.0 and ch["force_variant"] == 0
    assert len(calls) == len(tune.MECH_CANDIDATES)
    again = tune.tune_mechanics(params, inp, inp["side"] ** 3, cache=tune.TuneCache(path),
                                measure=lambda c: 1 / 0)
    assert again["box_factor"] == ch["box_factor"] and again["signature"] == ch["signature"]


def test_signature_buckets():
    p = dict(kind="mechanics", precision="mixed")
    a = tune.workload_signature(p, 10 ** 6, 10 ** 9)
    b = tune.workload_signature(p, int(1.1e6), 1.05e9)
    c = tune.workload_signature(p, 10 ** 6, 10 ** 10)
    assert a == b and a != c


def test_sir_box_candidates_are_valid():
    params = synth.sir_ensemble(runs=1)[0][0]
    L, r = 1024000, 6144
    cands = tune.sir_box_candidates(params, 20000)
    assert cands and all(L % nb == 0 and L // nb >= r for nb in cands)


@pytest.mark.gpu
def test_tuned_mechanics_knobs_keep_results():
    from paper_2006_06775_gb300 import bdm
    params, inp = synth.large_mechanics(n=300_000, seed=21, with_grid=False)
    choice = tune.tune_mechanics(params, inp, inp["side"] ** 3)
    assert len(choice["table"]) == len(tune.MECH_CANDIDATES)
    base = bdm.Sim(params)
    base.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    base.step(1)
    want = base.get_state()
    for cand in tune.MECH_CANDIDATES:
        sim = bdm.Sim(tune.mechanics_params(params, inp, cand))
        sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
        sim.step(1)
        got = sim.get_state()
        assert np.array_equal(got["neighbour_count"], want["neighbour_count"]), cand
        for a in ("x", "y", "z"):
            assert np.max(np.abs(got[a] - want[a])) < 2e-5, cand
        sim.close()


@pytest.mark.gpu
def test_force_variants_agree_over_ten_steps():
    from paper_2006_06775_gb300 import bdm
    for make in (lambda: synth.large_mechanics(n=100_000, seed=22, with_grid=False),
                 lambda: synth.served_mechanics(50_000, 23)):
        params, inp = make()
        states = []
        for v in (0, 1):
            sim = bdm.Sim(dict(params, force_variant=v))
            sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
            sim.step(10)
            states.append(sim.get_state())
            sim.close()
        a, b = states
        assert np.array_equal(a["box_id"], b["box_id"])
        assert np.array_equal(a["neighbour_count"], b["neighbour_count"])
        for k in ("x", "y", "z"):
            assert np.max(np.abs(a[k] - b[k])) < 1e-5


@pytest.mark.gpu
def test_tuned_sir_boxes_keep_states():
    from paper_2006_06775_gb300 import bdm
    ens = synth.sir_ensemble(runs=32)
    params = [p for p, _ in ens]
    inputs = [inp for _, inp in ens]
    choice = tune.tune_sir_batch(params, inputs)
    assert choice["sir_boxes"] in tune.sir_box_candidates(params[0], 20000)
    runs = {}
    for nb in (choice["sir_boxes"], 0):
        b = bdm.Batch([dict(p, sir_boxes=nb) for p in params])
        for k, inp in enumerate(inputs):
            b.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
        b.step(30)
        runs[nb] = [b.get_state(k) for k in (0, 13, 31)]
        b.close()
    for s1, s2 in zip(runs[choice["sir_boxes"]], runs[0]):
        for f in ("x", "y", "z", "sir_state", "neighbour_count"):
            assert np.array_equal(s1[f], s2[f]), f
