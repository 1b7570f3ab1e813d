"""Batched SIR ensemble (one persistent launch per step for all runs): every run is bit-identical
to the same run on its own handle and to the oracle; per-step S/I/R history; a grid-barrier wait
that runs out is reported as BDM_ETIMEOUT without faulting the GPU."""
import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "sir_state", "neighbour_count", "box_id")


def uneven_runs():
    """Runs of different sizes, domains, box counts and probabilities."""
    out = []
    specs = [(5000, 400.0, 16, 0.05), (1, 50.0, 2, 0.05), (3000, 150.0, 3, 0.05),
             (20000, 1000.0, 0, 0.05), (700, 100.0, 1, 0.05), (12000, 600.0, 0, 0.05),
             (2500, 90.0, 6, 0.6)]
    g = synth.rng(7, 7)
    for k, (n, dom, nb, frac) in enumerate(specs):
        p = dict(kind="sir", seed=3, run_id=k, sir_domain=dom, sir_radius=6.0, sir_step=5.0,
                 sir_boxes=nb, p_infect=float(g.uniform(0.1, 0.4)),
                 p_recover=float(g.uniform(0.01, 0.03)))
        x, y, z, st = synth.sir_run(n, 3, k, dom, infected_frac=frac)
        if n == 1:
            st[:] = 1
        out.append((p, dict(x=x, y=y, z=z, sir_state=st)))
    return out


@pytest.mark.parametrize("persistent_only", [False, True])
def test_batch_matches_single_handles_and_history(persistent_only):
    runs = uneven_runs()
    steps = 25
    batch = bdm.Batch([p for p, _ in runs], history_steps=64, persistent_only=persistent_only)
    for k, (_, inp) in enumerate(runs):
        batch.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
    batch.step(10)
    batch.step(15)
    hist = batch.counts(steps)
    assert hist.shape == (steps, len(runs), 3)
    for k, (p, inp) in enumerate(runs):
        single = bdm.Sim(p)
        single.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        for s in range(steps):
            single.step(1)
            st = single.get_state(fields=())
            assert np.array_equal(hist[s, k], st["sir_counts"]), (k, s)
        want = single.get_state()
        got = batch.get_state(k)
        assert got["step"] == steps
        for f in FIELDS:
            assert np.array_equal(got[f], want[f]), (k, f)
        assert np.array_equal(got["sir_counts"], want["sir_counts"])
        single.close()


@pytest.mark.parametrize("persistent_only", [False, True])
def test_batch_matches_oracle(persistent_only):
    all_runs = uneven_runs()
    runs = [all_runs[k] for k in (0, 1, 2, 6)]  # sparse, single agent, 3 boxes, dense infection
    batch = bdm.Batch([p for p, _ in runs], persistent_only=persistent_only)
    refs = []
    for k, (p, inp) in enumerate(runs):
        batch.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
        r = oracle.OracleSim(p)
        r.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        refs.append(r)
    batch.step(12)
    for k, r in enumerate(refs):
        r.step(12)
        want, got = r.get_state(), batch.get_state(k)
        for f in ("x", "y", "z", "sir_state", "neighbour_count", "box_id", "sir_counts"):
            assert np.array_equal(got[f], want[f]), (k, f)


def test_barrier_wait_that_runs_out_is_reported():
    runs = uneven_runs()[:2]
    batch = bdm.Batch([p for p, _ in runs], spin_limit=2000, barrier_extra=1)
    for k, (_, inp) in enumerate(runs):
        batch.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
    batch.step(1)
    with pytest.raises(bdm.BdmError) as e:
        batch.sync()
    assert e.value.code == bdm.BDM_ETIMEOUT
    batch.close()
    # the context stays usable: a normal batch afterwards runs and is correct
    ok = bdm.Batch([p for p, _ in runs])
    for k, (_, inp) in enumerate(runs):
        ok.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
    ok.step(3)
    ref = oracle.OracleSim(runs[0][0])
    ref.add_agents(runs[0][1]["x"], runs[0][1]["y"], runs[0][1]["z"], sir_state=runs[0][1]["sir_state"])
    ref.step(3)
    assert np.array_equal(ok.get_state(0)["sir_state"], ref.get_state()["sir_state"])


@pytest.mark.parametrize("boxes", [32, 40])
def test_full_ensemble_sampled_runs(boxes):
    """256 runs x 20,000 persons, the ensemble workload: sampled runs equal their single-run
    handles after 200 steps, and every step's counts sum to the run size (32 boxes per axis: one CTA
    per run in shared memory; 40: the persistent grid)."""
    ens = [(dict(p, sir_boxes=boxes), inp) for p, inp in synth.sir_ensemble()]
    batch = bdm.Batch([p for p, _ in ens], history_steps=200)
    for k, (_, inp) in enumerate(ens):
        batch.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
    batch.step(200)
    hist = batch.counts(200)
    assert np.all(hist.sum(axis=2) == 20000)
    assert np.all(np.diff(hist[:, :, 0].astype(np.int64), axis=0) <= 0)  # S never grows
    for k in (0, 77, 255):
        p, inp = ens[k]
        single = bdm.Sim(p)
        single.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        single.step(200)
        want, got = single.get_state(), batch.get_state(k)
        for f in FIELDS:
            assert np.array_equal(got[f], want[f]), (k, f)
        single.close()


@pytest.mark.parametrize("persistent_only", [False, True])
def test_batch_with_an_empty_run(persistent_only):
    """A run without agents sits between two others: it reports zero counts, and its neighbours
    still match the oracle."""
    all_runs = uneven_runs()
    runs = [all_runs[0], (dict(all_runs[2][0], run_id=50), None), all_runs[2]]
    batch = bdm.Batch([p for p, _ in runs], history_steps=8, persistent_only=persistent_only)
    for k, (_, inp) in enumerate(runs):
        if inp is not None:
            batch.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
    batch.step(6)
    empty = batch.get_state(1)
    assert empty["n"] == 0 and np.array_equal(empty["sir_counts"], [0, 0, 0])
    for k in (0, 2):
        p, inp = runs[k]
        ref = oracle.OracleSim(p)
        ref.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        ref.step(6)
        want, got = ref.get_state(), batch.get_state(k)
        for f in ("x", "y", "z", "sir_state", "neighbour_count", "box_id", "sir_counts"):
            assert np.array_equal(got[f], want[f]), (k, f)
    batch.close()
