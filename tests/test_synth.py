"""The synthetic neuron forest follows the pyramidal cell the paper prints (Sec. "Neuroscience use
case", tests/golden/pyramidal_cell.json): one apical and three basal dendrites on a 10 um soma,
branching with probability 0.038 (apical) and 0.006 (basal) per generation, apical dendrites growing
twice as fast (twice as long elements), and by default the large run's 5000 cells and 9e6 agents."""
import inspect
import json
import math
import os

import numpy as np

from paper_2006_06775_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pyramidal_cell.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_forest_defaults_are_the_large_run():
    g = golden()["large_run"]
    sig = inspect.signature(synth.neuron_forest).parameters
    assert sig["n_neurons"].default == g["initial_cells"]
    assert sig["n_agents"].default == g["agents"]


def test_forest_cells_branching_and_speed_follow_the_printed_cell():
    g = golden()
    params, f = synth.neuron_forest(400, 200_000, side=800.0, seed=12)
    m = f["mother"].astype(np.int64)
    soma = m < 0
    n_soma = int(soma.sum())
    assert n_soma == 400
    assert np.all(f["diameter"][soma] == g["initial_cell"]["soma_diameter_um"])
    roots = np.flatnonzero(~soma & (m >= 0) & soma[np.maximum(m, 0)])
    per_soma = np.bincount(m[roots], minlength=n_soma)
    cell = g["initial_cell"]
    assert np.all(per_soma == cell["apical_dendrites"] + cell["basal_dendrites"])
    # kinds from the element length class: apical rest lengths are twice the basal ones
    el = ~soma
    apical = el & (f["rest"] >= 3.0)
    basal = el & (f["rest"] < 3.0)
    ratio = f["rest"][apical].mean() / f["rest"][basal].mean()
    assert abs(ratio - g["apical_speed_over_basal"]) < 0.02
    assert int((apical[roots]).sum()) == n_soma * cell["apical_dendrites"]
    # branching: an element with daughters has two of them with the printed probability
    kids = np.bincount(m[el], minlength=len(m))
    for mask, p in ((apical, g["branching_probability_per_step"]["apical"]),
                    (basal, g["branching_probability_per_step"]["basal"])):
        parents = mask & (kids > 0)
        k = int(parents.sum())
        rate = float((kids[parents] == 2).sum()) / k
        assert abs(rate - p) < 5.0 * math.sqrt(p * (1.0 - p) / k) + 2.0 / k, (rate, p, k)
