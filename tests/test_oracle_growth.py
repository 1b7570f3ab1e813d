"""Pins of the oracle's growth and division behaviour (CPU only): exact volume bookkeeping, the
division rule, id assignment, and the geometry of the split.  The daughter offset distance and the
axis law are readings the paper does not fix; beyond these consistency checks they are unpinned."""
import math

import numpy as np

import oracle
from paper_2006_06775_gb300 import synth

VDIV = math.pi / 6.0 * 14.0 ** 3


def run_growth(steps, n=64, seed=61):
    params, inp = synth.spheroid(seed=seed)
    x, y, z, d = inp["x"][:n], inp["y"][:n], inp["z"][:n], inp["diameter"][:n]
    dd = d.astype(np.float64)
    v = (0.5235987755982988 * dd) * dd * dd
    hist = []
    for k in range(steps):
        r = oracle.grow_divide(x, y, z, d, v, 100.0, VDIV, 0.25, seed, 0, k)
        hist.append((x, y, z, d, v, r))
        x, y, z, d, v = r["x"], r["y"], r["z"], r["diameter"], r["volume"]
    return hist


def test_volume_bookkeeping_and_division_rule():
    for (x, y, z, d, v, r) in run_growth(25):
        n = len(x)
        grown = v + 100.0
        divides = grown >= VDIV
        m = n + int(divides.sum())
        assert len(r["x"]) == m
        # total volume grows by exactly n * dv (division halves without loss)
        assert abs(r["volume"].sum() - grown.sum()) <= 1e-9 * grown.sum()
        np.testing.assert_array_equal(r["volume"][:n][~divides], grown[~divides])
        np.testing.assert_array_equal(r["volume"][:n][divides], grown[divides] * 0.5)
        # daughter of the k-th divider (ascending id) is agent n + k
        np.testing.assert_array_equal(r["volume"][n:], grown[divides] * 0.5)
        assert np.all(r["volume"] < VDIV)


def test_split_geometry():
    hist = run_growth(25)
    seen = 0
    for (x, y, z, d, v, r) in hist:
        n = len(x)
        divides = np.nonzero(v + 100.0 >= VDIV)[0]
        for k, i in enumerate(divides):
            j = n + k
            mid = np.array([(r["x"][i] + r["x"][j]) / 2, (r["y"][i] + r["y"][j]) / 2,
                            (r["z"][i] + r["z"][j]) / 2])
            np.testing.assert_allclose(mid, [x[i], y[i], z[i]], atol=1e-12)
            sep = math.dist((r["x"][i], r["y"][i], r["z"][i]), (r["x"][j], r["y"][j], r["z"][j]))
            assert abs(sep - 2 * 0.25 * float(r["diameter"][j])) < 1e-12
            seen += 1
    assert seen >= 64


def test_diameter_follows_volume():
    for (_x, _y, _z, _d, _v, r) in run_growth(12):
        dd = r["diameter"].astype(np.float64)
        np.testing.assert_allclose(math.pi / 6 * dd ** 3, r["volume"], rtol=1e-6)


def test_division_axis_isotropic():
    n = 4000
    x = np.zeros(n); d = np.full(n, 14.0, np.float32)
    v = np.full(n, VDIV)
    r = oracle.grow_divide(x, x, x, d, v, 0.0, VDIV, 0.25, 9, 0, 3)
    u = np.stack([r["x"][n:] - r["x"][:n], r["y"][n:] - r["y"][:n], r["z"][n:] - r["z"][:n]], 1)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    assert np.all(np.abs(u.mean(axis=0)) < 4 / math.sqrt(3 * n))
    np.testing.assert_allclose((u ** 2).mean(axis=0), 1 / 3, atol=0.03)
