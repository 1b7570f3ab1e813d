"""Pins of the oracle's SIR model (CPU only): infected-neighbour counts against an all-pairs
minimum-image brute force, the invariants of the model, its special cases, the move distribution,
and the expected infections of the well-mixed model against the analytic SIR curves of the paper's
measles and influenza parameters (Sec. "Epidemiology use case")."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import synth


def brute_infected_counts(X, Y, Z, st, L, r):
    def mi(d):
        d = d.copy()
        d[d > L // 2] -= L
        d[d < -(L // 2)] += L
        return d
    X, Y, Z = (np.asarray(a, np.int64) for a in (X, Y, Z))
    dx = mi(X[:, None] - X[None, :])
    dy = mi(Y[:, None] - Y[None, :])
    dz = mi(Z[:, None] - Z[None, :])
    hit = (dx * dx + dy * dy + dz * dz) < r * r
    np.fill_diagonal(hit, False)
    hit &= (st[None, :] == 1)
    return hit.sum(axis=1).astype(np.uint32)


def population(n, L, seed, frac=0.2):
    g = synth.rng(seed, 3)
    X, Y, Z = (g.integers(0, L, n).astype(np.int32) for _ in range(3))
    st = (g.uniform(0, 1, n) < frac).astype(np.uint8)
    return X, Y, Z, st


@pytest.mark.parametrize("L,nb,r", [(600, 1, 50), (600, 2, 50), (600, 3, 100), (600, 6, 100),
                                    (600, 12, 50), (1000, 10, 100)])
def test_infected_counts_equal_brute_force(L, nb, r):
    X, Y, Z, st = population(400, L, L + nb)
    res = oracle.sir_step(X, Y, Z, st, L, nb, r, 7, 0.3, 0.1, 3, 0, 0)
    assert np.array_equal(res["infected_neighbours"], brute_infected_counts(X, Y, Z, st, L, r))


def test_invariants_and_counts():
    L, n = 2048, 3000
    X, Y, Z, st = population(n, L, 41, frac=0.05)
    prevS, prevR = (st == 0).sum(), (st == 2).sum()
    for step in range(40):
        res = oracle.sir_step(X, Y, Z, st, L, 16, 64, 40, 0.4, 0.05, 3, 1, step)
        X, Y, Z, st = res["X"], res["Y"], res["Z"], res["state"]
        S, I, R = res["counts"]
        assert S + I + R == n
        assert [S, I, R] == [(st == 0).sum(), (st == 1).sum(), (st == 2).sum()]
        assert S <= prevS and R >= prevR
        assert X.min() >= 0 and X.max() < L
        prevS, prevR = S, R


def test_no_infection_when_probability_zero():
    X, Y, Z, st = population(800, 512, 42, frac=0.3)
    S0 = (st == 0).sum()
    for step in range(10):
        res = oracle.sir_step(X, Y, Z, st, 512, 8, 60, 20, 0.0, 0.1, 3, 2, step)
        X, Y, Z, st = res["X"], res["Y"], res["Z"], res["state"]
        assert (st == 0).sum() == S0


def test_recovery_probability_one_lasts_one_step():
    X, Y, Z, st = population(800, 512, 43, frac=0.3)
    for step in range(10):
        res = oracle.sir_step(X, Y, Z, st, 512, 8, 60, 20, 0.5, 1.0, 3, 2, step)
        assert np.all(res["state"][st == 1] == 2)         # every infected recovers next step
        newly = (st == 0) & (res["state"] == 1)
        assert np.all(res["state"][newly] == 1)             # newly infected stay infected this step
        X, Y, Z, st = res["X"], res["Y"], res["Z"], res["state"]


def test_move_is_uniform_on_minus_s_to_s():
    L, s, n = 1 << 20, 3, 20000
    X = np.full(n, L // 2, np.int32)
    st = np.zeros(n, np.uint8)
    res = oracle.sir_step(X, X, X, st, L, 1, 1, s, 0.0, 0.0, 5, 0, 9)
    for a in ("X", "Y", "Z"):
        m = res[a].astype(np.int64) - L // 2
        assert m.min() == -s and m.max() == s
        hist = np.bincount(m + s, minlength=2 * s + 1)
        chi2 = ((hist - n / 7) ** 2 / (n / 7)).sum()
        assert chi2 < 30  # 6 dof


def test_infection_probability_matches_threshold():
    # every susceptible sits next to one infected agent: infections ~ Binomial(S, p)
    n, L, p = 20000, 1 << 20, 0.3
    g = synth.rng(44)
    X = (g.integers(0, 64, n // 2) * 16000).astype(np.int32)
    Y = (g.integers(0, 64, n // 2) * 16000).astype(np.int32)
    Z = np.arange(n // 2, dtype=np.int32) * 100
    Xs, Ys, Zs = np.concatenate([X, X]), np.concatenate([Y, Y]), np.concatenate([Z, Z + 1])
    st = np.concatenate([np.ones(n // 2, np.uint8), np.zeros(n // 2, np.uint8)])
    res = oracle.sir_step(Xs, Ys, Zs, st, L, 1, 2, 0, p, 0.0, 6, 0, 0)
    assert np.all(res["infected_neighbours"][n // 2:] >= 1)
    k = (res["state"][n // 2:] == 1).sum()
    mu, sd = p * n / 2, math.sqrt(n / 2 * p * (1 - p))
    assert abs(k - mu) < 4 * sd


def lattice_ball_fraction(L, r):
    """Fraction of the periodic lattice within minimum-image squared distance < r^2 (j != i)."""
    d = np.arange(L) - 0
    d = np.where(d > L // 2, d - L, d)
    d2 = d * d
    cnt = (d2[:, None, None] + d2[None, :, None] + d2[None, None, :] < r * r).sum() - 1
    return cnt / (L ** 3 - 1)


def well_mixed_runs(N, L, nb, r, p, q, I0, steps, runs, seed):
    """Step size (L-1)/2 with L odd makes each move uniform over the whole lattice, so positions
    are re-drawn every step: the well-mixed setting of the analytic SIR model."""
    s = (L - 1) // 2
    hist = []
    for run in range(runs):
        g = synth.rng(seed, run)
        X, Y, Z = (g.integers(0, L, N).astype(np.int32) for _ in range(3))
        st = np.zeros(N, np.uint8)
        st[:I0] = 1
        traj = [((st == 0).sum(), (st == 1).sum(), (st == 2).sum())]
        for k in range(steps):
            res = oracle.sir_step(X, Y, Z, st, L, nb, r, s, p, q, seed, run, k)
            X, Y, Z, st = res["X"], res["Y"], res["Z"], res["state"]
            traj.append(tuple(int(c) for c in res["counts"]))
        hist.append(traj)
    return np.array(hist, dtype=np.float64)  # (runs, steps+1, 3)


def _diseases():
    """(R0, T_R) of the paper's two diseases, from tests/golden/sir_diseases.json."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sir_diseases.json")
    with open(path) as f:
        d = json.load(f)["diseases"]
    return [(d[k]["R0"], d[k]["T_R_days"]) for k in ("measles", "influenza")]


DISEASES = _diseases()


@pytest.mark.parametrize("R0,TR", DISEASES)
def test_well_mixed_expected_infections_unbiased(R0, TR):
    """Given (S, I) at step start, the expected number of new infections in the well-mixed model is
    S p (1 - (1 - v)^I) exactly, with v the lattice-ball fraction.  Per run, the summed surprises
    are a martingale: their mean over independent runs must be 0 within 3.5 standard errors."""
    N, L, nb, r = 2000, 243, 9, 14
    v = lattice_ball_fraction(L, r)
    q = 1.0 / TR
    p = min(1.0, R0 * q / (N * v))
    h = well_mixed_runs(N, L, nb, r, p, q, 20, 60, 12, 51)
    S, I = h[:, :-1, 0], h[:, :-1, 1]
    newinf = S - h[:, 1:, 0]
    expected = S * p * (1 - (1 - v) ** I)
    D = (newinf - expected).sum(axis=1)
    se = D.std(ddof=1) / math.sqrt(len(D))
    assert abs(D.mean()) < 3.5 * se + 1.0
    recov = h[:, 1:, 2] - h[:, :-1, 2]
    Dr = (recov - q * I).sum(axis=1)
    assert abs(Dr.mean()) < 3.5 * Dr.std(ddof=1) / math.sqrt(len(Dr)) + 1.0


@pytest.mark.parametrize("R0,TR", DISEASES)
def test_well_mixed_mean_follows_sir_curves(R0, TR):
    """Ensemble mean of the agent model (10 runs, as in the paper's Fig. 4) against (a) the discrete
    mean-field recurrence of the same model and (b) the Kermack-McKendrick ODE with R0 = beta/gamma,
    gamma = 1/T_R (paper: measles R0 12.9, T_R 8 d; influenza R0 1.3, T_R 4.1 d), one step per day.
    The one-day step lags the continuous ODE in time, so (b) compares final size and peak height
    (measles: ODE peak N (1 - (1 + ln R0) / R0) = 1449 of 2000)."""
    N, L, nb, r, I0 = 2000, 243, 9, 14, 20
    v = lattice_ball_fraction(L, r)
    gamma = 1.0 / TR
    beta = R0 * gamma
    p = min(1.0, beta / (N * v))
    steps = 80 if R0 > 5 else 120
    h = well_mixed_runs(N, L, nb, r, p, gamma, I0, steps, 10, 52)
    mean = h.mean(axis=0)
    # (a) discrete mean-field recurrence
    S, I, R = N - I0, float(I0), 0.0
    mf = [(S, I, R)]
    for _ in range(steps):
        new = S * p * (1 - (1 - v) ** I)
        S, I, R = S - new, I + new - gamma * I, R + gamma * I
        mf.append((S, I, R))
    mf = np.array(mf)
    assert np.max(np.abs(mean[:, 1] - mf[:, 1])) < 0.06 * N
    assert abs(mean[-1, 0] - mf[-1, 0]) < 0.04 * N
    # (b) Kermack-McKendrick ODE, RK4 with 200 sub-steps per day
    def f(y):
        S, I, R = y
        return np.array([-beta * S * I / N, beta * S * I / N - gamma * I, gamma * I])
    y = np.array([N - float(I0), float(I0), 0.0])
    ode = [y.copy()]
    hh = 1.0 / 200
    for _ in range(steps):
        for _ in range(200):
            k1 = f(y); k2 = f(y + hh / 2 * k1); k3 = f(y + hh / 2 * k2); k4 = f(y + hh * k3)
            y = y + hh / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        ode.append(y.copy())
    ode = np.array(ode)
    # runs peak at different times, so compare the per-run peak and final size, within 3 SE + 3%
    peaks, final_s = h[:, :, 1].max(axis=1), h[:, -1, 0]
    se = lambda a: a.std(ddof=1) / math.sqrt(len(a))
    assert abs(peaks.mean() - ode[:, 1].max()) < 3 * se(peaks) + 0.03 * ode[:, 1].max()
    assert abs(final_s.mean() - ode[-1, 0]) < 3 * se(final_s) + 0.03 * N
