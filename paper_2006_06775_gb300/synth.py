"""Seeded synthetic workloads shaped like the paper's use cases.

This module only draws random inputs and holds the parameter recipes of the workloads; it contains
none of the simulation's arithmetic.  Both the CUDA path and the FP64 oracle are fed from here.

Workloads (BioDynaMo, arXiv 2006.06775; Sec. "Performance" names the cell growth and division
benchmark, Sec. "Oncology use case" the tumour spheroid, Sec. "Epidemiology use case" the SIR model):

  plain_mechanics     4096 spheres, centres U[0,160)^3 um, diameters U[8,12] um, seed 0, FP64,
                      repulsion 2.0, attraction 1.0, dt 0.01, displacement cap 3 um, 10 steps.
  spheroid            512 cells on an 8^3 lattice (spacing 12 um, centred on the origin,
                      jitter U[-0.5,0.5] um per axis), diameter 10 um, seed 1; growth 100 um^3 per
                      step, division at diameter 14 um; secretion 1.0 per cell per step into a 128^3
                      FP32 grid (voxel 10 um, origin -640 um, D 0.4, decay 0.01, dt 1, closed walls).
  large_mechanics     10^8 spheres at 0.3 volume fraction (cube side 5662 um), diameters U[8,12],
                      seed 2; a 512^3 FP32 grid spanning the cube co-stepped (D 0.4, decay 0.01, dt 1)
                      from a seeded smooth random field.
  sir_ensemble        256 runs x 20,000 persons in a 1000 um periodic cube, 2% infected, step 5 um,
                      infection radius 6 um, p_inf ~ U[0.1,0.4], p_rec ~ U[0.01,0.03] per run, seed 3.
  served_stream       Poisson arrivals (200/s), log-uniform sizes 1e3..1e6 agents, 50..500 steps,
                      70% mechanics / 30% SIR, seed 4.
  settled_mechanics   a settled lattice (spacing 14 um, no contacts) around a central ball of
                      overlapping agents at 0.3 volume fraction (10% of the agents), seed 5: the
                      workload on which skipping stationary agents is measured.
  neuron_forest       5000 somata (10 um) in a 2000 um cube with one apical and three basal
                      dendrite trees each (branching 0.038 / 0.006 per generation, apical elements
                      twice as long), 9e6 agents, seed 6: the large pyramidal-cell run's size.
"""
import math
from dataclasses import dataclass

import numpy as np


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Counter-based Philox bit generator keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=(int(stream) << 32) | int(seed)))


# ------------------------------------------------------------------------------------------------
# Mechanics populations
# ------------------------------------------------------------------------------------------------
MECH_DEFAULTS = dict(kind="mechanics", dt=0.01, repulsion=2.0, attraction=1.0,
                     max_displacement=3.0, interaction_radius=0.0, box_length=0.0)

VOLUME_FRACTION_LARGE = 0.3
MEAN_SPHERE_VOLUME_8_12 = math.pi / 6.0 * (12.0 ** 4 - 8.0 ** 4) / (4.0 * 4.0)  # E[d^3] = 544.5*6/pi


def uniform_spheres(n: int, side: float, seed: int, stream: int = 0, dmin=8.0, dmax=12.0):
    """n centres uniform in [0, side)^3 and diameters uniform in [dmin, dmax] (float32)."""
    g = rng(seed, stream)
    x = g.uniform(0.0, side, n)
    y = g.uniform(0.0, side, n)
    z = g.uniform(0.0, side, n)
    d = g.uniform(dmin, dmax, n).astype(np.float32)
    return x, y, z, d


def plain_mechanics(n: int = 4096, side: float = 160.0, seed: int = 0):
    """Plain-mechanics population (default: 4096 agents in a 160 um cube)."""
    x, y, z, d = uniform_spheres(n, side, seed)
    params = dict(MECH_DEFAULTS, precision="fp64", seed=seed)
    return params, dict(x=x, y=y, z=z, diameter=d)


def large_side(n: int, volume_fraction: float = VOLUME_FRACTION_LARGE) -> float:
    """Cube side that puts n spheres (diameters U[8,12]) at the given volume fraction."""
    return (n * MEAN_SPHERE_VOLUME_8_12 / volume_fraction) ** (1.0 / 3.0)


def large_mechanics(n: int = 100_000_000, seed: int = 2, grid_n: int = 512, with_grid=True,
                    grid_side=None):
    """Large mechanics + diffusion population at 0.3 volume fraction (side 5662 um at 10^8).
    The substance grid spans grid_side (default: the population's cube)."""
    side = large_side(n)
    x, y, z, d = uniform_spheres(n, side, seed)
    params = dict(MECH_DEFAULTS, precision="mixed", seed=seed)
    inputs = dict(x=x, y=y, z=z, diameter=d, side=side)
    if with_grid and grid_n:
        gs = side if grid_side is None else grid_side
        params.update(diffusion_enabled=1, grid_n=(grid_n, grid_n, grid_n),
                      grid_origin=(0.0, 0.0, 0.0), voxel=gs / grid_n, diffusion_coeff=0.4,
                      decay=0.01, dt_diffusion=1.0, secretion=0.0)
        inputs["grid"] = smooth_field(grid_n, seed)
    return params, inputs


def settled_mechanics(n: int = 10_000_000, active_frac: float = 0.1, seed: int = 5,
                      spacing: float = 14.0, jitter: float = 0.5):
    """A settled tissue with one active region: agents on a jittered cubic lattice (spacing 14 um,
    so no two are closer than 13 um, beyond the largest diameter: no contacts, no forces), and a
    central ball holding `active_frac` of the agents as a random packing at 0.3 volume fraction,
    which relaxes outward into the lattice.  Diameters U[8,12] um; mixed precision."""
    g = rng(seed)
    n_act = int(round(n * active_frac))
    n_lat = n - n_act
    rb = (3.0 * n_act * MEAN_SPHERE_VOLUME_8_12 / VOLUME_FRACTION_LARGE / (4.0 * math.pi)) ** (1.0 / 3.0)
    # active ball: radius ~ U^(1/3), direction uniform
    r = rb * g.uniform(0.0, 1.0, n_act) ** (1.0 / 3.0)
    v = g.normal(size=(n_act, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    act = v * r[:, None]
    # lattice points outside the ball (one spacing of margin), nearest to the centre first
    m = int(math.ceil(((n_lat + 4.0 / 3.0 * math.pi * (rb + 2 * spacing) ** 3 / spacing ** 3) * 1.05)
                      ** (1.0 / 3.0))) + 2
    idx = np.arange(m, dtype=np.float64) - (m - 1) / 2.0
    zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    lat = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1) * spacing
    dist = np.linalg.norm(lat, axis=1)
    keep = np.nonzero(dist > rb + spacing)[0]
    keep = keep[np.argsort(dist[keep], kind="stable")[:n_lat]]
    lat = lat[keep] + g.uniform(-jitter, jitter, (n_lat, 3))
    P = np.concatenate([act, lat])
    d = g.uniform(8.0, 12.0, n).astype(np.float32)
    params = dict(MECH_DEFAULTS, precision="mixed", seed=seed)
    return params, dict(x=P[:, 0].copy(), y=P[:, 1].copy(), z=P[:, 2].copy(), diameter=d,
                        n_active=n_act, ball_radius=rb)


def smooth_field(n: int, seed: int, modes: int = 6) -> np.ndarray:
    """Seeded smooth positive random field of shape (n, n, n), float32: a sum of a few low-frequency
    separable cosines around 1.0."""
    g = rng(seed, 7)
    t = (np.arange(n, dtype=np.float64) + 0.5) / n
    field = np.ones((n, n, n), np.float32)
    for _ in range(modes):
        kx, ky, kz = g.integers(1, 5, 3)
        px, py, pz = g.uniform(0, 2 * math.pi, 3)
        a = g.uniform(0.05, 0.15)
        fx = np.cos(2 * math.pi * kx * t + px).astype(np.float32)
        fy = np.cos(2 * math.pi * ky * t + py).astype(np.float32)
        fz = np.cos(2 * math.pi * kz * t + pz).astype(np.float32)
        field += np.float32(a) * fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    return field


def spheroid(seed: int = 1, lattice: int = 8, spacing: float = 12.0, diameter: float = 10.0,
             grid_n: int = 128):
    """Tumour-spheroid start: lattice^3 cells centred on the origin with +-0.5 um jitter."""
    g = rng(seed)
    idx = np.arange(lattice, dtype=np.float64) - (lattice - 1) / 2.0
    zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    n = lattice ** 3
    x = xx.reshape(-1) * spacing + g.uniform(-0.5, 0.5, n)
    y = yy.reshape(-1) * spacing + g.uniform(-0.5, 0.5, n)
    z = zz.reshape(-1) * spacing + g.uniform(-0.5, 0.5, n)
    d = np.full(n, diameter, np.float32)
    division_diameter = 14.0
    params = dict(MECH_DEFAULTS, precision="mixed", seed=seed, growth_enabled=1,
                  growth_volume=100.0,
                  division_volume=math.pi / 6.0 * division_diameter ** 3,
                  division_offset_frac=0.25, interaction_radius=division_diameter,
                  diffusion_enabled=1, grid_n=(grid_n, grid_n, grid_n),
                  grid_origin=(-640.0, -640.0, -640.0), voxel=10.0, diffusion_coeff=0.4,
                  decay=0.01, dt_diffusion=1.0, secretion=1.0)
    return params, dict(x=x, y=y, z=z, diameter=d)


# ------------------------------------------------------------------------------------------------
# SIR ensemble
# ------------------------------------------------------------------------------------------------
SIR_UNIT = 1.0 / 1024.0  # positions are drawn on the 2^-10 um lattice the SIR model runs on


def sir_run(n: int, seed: int, run: int, domain: float = 1000.0, infected_frac: float = 0.02):
    """One SIR population: lattice-exact uniform positions, the first floor(f n) agents of a seeded
    permutation infected.  Returns positions in um and the state vector (0 S, 1 I, 2 R)."""
    g = rng(seed, 1000 + run)
    units = int(round(domain / SIR_UNIT))
    X = g.integers(0, units, n)
    Y = g.integers(0, units, n)
    Z = g.integers(0, units, n)
    state = np.zeros(n, np.uint8)
    state[g.permutation(n)[: int(math.floor(infected_frac * n))]] = 1
    return X * SIR_UNIT, Y * SIR_UNIT, Z * SIR_UNIT, state


def sir_ensemble(runs: int = 256, n: int = 20_000, seed: int = 3, domain: float = 1000.0,
                 boxes: int = 40):
    """Per-run parameters and populations of the batched SIR ensemble."""
    g = rng(seed, 999)
    p_inf = g.uniform(0.1, 0.4, runs)
    p_rec = g.uniform(0.01, 0.03, runs)
    out = []
    for r in range(runs):
        params = dict(kind="sir", seed=seed, run_id=r, sir_domain=domain, sir_radius=6.0,
                      sir_step=5.0, sir_boxes=boxes, p_infect=float(p_inf[r]),
                      p_recover=float(p_rec[r]))
        x, y, z, st = sir_run(n, seed, r, domain)
        out.append((params, dict(x=x, y=y, z=z, sir_state=st)))
    return out


# ------------------------------------------------------------------------------------------------
# Served request stream
# ------------------------------------------------------------------------------------------------
@dataclass
class Request:
    rid: int
    arrival: float   # seconds after stream start
    kind: str        # "mechanics" | "sir"
    n: int
    steps: int
    seed: int


def request_stream(count: int = 2000, rate: float = 200.0, seed: int = 4, nmin=1e3, nmax=1e6,
                   smin=50, smax=500, mech_frac=0.7):
    """Poisson arrivals with log-uniform sizes and uniform step counts."""
    g = rng(seed, 5)
    gaps = g.exponential(1.0 / rate, count)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(g.uniform(math.log(nmin), math.log(nmax), count)).astype(np.int64)
    steps = g.integers(smin, smax + 1, count)
    kinds = np.where(g.uniform(0, 1, count) < mech_frac, "mechanics", "sir")
    return [Request(i, float(t[i]), str(kinds[i]), int(sizes[i]), int(steps[i]), seed * 100000 + i)
            for i in range(count)]


def served_mechanics(n: int, seed: int, density: float = 4096 / 160.0 ** 3):
    """A served mechanics request: plain-mechanics density, cube side scaled with n^(1/3)."""
    side = (n / density) ** (1.0 / 3.0)
    x, y, z, d = uniform_spheres(n, side, seed)
    params = dict(MECH_DEFAULTS, precision="mixed", seed=seed)
    return params, dict(x=x, y=y, z=z, diameter=d)


def served_sir(n: int, seed: int, density: float = 20_000 / 1000.0 ** 3, boxes_per_side=None):
    """A served SIR request at the ensemble's density (domain scaled with n^(1/3), rounded to a whole
    number of um so the box count divides the lattice)."""
    domain = float(max(20, int(round((n / density) ** (1.0 / 3.0)))))
    g = rng(seed, 11)
    p_inf = float(g.uniform(0.1, 0.4))
    p_rec = float(g.uniform(0.01, 0.03))
    x, y, z, st = sir_run(n, seed, 0, domain)
    params = dict(kind="sir", seed=seed, run_id=0, sir_domain=domain, sir_radius=6.0, sir_step=5.0,
                  sir_boxes=boxes_per_side or 0, p_infect=p_inf, p_recover=p_rec)
    return params, dict(x=x, y=y, z=z, sir_state=st)


# ------------------------------------------------------------------------------------------------
# Neuron forest (Sec. "Neuroscience use case": pyramidal cells with one apical and three basal
# dendrites on a 10 um soma; branching probabilities 0.038 apical and 0.006 basal per step; apical
# dendrites grow twice as fast; the large run holds 5000 cells and 9 million agents)
# ------------------------------------------------------------------------------------------------
NEURITE_DEFAULTS = dict(kind="neurite", dt=0.01, repulsion=2.0, attraction=1.0,
                        max_displacement=3.0, spring=10.0, interaction_radius=0.0)


def _unit(v):
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def neuron_forest(n_neurons: int = 5000, n_agents: int = 9_000_000, side: float = 2000.0,
                  seed: int = 6, soma_diameter: float = 10.0, stretch: float = 0.1,
                  persistence: float = 0.35):
    """Somata uniform in [0, side)^3, each with one apical and three basal dendrites grown as random
    binary trees, one element per tip per generation, until the forest holds n_agents agents
    (somata first, then elements generation by generation, so every mother precedes its daughters).
    Element rest lengths: basal U[1.5, 2.5] um, apical U[3, 5] um; actual lengths are the rest length
    times U[1 - stretch, 1 + stretch]; diameters taper from 1.5 (apical) / 1.2 (basal) by 0.5% per
    generation down to 0.5 um.  A root element starts on the soma surface (offset r_soma * direction);
    every other element starts at its mother's distal point (offset 0).  Directions follow a
    persistent random walk; a branch point spawns two daughters deflected to either side."""
    if n_agents < n_neurons:
        raise ValueError("n_agents must cover the somata")
    g = rng(seed, 9)
    cx = g.uniform(0.0, side, n_neurons)
    cy = g.uniform(0.0, side, n_neurons)
    cz = g.uniform(0.0, side, n_neurons)
    cols = {k: [a] for k, a in (("x", cx), ("y", cy), ("z", cz))}
    cols["diameter"] = [np.full(n_neurons, soma_diameter)]
    cols["rest"] = [np.zeros(n_neurons)]
    cols["mother"] = [np.full(n_neurons, -1, np.int64)]
    for k in ("ox", "oy", "oz"):
        cols[k] = [np.zeros(n_neurons)]
    # tips: one apical (kind 1) and three basal (kind 0) per soma
    kind = np.tile(np.array([1, 0, 0, 0], np.int8), n_neurons)
    soma = np.repeat(np.arange(n_neurons), 4)
    d = g.normal(size=(4 * n_neurons, 3))
    d[kind == 1] = d[kind == 1] * 0.2 + np.array([0.0, 0.0, 1.0])
    d[kind == 0] = d[kind == 0] + np.array([0.0, 0.0, -0.5])
    d = _unit(d)
    r_s = 0.5 * soma_diameter
    mother = soma.astype(np.int64)
    base = np.stack([cx[soma], cy[soma], cz[soma]], 1)
    off = r_s * d
    prox = base + off
    diam = np.where(kind == 1, 1.5, 1.2)
    total = n_neurons
    while total < n_agents:
        take = min(len(mother), n_agents - total)
        mother, prox, off, d, diam, kind = (mother[:take], prox[:take], off[:take], d[:take],
                                            diam[:take], kind[:take])
        d = _unit(d + persistence * g.normal(size=d.shape))
        rest = np.where(kind == 1, g.uniform(3.0, 5.0, take), g.uniform(1.5, 2.5, take))
        length = rest * g.uniform(1.0 - stretch, 1.0 + stretch, take)
        dist = prox + d * length[:, None]
        idx = np.arange(total, total + take)
        for k, a in (("x", dist[:, 0]), ("y", dist[:, 1]), ("z", dist[:, 2]), ("diameter", diam),
                     ("rest", rest), ("mother", mother), ("ox", off[:, 0]), ("oy", off[:, 1]),
                     ("oz", off[:, 2])):
            cols[k].append(a)
        total += take
        # next generation: every element continues; a branch point adds a second daughter
        branch = g.uniform(size=take) < np.where(kind == 1, 0.038, 0.006)
        perp = _unit(np.cross(d, g.normal(size=d.shape)))
        d_next = np.where(branch[:, None], _unit(d + 0.6 * perp), d)
        d_extra = _unit(d[branch] - 0.6 * perp[branch])
        mother = np.concatenate([idx, idx[branch]])
        prox = np.concatenate([dist, dist[branch]])
        d = np.concatenate([d_next, d_extra])
        dn = np.maximum(diam * 0.995, 0.5)
        diam = np.concatenate([dn, dn[branch]])
        kind = np.concatenate([kind, kind[branch]])
        off = np.zeros_like(prox)
    inp = {k: np.concatenate(v) for k, v in cols.items()}
    inp["mother"] = inp["mother"].astype(np.int32)
    params = dict(NEURITE_DEFAULTS, seed=seed)
    return params, inp
