"""GPU parity of the FTCS diffusion stencil and its FP64 mass total against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu

# FP32 stencil vs FP64 oracle: each step adds ~1 ulp (6e-8 relative) per voxel.
FIELD_REL = 1e-5
MASS_REL = 1e-6


def diffusion_params(n, voxel=10.0, D=0.4, decay=0.01):
    return dict(kind="mechanics", precision="mixed", dt=0.01, repulsion=2.0, attraction=1.0,
                max_displacement=3.0, diffusion_enabled=1, grid_n=n, grid_origin=(0.0, 0.0, 0.0),
                voxel=voxel, diffusion_coeff=D, decay=decay, dt_diffusion=1.0, secretion=0.0,
                capacity=1, box_capacity=16)


@pytest.mark.parametrize("shape", [(128, 128, 128), (37, 21, 50), (1, 1, 1), (33, 9, 17)])
def test_ftcs_matches_oracle(shape):
    nx, ny, nz = shape
    u0 = synth.rng(71).uniform(0.0, 2.0, (nz, ny, nx)).astype(np.float32)
    params = diffusion_params(shape)
    sim = bdm.Sim(params)
    sim.set_grid(u0)
    sim.diffusion_step(20)
    got = sim.get_state(fields=("grid",))
    u = u0.astype(np.float64)
    lam, mu_dt = oracle.ftcs_coefficients(0.4, 1.0, 10.0, 0.01)
    for _ in range(20):
        u, mass = oracle.ftcs(u, lam, mu_dt)
    g = got["grid"].reshape(nz, ny, nx)
    assert np.max(np.abs(g - u) / np.maximum(np.abs(u), 1e-3)) < FIELD_REL
    assert abs(got["mass_total"] - mass) <= MASS_REL * mass


def test_mass_conserved_without_decay():
    u0 = synth.rng(72).uniform(0.0, 2.0, (64, 64, 64)).astype(np.float32)
    sim = bdm.Sim(diffusion_params((64, 64, 64), decay=0.0))
    sim.set_grid(u0)
    m0 = float(u0.astype(np.float64).sum())
    sim.diffusion_step(50)
    st = sim.get_state(fields=("grid",))
    assert abs(st["mass_total"] - m0) <= 2e-6 * m0
    assert abs(st["mass_total"] - st["grid"].astype(np.float64).sum()) <= 1e-9 * m0


def test_full_size_512_sampled_blocks():
    """512^3 grid of the large workload: mass recurrence and sampled 40^3 blocks against the oracle
    run on the block plus a halo as wide as the number of steps."""
    n = 512
    params, inp = synth.large_mechanics(n=1000, seed=2, grid_side=synth.large_side(10 ** 8))
    params = dict(params, capacity=1000, box_capacity=1 << 12)
    u0 = inp["grid"]
    sim = bdm.Sim(params)
    sim.set_grid(u0)
    steps = 3
    sim.diffusion_step(steps)
    st = sim.get_state(fields=("grid",))
    g = st["grid"].reshape(n, n, n)
    lam, mu_dt = oracle.ftcs_coefficients(params["diffusion_coeff"], params["dt_diffusion"],
                                          params["voxel"], params["decay"])
    m = float(u0.astype(np.float64).sum())
    for _ in range(steps):
        m *= (1.0 - mu_dt)
    assert abs(st["mass_total"] - m) <= 1e-6 * m
    rng = synth.rng(73)
    for corner in ([0, 0, 0], [n - 40, n - 40, n - 40], list(rng.integers(10, n - 50, 3))):
        lo = [max(c - steps, 0) for c in corner]
        hi = [min(c + 40 + steps, n) for c in corner]
        block = u0[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].astype(np.float64)
        for _ in range(steps):
            block, _m = oracle.ftcs(block, lam, mu_dt)
        # interior of the block (walls of the block that are not grid walls are `steps` away)
        sl = tuple(slice(c - l, c - l + 40) for c, l in zip(corner, lo))
        want = block[sl]
        have = g[corner[0]:corner[0] + 40, corner[1]:corner[1] + 40, corner[2]:corner[2] + 40]
        assert np.max(np.abs(have - want) / np.abs(want)) < FIELD_REL
