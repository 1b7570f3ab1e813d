"""The allocation-free diffusion step (bdm_diffusion_step_noalloc) against the regular handle path.

Callers that cannot allocate device memory (an application that owns all device memory through its
own pool, code running while another framework captures a CUDA graph, latency-critical loops that
cannot take cudaMalloc's implicit synchronisation) pass their own device buffers; the library keeps
its scratch in a fixed static device array.  This test plays such a caller: its buffers come from
PyTorch, and two calls in a row must match two steps of the handle's bdm_diffusion_step within the
diffusion tests' tolerances.  It lives in its own file so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2006_06775_gb300 import bdm, synth

pytestmark = pytest.mark.gpu

FIELD_REL = 1e-5  # as the other diffusion parity tests
MASS_REL = 1e-6


def _handle_steps(shape, u0, D, dt, h, decay, n):
    """n steps of the regular handle path (bdm_diffusion_step): fields and FP64 mass totals."""
    nx, ny, nz = shape
    params = dict(kind="mechanics", precision="mixed", dt=0.01, repulsion=2.0, attraction=1.0,
                  max_displacement=3.0, diffusion_enabled=1, grid_n=shape,
                  grid_origin=(0.0, 0.0, 0.0), voxel=h, diffusion_coeff=D, decay=decay,
                  dt_diffusion=dt, secretion=0.0, capacity=1, box_capacity=16)
    sim = bdm.Sim(params)
    sim.set_grid(u0)
    want = []
    for _ in range(n):
        sim.diffusion_step(1)
        st = sim.get_state(fields=("grid",))
        want.append((st["grid"].reshape(nz, ny, nx).copy(), st["mass_total"]))
    sim.close()
    return want


def test_noalloc_step_matches_handle_path_twice():
    import torch

    shape = (96, 40, 72)  # nx, ny, nz: several blocks in each direction with ragged edges
    nx, ny, nz = shape
    D, dt, h, decay = 0.4, 1.0, 10.0, 0.01
    u0 = synth.rng(91).uniform(0.0, 2.0, (nz, ny, nx)).astype(np.float32)

    want = _handle_steps(shape, u0, D, dt, h, decay, 2)

    stream = torch.cuda.Stream()
    a = torch.from_numpy(u0).to("cuda")
    b = torch.empty_like(a)
    mass = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    src, dst = a, b
    for k in range(2):
        rc = bdm.bdm_diffusion_step_noalloc(src.data_ptr(), dst.data_ptr(), shape, D, dt, h,
                                            decay, mass.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert rc == bdm.BDM_OK
        stream.synchronize()
        got = dst.cpu().numpy()
        ref, ref_mass = want[k]
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)) <= FIELD_REL
        assert abs(float(mass.item()) - ref_mass) <= MASS_REL * abs(ref_mass)
        src, dst = dst, src


def test_noalloc_rejects_grids_beyond_its_scratch():
    # 32 x 8 x 16-voxel blocks: 2048 x 2048 x 16 needs 64 * 256 * 1 = 16,384 blocks (accepted in
    # principle); 4096 x 4096 x 64 needs 128 * 512 * 4 = 262,144 > 65,536 and must be refused
    # before anything is launched (the pointers are never dereferenced).
    rc = bdm.bdm_diffusion_step_noalloc(1 << 20, 2 << 20, (4096, 4096, 64), 0.4, 1.0, 10.0, 0.01)
    assert rc == bdm.BDM_EINVAL
    rc = bdm.bdm_diffusion_step_noalloc(1 << 20, 1 << 20, (8, 8, 8), 0.4, 1.0, 10.0, 0.01)
    assert rc == bdm.BDM_EINVAL  # input and output must differ


@pytest.mark.parametrize("shape,offset,with_mass", [
    ((45, 21, 33), 0, True),    # x extent not a multiple of 4: the scalar FTCS kernel
    ((64, 24, 20), 1, False),   # grids one float past a 16-byte boundary: scalar kernel, no mass
])
def test_noalloc_scalar_kernel_and_no_mass(shape, offset, with_mass):
    """The scalar FTCS kernel through the allocation-free entry point (a ragged x extent, or buffers
    that are not 16-byte aligned), with and without the mass slot, two calls in a row against the
    handle path."""
    import torch

    nx, ny, nz = shape
    D, dt, h, decay = 0.4, 1.0, 10.0, 0.01
    u0 = synth.rng(92 + offset).uniform(0.0, 2.0, (nz, ny, nx)).astype(np.float32)
    want = _handle_steps(shape, u0, D, dt, h, decay, 2)
    nv = nx * ny * nz
    stream = torch.cuda.Stream()
    a_buf = torch.zeros(nv + offset, dtype=torch.float32, device="cuda")
    b_buf = torch.zeros(nv + offset, dtype=torch.float32, device="cuda")
    a, b = a_buf[offset:], b_buf[offset:]
    a.copy_(torch.from_numpy(u0.reshape(-1)).to("cuda"))
    mass = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    src, dst = a, b
    for k in range(2):
        rc = bdm.bdm_diffusion_step_noalloc(src.data_ptr(), dst.data_ptr(), shape, D, dt, h, decay,
                                            mass.data_ptr() if with_mass else None,
                                            ctypes.c_void_p(stream.cuda_stream))
        assert rc == bdm.BDM_OK
        stream.synchronize()
        got = dst.cpu().numpy().reshape(nz, ny, nx)
        ref, ref_mass = want[k]
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)) <= FIELD_REL
        if with_mass:
            assert abs(float(mass.item()) - ref_mass) <= MASS_REL * abs(ref_mass)
        else:
            assert float(mass.item()) == 0.0
        src, dst = dst, src
