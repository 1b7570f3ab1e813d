"""The C-ABI library builds, loads and exports every function the headers declare (CPU only: no
compute call is made; bdm_create is only asked to validate parameters)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2006_06775_gb300 import bdm
from paper_2006_06775_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(bdm_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return bdm.load(build_if_missing=False)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("bdm_create", "bdm_add_agents", "bdm_step", "bdm_diffusion_step",
                     "bdm_get_state", "bdm_destroy", "bdm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in libbuild.NVCC_FLAGS
    assert sum(f == "-gencode" for f in libbuild.NVCC_FLAGS) == 1


def test_struct_size_check_matches_c_layout(lib):
    p = bdm.make_params({"kind": "mechanics", "precision": "fp64", "dt": 0.01, "repulsion": 2.0,
                         "attraction": 1.0, "max_displacement": 3.0})
    h = ctypes.c_void_p()
    bad = bdm.Params.from_buffer_copy(p)
    bad.struct_size = ctypes.sizeof(bdm.Params) - 8
    rc = lib.bdm_create(ctypes.byref(bad), ctypes.byref(h))
    assert rc == bdm.BDM_EINVAL
    assert b"struct_size" in lib.bdm_last_error(h)
    lib.bdm_destroy(h)
    # with the binding's size the parameter check passes; without a GPU creation then fails with
    # BDM_ECUDA (or succeeds on a GPU machine)
    h = ctypes.c_void_p()
    rc = lib.bdm_create(ctypes.byref(p), ctypes.byref(h))
    assert rc in (bdm.BDM_OK, bdm.BDM_ECUDA), lib.bdm_last_error(h)
    lib.bdm_destroy(h)


@pytest.mark.parametrize("change,fragment", [
    ({"max_displacement": 0.0}, b"max_displacement"),
    ({"box_length": 5.0, "interaction_radius": 10.0}, b"box_length"),
    ({"diffusion_enabled": 1, "grid_n": (8, 8, 8), "voxel": 1.0, "diffusion_coeff": 1.0,
      "dt_diffusion": 1.0}, b"unstable"),
    ({"growth_enabled": 1, "division_volume": 10.0}, b"capacity"),
])
def test_invalid_parameters_are_rejected(lib, change, fragment):
    d = {"kind": "mechanics", "precision": "mixed", "dt": 0.01, "repulsion": 2.0,
         "attraction": 1.0, "max_displacement": 3.0}
    d.update(change)
    p = bdm.make_params(d)
    h = ctypes.c_void_p()
    rc = lib.bdm_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == bdm.BDM_EINVAL
    assert fragment in lib.bdm_last_error(h)
    lib.bdm_destroy(h)


def test_sir_parameters_are_checked(lib):
    p = bdm.make_params({"kind": "sir", "sir_domain": 100.0, "sir_radius": 6.0, "sir_step": 200.0,
                         "p_infect": 0.5, "p_recover": 0.1})
    h = ctypes.c_void_p()
    assert lib.bdm_create(ctypes.byref(p), ctypes.byref(h)) == bdm.BDM_EINVAL
    lib.bdm_destroy(h)
    p = bdm.make_params({"kind": "sir", "sir_domain": 100.0, "sir_radius": 6.0, "sir_step": 5.0,
                         "p_infect": 1.5, "p_recover": 0.1})
    h = ctypes.c_void_p()
    assert lib.bdm_create(ctypes.byref(p), ctypes.byref(h)) == bdm.BDM_EINVAL
    lib.bdm_destroy(h)


@pytest.mark.parametrize("change,fragment", [
    ({"precision": 7}, b"precision"),
    ({"dt": 0.0}, b"dt"),
    ({"max_displacement": -1.0}, b"max_displacement"),
    ({"capacity": 0}, b"capacity"),
    ({"capacity": (1 << 27) + 1}, b"2^27"),
    ({"interaction_radius": float("nan")}, b"interaction_radius"),
])
def test_neurite_parameters_are_rejected_before_any_cuda_call(lib, change, fragment):
    p = bdm.NeuriteParams()
    p.struct_size = ctypes.sizeof(bdm.NeuriteParams)
    p.precision = bdm.BDM_MIXED
    p.dt, p.repulsion, p.attraction, p.max_displacement, p.spring = 0.01, 2.0, 1.0, 3.0, 10.0
    p.capacity = 1000
    for k, v in change.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    rc = lib.bdm_neurite_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == bdm.BDM_EINVAL
    assert fragment in lib.bdm_neurite_last_error(h)
    lib.bdm_neurite_destroy(h)


def test_neurite_struct_size_check(lib):
    p = bdm.NeuriteParams()
    p.struct_size = ctypes.sizeof(bdm.NeuriteParams) - 8
    h = ctypes.c_void_p()
    assert lib.bdm_neurite_create(ctypes.byref(p), ctypes.byref(h)) == bdm.BDM_EINVAL
    assert not h.value
    # valid parameters pass validation; without a GPU creation then fails with BDM_ECUDA
    p.struct_size = ctypes.sizeof(bdm.NeuriteParams)
    p.precision, p.dt, p.max_displacement, p.capacity = bdm.BDM_FP64, 0.01, 3.0, 100
    rc = lib.bdm_neurite_create(ctypes.byref(p), ctypes.byref(h))
    assert rc in (bdm.BDM_OK, bdm.BDM_ECUDA), lib.bdm_neurite_last_error(h)
    lib.bdm_neurite_destroy(h)


def test_headers_compile_as_plain_c(tmp_path):
    """The boundary is plain C: every public header compiles as C99 (-pedantic, no warnings)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    heads = sorted(os.path.basename(h) for h in glob.glob(os.path.join(ROOT, "include", "*.h")))
    src = tmp_path / "headers.c"
    src.write_text("".join('#include "%s"\n' % h for h in heads) + "int main(void) { return 0; }\n")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I" + os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_noalloc_rejects_wrapping_and_unlaunchable_grids_on_cpu(lib):
    """The allocation-free diffusion step refuses, before any CUDA call, grids whose block count
    would wrap a 32-bit product (2^31 - 1 x 512 x 1 gives 2^26 * 64 = 2^32 blocks of 32 x 8 x 16)
    and grids beyond the launch limits (more than 65,535 blocks along y), so no pointer is touched."""
    for shape in ((2**31 - 1, 512, 1), (8, 8 * 65536, 16), (8, 8, 16 * 65536)):
        rc = bdm.bdm_diffusion_step_noalloc(1 << 20, 2 << 20, shape, 0.4, 1.0, 10.0, 0.01)
        assert rc == bdm.BDM_EINVAL, shape


def test_create_rejects_unlaunchable_diffusion_grid(lib):
    p = bdm.make_params({"kind": "mechanics", "precision": "mixed", "dt": 0.01, "repulsion": 2.0,
                         "attraction": 1.0, "max_displacement": 3.0, "diffusion_enabled": 1,
                         "grid_n": (8, 8 * 65536, 16), "voxel": 10.0, "diffusion_coeff": 0.4,
                         "dt_diffusion": 1.0, "decay": 0.01})
    h = ctypes.c_void_p()
    rc = lib.bdm_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == bdm.BDM_EINVAL
    assert b"launch limits" in lib.bdm_last_error(h)
    lib.bdm_destroy(h)


@pytest.mark.parametrize("precision,slots,cap", [(7, 4, 100), (bdm.BDM_MIXED, 0, 100),
                                                  (bdm.BDM_FP64, 4, 0), (bdm.BDM_MIXED, 1 << 16, 1 << 16)])
def test_mbatch_create_rejects_bad_shapes_before_any_cuda_call(lib, precision, slots, cap):
    """A bad precision, an empty pool or a pool of 2^31 agent places or more is refused before any
    stream or device memory is created (this runs without a GPU)."""
    h = ctypes.c_void_p()
    rc = lib.bdm_mbatch_create(precision, slots, cap, None, ctypes.byref(h))
    assert rc == bdm.BDM_EINVAL
    assert b"below 2^31" in lib.bdm_mbatch_last_error(h)
    lib.bdm_mbatch_destroy(h)
