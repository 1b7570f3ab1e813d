"""Thin ctypes binding of libbdm.so (the C ABI in include/bdm.h).

Functions carry the C names and only marshal arguments; every step of the simulation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library cannot be loaded, ``load()``
raises.  ``Sim`` is a convenience wrapper over the same calls that routes device allocations through
PyTorch's caching allocator and enqueues work on a PyTorch stream.
"""
import ctypes
import os

import numpy as np

from . import build as _build

BDM_OK, BDM_EINVAL, BDM_ENOMEM, BDM_ECUDA, BDM_ESTATE, BDM_ETIMEOUT, BDM_EBUDGET = 0, -1, -2, -3, -4, -5, -6
BDM_MECHANICS, BDM_SIR = 0, 1
BDM_FP64, BDM_MIXED = 0, 1

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("kind", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("record_diagnostics", ctypes.c_int32),
        ("dt", ctypes.c_double), ("repulsion", ctypes.c_double), ("attraction", ctypes.c_double),
        ("max_displacement", ctypes.c_double), ("interaction_radius", ctypes.c_double),
        ("box_length", ctypes.c_double), ("skin", ctypes.c_double),
        ("growth_enabled", ctypes.c_int32), ("force_variant", ctypes.c_int32),
        ("growth_volume", ctypes.c_double), ("division_volume", ctypes.c_double),
        ("division_offset_frac", ctypes.c_double),
        ("diffusion_enabled", ctypes.c_int32), ("grid_n", ctypes.c_int32 * 3),
        ("grid_origin", ctypes.c_double * 3), ("voxel", ctypes.c_double),
        ("diffusion_coeff", ctypes.c_double), ("decay", ctypes.c_double),
        ("dt_diffusion", ctypes.c_double), ("secretion", ctypes.c_double),
        ("sir_domain", ctypes.c_double), ("sir_radius", ctypes.c_double),
        ("sir_step", ctypes.c_double), ("p_infect", ctypes.c_double),
        ("p_recover", ctypes.c_double), ("sir_boxes", ctypes.c_int32),
        ("reserved2", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("run_id", ctypes.c_uint32), ("reserved3", ctypes.c_uint32),
        ("capacity", ctypes.c_uint64), ("box_capacity", ctypes.c_uint64),
        ("skip_stationary", ctypes.c_int32), ("reserved4", ctypes.c_int32),
        ("brownian_sigma", ctypes.c_double), ("p_apoptosis", ctypes.c_double),
        ("chemotaxis", ctypes.c_double),
        ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
    ]


class State(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
        ("n", ctypes.c_uint64), ("step", ctypes.c_uint64),
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
        ("diameter", ctypes.c_void_p), ("volume", ctypes.c_void_p), ("sir_state", ctypes.c_void_p),
        ("neighbour_count", ctypes.c_void_p), ("box_id", ctypes.c_void_p), ("grid", ctypes.c_void_p),
        ("mass_total", ctypes.c_double), ("sir_counts", ctypes.c_uint32 * 3),
        ("grid_rebuilds", ctypes.c_uint32), ("grid_origin_q", ctypes.c_int64 * 3),
        ("grid_box_q", ctypes.c_int64), ("grid_dims", ctypes.c_int64 * 3),
        ("list_entries", ctypes.c_uint64), ("stationary_skipped", ctypes.c_uint64),
    ]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("history_steps", ctypes.c_uint32),
                ("spin_limit", ctypes.c_uint32), ("barrier_extra", ctypes.c_uint32),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("persistent_only", ctypes.c_uint32),
                ("reserved0", ctypes.c_uint32)]


class NeuriteParams(ctypes.Structure):
    """Mirror of bdm_neurite_params (include/bdm_neurite.h)."""
    _fields_ = [("struct_size", ctypes.c_uint32), ("precision", ctypes.c_int32),
                ("dt", ctypes.c_double), ("repulsion", ctypes.c_double),
                ("attraction", ctypes.c_double), ("max_displacement", ctypes.c_double),
                ("spring", ctypes.c_double), ("interaction_radius", ctypes.c_double),
                ("capacity", ctypes.c_uint64), ("box_capacity", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("skin", ctypes.c_double)]


_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libbdm.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libbdm.so is not built (run __graft_entry__.build()); no CPU fallback")
    L = ctypes.CDLL(_build.LIB)
    vp, i32, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
    L.bdm_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(vp)]
    L.bdm_add_agents.argtypes = [vp, sz, vp, vp, vp, vp, vp, vp]
    L.bdm_set_grid.argtypes = [vp, vp]
    L.bdm_set_step.argtypes = [vp, u64]
    L.bdm_reset.argtypes = [vp]
    L.bdm_step.argtypes = [vp, i32]
    L.bdm_diffusion_step.argtypes = [vp, i32]
    L.bdm_get_state.argtypes = [vp, ctypes.POINTER(State)]
    L.bdm_destroy.argtypes = [vp]
    L.bdm_destroy.restype = None
    L.bdm_last_error.argtypes = [vp]
    L.bdm_last_error.restype = ctypes.c_char_p
    L.bdm_profile.argtypes = [vp, i32]
    L.bdm_kernel_times.argtypes = [vp, ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
    L.bdm_launch_count.restype = u64
    L.bdm_version.restype = ctypes.c_char_p
    L.bdm_philox.argtypes = [sz, vp, vp, vp]
    L.bdm_diffusion_step_noalloc.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, vp, vp]
    L.bdm_batch_create.argtypes = [ctypes.POINTER(Params), i32, ctypes.POINTER(BatchOptions),
                                   ctypes.POINTER(vp)]
    L.bdm_batch_add_agents.argtypes = [vp, i32, sz, vp, vp, vp, vp]
    L.bdm_batch_step.argtypes = [vp, i32]
    L.bdm_batch_sync.argtypes = [vp]
    L.bdm_batch_get_state.argtypes = [vp, i32, ctypes.POINTER(State)]
    L.bdm_batch_counts.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
    L.bdm_batch_destroy.argtypes = [vp]
    L.bdm_batch_destroy.restype = None
    L.bdm_batch_last_error.argtypes = [vp]
    L.bdm_batch_last_error.restype = ctypes.c_char_p
    L.bdm_mbatch_create.argtypes = [i32, i32, sz, vp, ctypes.POINTER(vp)]
    L.bdm_mbatch_load.argtypes = [vp, i32, ctypes.POINTER(Params), sz, vp, vp, vp, vp, i32]
    L.bdm_mbatch_step.argtypes = [vp, i32]
    L.bdm_mbatch_poll.argtypes = [vp, vp]
    L.bdm_mbatch_get_state.argtypes = [vp, i32, ctypes.POINTER(State)]
    L.bdm_mbatch_release.argtypes = [vp, i32]
    L.bdm_mbatch_destroy.argtypes = [vp]
    L.bdm_mbatch_destroy.restype = None
    L.bdm_mbatch_last_error.argtypes = [vp]
    L.bdm_mbatch_last_error.restype = ctypes.c_char_p
    L.bdm_neurite_create.argtypes = [ctypes.POINTER(NeuriteParams), ctypes.POINTER(vp)]
    L.bdm_neurite_set_agents.argtypes = [vp, sz] + [vp] * 9
    L.bdm_neurite_step.argtypes = [vp, i32]
    L.bdm_neurite_get_state.argtypes = [vp, ctypes.POINTER(sz), vp, vp, vp, vp,
                                        ctypes.POINTER(ctypes.c_double)]
    L.bdm_neurite_profile.argtypes = [vp, i32]
    L.bdm_neurite_list_info.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]
    L.bdm_neurite_kernel_times.argtypes = [vp, ctypes.POINTER(KernelTime), i32,
                                           ctypes.POINTER(i32)]
    L.bdm_neurite_destroy.argtypes = [vp]
    L.bdm_neurite_destroy.restype = None
    L.bdm_neurite_last_error.argtypes = [vp]
    L.bdm_neurite_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


class BdmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bdm error %d: %s" % (code, msg))
        self.code = code


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, handle=None):
    if rc != BDM_OK:
        msg = load().bdm_last_error(handle).decode() if handle else ""
        raise BdmError(rc, msg)


def make_params(d: dict) -> Params:
    """Build a Params struct from a parameter dictionary (unknown keys are ignored)."""
    p = Params()
    p.struct_size = ctypes.sizeof(Params)
    kind = d.get("kind", "mechanics")
    p.kind = BDM_SIR if kind in ("sir", BDM_SIR) else BDM_MECHANICS
    prec = d.get("precision", "mixed")
    p.precision = BDM_FP64 if prec in ("fp64", BDM_FP64) else BDM_MIXED
    for name in ("dt", "repulsion", "attraction", "max_displacement", "interaction_radius",
                 "box_length", "skin", "growth_volume", "division_volume", "division_offset_frac", "voxel",
                 "diffusion_coeff", "decay", "dt_diffusion", "secretion", "sir_domain", "sir_radius",
                 "sir_step", "p_infect", "p_recover", "brownian_sigma", "p_apoptosis", "chemotaxis"):
        if name in d:
            setattr(p, name, float(d[name]))
    for name in ("growth_enabled", "force_variant", "diffusion_enabled", "sir_boxes", "skip_stationary"):
        if name in d:
            setattr(p, name, int(d[name]))
    if "grid_n" in d:
        p.grid_n[:] = [int(v) for v in d["grid_n"]]
    if "grid_origin" in d:
        p.grid_origin[:] = [float(v) for v in d["grid_origin"]]
    p.seed = int(d.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    p.run_id = int(d.get("run_id", 0))
    p.capacity = int(d.get("capacity", 0))
    p.box_capacity = int(d.get("box_capacity", 0))
    return p


# ---- the C calls, by name -----------------------------------------------------------------------
def bdm_create(params: Params):
    h = ctypes.c_void_p()
    rc = load().bdm_create(ctypes.byref(params), ctypes.byref(h))
    if rc != BDM_OK:
        msg = load().bdm_last_error(h).decode() if h else ""
        if h:
            load().bdm_destroy(h)
        raise BdmError(rc, msg)
    return h


def bdm_add_agents(h, x, y, z, diameter=None, volume=None, sir_state=None):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    d = None if diameter is None else np.ascontiguousarray(diameter, np.float32)
    v = None if volume is None else np.ascontiguousarray(volume, np.float64)
    s = None if sir_state is None else np.ascontiguousarray(sir_state, np.uint8)
    _check(load().bdm_add_agents(h, len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(d), _ptr(v), _ptr(s)), h)


def bdm_set_grid(h, values):
    v = np.ascontiguousarray(values, np.float32)
    _check(load().bdm_set_grid(h, _ptr(v)), h)


def bdm_set_step(h, step: int):
    _check(load().bdm_set_step(h, int(step)), h)


def bdm_reset(h):
    _check(load().bdm_reset(h), h)


def bdm_step(h, n: int = 1):
    _check(load().bdm_step(h, int(n)), h)


def bdm_diffusion_step(h, n: int = 1):
    _check(load().bdm_diffusion_step(h, int(n)), h)


FIELDS = ("x", "y", "z", "diameter", "volume", "sir_state", "neighbour_count", "box_id", "grid")
_DTYPES = {"x": np.float64, "y": np.float64, "z": np.float64, "diameter": np.float32,
           "volume": np.float64, "sir_state": np.uint8, "neighbour_count": np.uint32,
           "box_id": np.uint32, "grid": np.float32}


def bdm_get_state(h, fields=FIELDS, grid_size=0, out=None):
    """Read the state in agent-id order.  ``out`` may supply preallocated (e.g. pinned) arrays."""
    L = load()
    st = State()
    st.struct_size = ctypes.sizeof(State)
    _check(L.bdm_get_state(h, ctypes.byref(st)), h)
    n = st.n
    arrays = {}
    st2 = State()
    st2.struct_size = ctypes.sizeof(State)
    for f in fields:
        if f == "grid" and not grid_size:
            continue
        size = grid_size if f == "grid" else n
        a = out.get(f) if out else None
        if a is None:
            a = np.empty(size, _DTYPES[f])
        arrays[f] = a
        setattr(st2, f, a.ctypes.data)
    _check(L.bdm_get_state(h, ctypes.byref(st2)), h)
    res = dict(arrays)
    res.update(n=int(st2.n), step=int(st2.step), mass_total=float(st2.mass_total),
               sir_counts=np.array(st2.sir_counts[:], np.uint32), grid_rebuilds=int(st2.grid_rebuilds),
               list_entries=int(st2.list_entries), stationary_skipped=int(st2.stationary_skipped),
               grid_origin_q=np.array(st2.grid_origin_q[:], np.int64),
               grid_box_q=int(st2.grid_box_q), grid_dims=np.array(st2.grid_dims[:], np.int64))
    return res


def bdm_destroy(h):
    if h:
        load().bdm_destroy(h)


def bdm_last_error(h) -> str:
    return load().bdm_last_error(h).decode()


def bdm_profile(h, enable=True):
    _check(load().bdm_profile(h, 1 if enable else 0), h)


def bdm_kernel_times(h):
    L = load()
    arr = (KernelTime * 64)()
    cnt = ctypes.c_int(0)
    _check(L.bdm_kernel_times(h, arr, 64, ctypes.byref(cnt)), h)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(cnt.value, 64))}


def bdm_launch_count() -> int:
    return int(load().bdm_launch_count())


def bdm_version() -> str:
    return load().bdm_version().decode()


def bdm_philox(ctr, key):
    """Philox4x32-10 blocks computed by the library's device generator: ctr (n,4), key (n,2)."""
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, np.uint32).reshape(-1, 2),
                                               (ctr.shape[0], 2)))
    out = np.zeros_like(ctr)
    _check(load().bdm_philox(ctr.shape[0], _ptr(ctr), _ptr(key), _ptr(out)))
    return out


def bdm_diffusion_step_noalloc(u_ptr, out_ptr, grid_n, diffusion_coeff, dt_diffusion, voxel,
                               decay, mass_ptr=None, stream=None):
    """One FTCS step on caller-owned DEVICE buffers (integer device addresses); allocates nothing.
    Returns the bdm status code."""
    gn = (ctypes.c_int32 * 3)(*[int(v) for v in grid_n])
    return load().bdm_diffusion_step_noalloc(u_ptr, out_ptr, gn, float(diffusion_coeff),
                                             float(dt_diffusion), float(voxel), float(decay),
                                             mass_ptr, stream)


def _bcheck(rc, b):
    if rc != BDM_OK:
        raise BdmError(rc, load().bdm_batch_last_error(b).decode() if b else "")


def bdm_batch_create(param_list, options=None):
    arr = (Params * len(param_list))(*param_list)
    b = ctypes.c_void_p()
    rc = load().bdm_batch_create(arr, len(param_list), ctypes.byref(options) if options else None,
                                 ctypes.byref(b))
    if rc != BDM_OK:
        msg = load().bdm_batch_last_error(b).decode() if b else ""
        if b:
            load().bdm_batch_destroy(b)
        raise BdmError(rc, msg)
    return b


def bdm_batch_add_agents(b, sim, x, y, z, sir_state=None):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    s = None if sir_state is None else np.ascontiguousarray(sir_state, np.uint8)
    _bcheck(load().bdm_batch_add_agents(b, int(sim), len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(s)), b)


def bdm_batch_step(b, n=1):
    _bcheck(load().bdm_batch_step(b, int(n)), b)


def bdm_batch_sync(b):
    _bcheck(load().bdm_batch_sync(b), b)


def bdm_batch_get_state(b, sim, fields=("x", "y", "z", "sir_state", "neighbour_count", "box_id")):
    L = load()
    st = State()
    st.struct_size = ctypes.sizeof(State)
    _bcheck(L.bdm_batch_get_state(b, int(sim), ctypes.byref(st)), b)
    n = st.n
    arrays = {f: np.empty(n, _DTYPES[f]) for f in fields}
    st2 = State()
    st2.struct_size = ctypes.sizeof(State)
    for f, a in arrays.items():
        setattr(st2, f, a.ctypes.data)
    _bcheck(L.bdm_batch_get_state(b, int(sim), ctypes.byref(st2)), b)
    arrays.update(n=int(st2.n), step=int(st2.step), sir_counts=np.array(st2.sir_counts[:], np.uint32))
    return arrays


def bdm_batch_counts(b, runs, max_steps):
    out = np.zeros((max_steps, runs, 3), np.uint32)
    got = ctypes.c_int(0)
    _bcheck(load().bdm_batch_counts(b, _ptr(out), int(max_steps), ctypes.byref(got)), b)
    return out[: got.value]


def bdm_batch_destroy(b):
    if b:
        load().bdm_batch_destroy(b)


class MechBatch:
    """Pool of mechanics simulation slots advanced together (bdm_mbatch_*): load a simulation into a
    free slot with its step target, step the pool, poll, read a finished slot, release it."""

    def __init__(self, precision="mixed", slots=64, slot_capacity=32768, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.slots = int(slots)
        self.slot_capacity = int(slot_capacity)
        prec = {"fp64": 0, "mixed": 1}[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        rc = load().bdm_mbatch_create(prec, self.slots, self.slot_capacity,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != BDM_OK:
            msg = load().bdm_mbatch_last_error(h).decode() if h else ""
            if h:
                load().bdm_mbatch_destroy(h)
            raise BdmError(rc, msg)
        self.h = h

    def _check(self, rc):
        if rc != BDM_OK:
            raise BdmError(rc, load().bdm_mbatch_last_error(self.h).decode())

    def load_sim(self, slot, params, x, y, z, diameter, steps):
        p = make_params(dict(params, kind="mechanics"))
        x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
        d = np.ascontiguousarray(diameter, np.float32)
        self._check(load().bdm_mbatch_load(self.h, int(slot), ctypes.byref(p), len(x), _ptr(x), _ptr(y),
                                           _ptr(z), _ptr(d), int(steps)))

    def step(self, n=1):
        self._check(load().bdm_mbatch_step(self.h, int(n)))

    def poll(self):
        out = np.empty(self.slots, np.int32)
        self._check(load().bdm_mbatch_poll(self.h, _ptr(out)))
        return out

    def get_state(self, slot, fields=("x", "y", "z", "diameter", "neighbour_count", "box_id")):
        L = load()
        st = State()
        st.struct_size = ctypes.sizeof(State)
        self._check(L.bdm_mbatch_get_state(self.h, int(slot), ctypes.byref(st)))
        n = st.n
        arrays = {f: np.empty(n, _DTYPES[f]) for f in fields}
        st2 = State()
        st2.struct_size = ctypes.sizeof(State)
        for f, a in arrays.items():
            setattr(st2, f, a.ctypes.data)
        self._check(L.bdm_mbatch_get_state(self.h, int(slot), ctypes.byref(st2)))
        res = dict(arrays)
        res.update(n=int(st2.n), step=int(st2.step), grid_origin_q=np.array(st2.grid_origin_q[:], np.int64),
                   grid_box_q=int(st2.grid_box_q), grid_dims=np.array(st2.grid_dims[:], np.int64))
        return res

    def release(self, slot):
        self._check(load().bdm_mbatch_release(self.h, int(slot)))

    def close(self):
        if self.h:
            load().bdm_mbatch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched SIR ensemble: one persistent launch per step for every run; memory from PyTorch."""

    def __init__(self, param_dicts, history_steps=0, spin_limit=0, barrier_extra=0, stream=None,
                 torch_memory=True, persistent_only=False):
        import torch
        self.runs = len(param_dicts)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        opt = BatchOptions()
        opt.struct_size = ctypes.sizeof(BatchOptions)
        opt.history_steps = int(history_steps)
        opt.spin_limit = int(spin_limit)
        opt.barrier_extra = int(barrier_extra)
        opt.persistent_only = 1 if persistent_only else 0
        opt.stream = self.stream.cuda_stream
        self._allocator = None
        if torch_memory:
            self._allocator = TorchAllocator(self.stream)
            opt.alloc = self._allocator.alloc_fn
            opt.free = self._allocator.free_fn
        self._opt = opt
        self.h = bdm_batch_create([make_params(d) for d in param_dicts], opt)

    def add_agents(self, sim, x, y, z, sir_state=None):
        bdm_batch_add_agents(self.h, sim, x, y, z, sir_state)

    def step(self, n=1):
        bdm_batch_step(self.h, n)

    def sync(self):
        bdm_batch_sync(self.h)

    def get_state(self, sim, **kw):
        return bdm_batch_get_state(self.h, sim, **kw)

    def counts(self, max_steps):
        return bdm_batch_counts(self.h, self.runs, max_steps)

    def close(self):
        if self.h:
            bdm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience wrapper ----------------------------------------------------------------------------
class TorchAllocator:
    """Device allocations through PyTorch's caching allocator on a given stream."""

    def __init__(self, stream):
        import torch
        self._torch = torch
        self.stream = stream
        self.device = stream.device.index if stream.device.index is not None else 0
        self.live = {}

        def _alloc(nbytes, user):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:  # out of memory -> the library reports BDM_ENOMEM
                return None
            self.live[ptr] = nbytes
            return ptr

        def _free(ptr, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class Sim:
    """One simulation handle.  params: dict as produced by ``synth``; device memory from PyTorch."""

    def __init__(self, params: dict, stream=None, torch_memory: bool = True):
        import torch
        self.params = dict(params)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        p = make_params(self.params)
        p.stream = self.stream.cuda_stream
        self._allocator = None
        if torch_memory:
            self._allocator = TorchAllocator(self.stream)
            p.alloc = self._allocator.alloc_fn
            p.free = self._allocator.free_fn
        self._p = p
        self.h = bdm_create(p)
        gn = self.params.get("grid_n")
        self.grid_size = int(np.prod(gn)) if (gn and self.params.get("diffusion_enabled")) else 0

    def add_agents(self, x, y, z, diameter=None, volume=None, sir_state=None):
        bdm_add_agents(self.h, x, y, z, diameter, volume, sir_state)

    def set_grid(self, values):
        bdm_set_grid(self.h, np.asarray(values, np.float32).reshape(-1))

    def set_step(self, step):
        bdm_set_step(self.h, step)

    def reset(self):
        bdm_reset(self.h)

    def step(self, n=1):
        bdm_step(self.h, n)

    def diffusion_step(self, n=1):
        bdm_diffusion_step(self.h, n)

    def state_fields(self):
        """The fields this handle writes: no diameter or volume for SIR, no SIR state for
        mechanics, and volume only with growth."""
        if self.params.get("kind", "mechanics") in ("sir", BDM_SIR):
            skip = {"diameter", "volume"}
        else:
            skip = {"sir_state"} | (set() if self.params.get("growth_enabled") else {"volume"})
        return tuple(f for f in FIELDS if f not in skip)

    def get_state(self, fields=None, out=None):
        have = self.state_fields()
        if fields is None:
            fields = have
        missing = [f for f in fields if f not in have and f != "grid"]
        if missing:
            raise ValueError("this handle does not hold %s" % ", ".join(missing))
        return bdm_get_state(self.h, fields, self.grid_size, out)

    def profile(self, enable=True):
        bdm_profile(self.h, enable)

    def kernel_times(self):
        return bdm_kernel_times(self.h)

    def close(self):
        if self.h:
            bdm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------------------
# Neurite mechanics (include/bdm_neurite.h)
# ------------------------------------------------------------------------------------------------
NEURITE_FIELDS = ("x", "y", "z", "diameter", "rest", "mother", "ox", "oy", "oz")


class Neurite:
    """One neurite-mechanics handle (somata and neurite elements).  params: dict as produced by
    ``synth.neuron_forest`` plus ``precision`` ("mixed" or "fp64"), ``capacity`` and optionally
    ``box_capacity`` (default 8 * capacity + 4096 grid boxes)."""

    def __init__(self, params: dict, stream=None):
        import torch
        self.params = dict(params)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        p = NeuriteParams()
        p.struct_size = ctypes.sizeof(NeuriteParams)
        p.precision = BDM_MIXED if self.params.get("precision", "mixed") == "mixed" else BDM_FP64
        for k in ("dt", "repulsion", "attraction", "max_displacement", "spring",
                  "interaction_radius", "skin"):
            setattr(p, k, float(self.params.get(k, 0.0)))
        p.capacity = int(self.params.get("capacity", 1 << 20))
        # grid room for arbors that spread well beyond their somata (the library's own default,
        # 2 * capacity + 4096 boxes, suits compact populations)
        p.box_capacity = int(self.params.get("box_capacity", 0)) or 8 * p.capacity + 4096
        p.stream = self.stream.cuda_stream
        L = load()
        h = ctypes.c_void_p()
        rc = L.bdm_neurite_create(ctypes.byref(p), ctypes.byref(h))
        if rc != BDM_OK:
            msg = L.bdm_neurite_last_error(h).decode() if h.value else ""
            L.bdm_neurite_destroy(h)
            raise BdmError(rc, msg)
        self.h = h
        self._keep = None

    def _check(self, rc):
        if rc != BDM_OK:
            raise BdmError(rc, load().bdm_neurite_last_error(self.h).decode())

    def set_agents(self, inp: dict):
        """inp: x, y, z, diameter, rest, ox, oy, oz (float64) and mother (int32), one entry per
        agent in id order."""
        arrs = [np.ascontiguousarray(inp[k], np.int32 if k == "mother" else np.float64)
                for k in NEURITE_FIELDS]
        n = len(arrs[0])
        if any(len(a) != n for a in arrs):
            raise ValueError("neurite input arrays differ in length")
        self._keep = arrs  # alive until the copies are done (the call synchronises)
        self._check(load().bdm_neurite_set_agents(self.h, n, *[_ptr(a) for a in arrs]))
        self._keep = None

    def step(self, n: int = 1):
        self._check(load().bdm_neurite_step(self.h, int(n)))

    def get_state(self) -> dict:
        L = load()
        n = ctypes.c_size_t(0)
        self._check(L.bdm_neurite_get_state(self.h, ctypes.byref(n), None, None, None, None,
                                            None))
        n = n.value
        out = {k: np.zeros(n) for k in ("x", "y", "z")}
        nbr = np.zeros(n, np.uint32)
        Lr = ctypes.c_double(0.0)
        m = ctypes.c_size_t(0)
        self._check(L.bdm_neurite_get_state(self.h, ctypes.byref(m), _ptr(out["x"]),
                                            _ptr(out["y"]), _ptr(out["z"]), _ptr(nbr),
                                            ctypes.byref(Lr)))
        out.update(n=n, neighbour_count=nbr, L=Lr.value)
        return out

    def profile(self, enable=True):
        self._check(load().bdm_neurite_profile(self.h, 1 if enable else 0))

    def list_info(self):
        """(rebuilds so far, entries listed by the last rebuild); both 0 without a skin."""
        rb, ent = ctypes.c_uint64(0), ctypes.c_uint64(0)
        self._check(load().bdm_neurite_list_info(self.h, ctypes.byref(rb), ctypes.byref(ent)))
        return int(rb.value), int(ent.value)

    def kernel_times(self):
        arr = (KernelTime * 64)()
        cnt = ctypes.c_int(0)
        self._check(load().bdm_neurite_kernel_times(self.h, arr, 64, ctypes.byref(cnt)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
                for i in range(min(cnt.value, 64))}

    def close(self):
        if self.h is not None and self.h.value:
            load().bdm_neurite_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
