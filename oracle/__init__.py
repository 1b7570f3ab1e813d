"""FP64 CPU oracle for the agent-mechanics hot path -- TEST INFRASTRUCTURE.

A plain, slow, obviously correct restatement of what one simulation step computes, used only by the
tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``.  The product
library never imports or links it and shares no code with it.  Each function cites the passage of
BioDynaMo (arXiv 2006.06775) it follows, or the reading of the paper that fills a gap (readings
R1-R20 are listed with their justification in the design notes at the repository root).

Functions without an independent pin: the daughter offset distance and the division axis law (R7)
are readings the paper does not fix; their tests check internal consistency only (parity unpinned).
The oncology behaviours (Brownian migration R13, apoptosis R14) and chemotaxis (R15) are readings
too: the paper names them but prints neither law nor rate.  Their tests pin distributional facts (standard normal
deviates, binomial survival, order kept), not the paper's parameters.  Neurite mechanics (R16-R20)
follows a force law the paper does not print (it names the Cortex3D model): its tests pin the
geometry (closest points against brute-force minimisation), the spring and lever split against
closed forms, and the conservation of the total force; the law itself is parity unpinned.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class MechParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("k_rep", ctypes.c_double), ("gamma_att", ctypes.c_double),
                ("max_disp", ctypes.c_double), ("interaction_radius", ctypes.c_double),
                ("box_length", ctypes.c_double)]


class NeuriteParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("k_rep", ctypes.c_double), ("gamma_att", ctypes.c_double),
                ("max_disp", ctypes.c_double), ("k_spring", ctypes.c_double),
                ("interaction_radius", ctypes.c_double)]


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_philox4x32_10_n.argtypes = [ctypes.c_size_t, _u32p, _u32p, _u32p]
        L.orc_grid.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f32p, ctypes.c_double,
                               ctypes.c_double, _f64p, _u32p]
        L.orc_mech_step.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f32p,
                                    ctypes.POINTER(MechParams), _f64p, _f64p, _f64p, _u32p, _u32p,
                                    _f64p, _f64p, _f64p, _f64p]
        L.orc_grow_divide.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f32p, _f64p,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.POINTER(ctypes.c_size_t)]
        L.orc_apoptosis.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f32p, _f64p,
                                    ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32]
        L.orc_apoptosis.restype = ctypes.c_size_t
        L.orc_brownian.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, ctypes.c_double,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_chemotaxis.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                     _f64p, _i64p, _f64p, ctypes.c_double, ctypes.c_double]
        L.orc_secrete.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f64p, _i64p, _f64p,
                                  ctypes.c_double, ctypes.c_double]
        L.orc_ftcs.argtypes = [_i64p, _f64p, _f64p, ctypes.c_double, ctypes.c_double]
        L.orc_ftcs.restype = ctypes.c_double
        L.orc_sir_step.argtypes = [ctypes.c_size_t, _i32p, _i32p, _i32p, _u8p, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, _i32p, _i32p, _i32p, _u8p, _u32p, _u32p, _u32p]
        L.orc_segment_closest.argtypes = [_f64p, _f64p, _f64p, _f64p,
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.orc_neurite_step.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f64p, _f64p, _i32p,
                                       _f64p, _f64p, _f64p, ctypes.POINTER(NeuriteParams), _f64p,
                                       _f64p, _f64p, _u32p, ctypes.POINTER(ctypes.c_double),
                                       _f64p, _f64p, _f64p]
        L.orc_neurite_sample.argtypes = [ctypes.c_size_t, _f64p, _f64p, _f64p, _f64p, _f64p,
                                         _i32p, _f64p, _f64p, _f64p,
                                         ctypes.POINTER(NeuriteParams), ctypes.c_size_t, _i64p,
                                         _f64p, _f64p, _f64p, _u32p,
                                         ctypes.POINTER(ctypes.c_double)]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().orc_num_threads()


# ------------------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# ------------------------------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x32-10 blocks: ctr (n, 4) uint32, key (n, 2) uint32 -> (n, 4) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32).reshape(-1, 2),
                                               (ctr.shape[0], 2)))
    out = np.zeros_like(ctr)
    lib().orc_philox4x32_10_n(ctr.shape[0], ctr.reshape(-1), key.reshape(-1), out.reshape(-1))
    return out


# ------------------------------------------------------------------------------------------------
# Grid and mechanics (paper Sec. "Simulation concepts"; readings R1-R5)
# ------------------------------------------------------------------------------------------------
GRID_Q = 20  # fixed-point bits of the grid lattice (reading R5)


def _grid_dict(g):
    return {"origin_q": g[0:3].astype(np.int64), "R": float(g[3]), "L": float(g[4]),
            "Lq": int(g[5]), "dims": g[6:9].astype(np.int64), "nbox": int(g[9])}


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def grid(x, y, z, diam, interaction_radius=0.0, box_length=0.0):
    """Grid of one step: returns (grid dict, box id per agent)."""
    n = len(x)
    g = np.zeros(10)
    box = np.zeros(n, np.uint32)
    rc = lib().orc_grid(n, _f64(x), _f64(y), _f64(z), _f32(diam), interaction_radius, box_length,
                        g, box)
    if rc:
        raise ValueError("orc_grid rejected the input (%d)" % rc)
    return _grid_dict(g), box


def mech_step(x, y, z, diam, dt, repulsion, attraction, max_displacement, interaction_radius=0.0,
              box_length=0.0, want_force=False):
    """One Jacobi mechanics step.  Returns dict of new x, y, z, neighbour counts, box ids, grid."""
    n = len(x)
    p = MechParams(dt, repulsion, attraction, max_displacement, interaction_radius, box_length)
    out = {k: np.zeros(n) for k in ("x", "y", "z", "fx", "fy", "fz")}
    nbr = np.zeros(n, np.uint32)
    box = np.zeros(n, np.uint32)
    g = np.zeros(10)
    rc = lib().orc_mech_step(n, _f64(x), _f64(y), _f64(z), _f32(diam), ctypes.byref(p),
                             out["x"], out["y"], out["z"], nbr, box, g, out["fx"], out["fy"],
                             out["fz"])
    if rc:
        raise ValueError("orc_mech_step rejected the input (%d)" % rc)
    res = {"x": out["x"], "y": out["y"], "z": out["z"], "neighbour_count": nbr, "box_id": box,
           "grid": _grid_dict(g) if n else None}
    if want_force:
        res["force"] = np.stack([out["fx"], out["fy"], out["fz"]], axis=1)
    return res


# ------------------------------------------------------------------------------------------------
# Neurite mechanics (paper Sec. "Neuroscience module"; readings R16-R20)
# ------------------------------------------------------------------------------------------------
def segment_closest(p0, u, q0, v):
    """Parameters (s, t) in [0, 1]^2 of the closest points of segments p0 + s u and q0 + t v."""
    s, t = ctypes.c_double(), ctypes.c_double()
    lib().orc_segment_closest(_f64(p0), _f64(u), _f64(q0), _f64(v), ctypes.byref(s),
                              ctypes.byref(t))
    return s.value, t.value


def neurite_step(x, y, z, diam, rest, mother, ox, oy, oz, dt, repulsion, attraction,
                 max_displacement, spring, interaction_radius=0.0):
    """One Jacobi step of neurite mechanics (brute force over all pairs).  Returns a dict of new
    x, y, z, neighbour counts, the radius L and each agent's total force (n, 3)."""
    n = len(x)
    p = NeuriteParams(dt, repulsion, attraction, max_displacement, spring, interaction_radius)
    out = {k: np.zeros(n) for k in ("x", "y", "z", "fx", "fy", "fz")}
    nbr = np.zeros(n, np.uint32)
    L = ctypes.c_double(0.0)
    rc = lib().orc_neurite_step(n, _f64(x), _f64(y), _f64(z), _f64(diam), _f64(rest),
                                np.ascontiguousarray(mother, dtype=np.int32), _f64(ox), _f64(oy),
                                _f64(oz), ctypes.byref(p), out["x"], out["y"], out["z"], nbr,
                                ctypes.byref(L), out["fx"], out["fy"], out["fz"])
    if rc:
        raise ValueError("orc_neurite_step rejected the input (%d)" % rc)
    return {"x": out["x"], "y": out["y"], "z": out["z"], "neighbour_count": nbr, "L": L.value,
            "force": np.stack([out["fx"], out["fy"], out["fz"]], axis=1)}


def neurite_sample(x, y, z, diam, rest, mother, ox, oy, oz, dt, repulsion, attraction,
                   max_displacement, spring, idx, interaction_radius=0.0):
    """neurite_step's result for the agents idx only: dict of x, y, z, neighbour counts (sample
    order) and L."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = len(idx)
    p = NeuriteParams(dt, repulsion, attraction, max_displacement, spring, interaction_radius)
    out = {k: np.zeros(m) for k in ("x", "y", "z")}
    nbr = np.zeros(m, np.uint32)
    L = ctypes.c_double(0.0)
    rc = lib().orc_neurite_sample(len(x), _f64(x), _f64(y), _f64(z), _f64(diam), _f64(rest),
                                  np.ascontiguousarray(mother, dtype=np.int32), _f64(ox),
                                  _f64(oy), _f64(oz), ctypes.byref(p), m, idx, out["x"],
                                  out["y"], out["z"], nbr, ctypes.byref(L))
    if rc:
        raise ValueError("orc_neurite_sample rejected the input (%d)" % rc)
    out.update(neighbour_count=nbr, L=L.value)
    return out


def grow_divide(x, y, z, diam, vol, growth_volume, division_volume, offset_frac, seed, run, step):
    """Growth + division (reading R7).  Returns new arrays (daughters appended)."""
    n = len(x)
    cap = 2 * n
    arrs = {}
    for name, src, dt in (("x", x, np.float64), ("y", y, np.float64), ("z", z, np.float64),
                          ("diameter", diam, np.float32), ("volume", vol, np.float64)):
        a = np.zeros(max(cap, 1), dt)
        a[:n] = src
        arrs[name] = a
    n_out = ctypes.c_size_t(0)
    lib().orc_grow_divide(n, arrs["x"], arrs["y"], arrs["z"], arrs["diameter"], arrs["volume"],
                          growth_volume, division_volume, offset_frac, seed & 0xFFFFFFFF,
                          run & 0xFFFFFFFF, step & 0xFFFFFFFF, ctypes.byref(n_out))
    m = n_out.value
    return {k: v[:m].copy() for k, v in arrs.items()}


def apoptosis(x, y, z, diam, vol, p_apoptosis, seed, run, step):
    """Apoptosis at step start (reading R14).  Returns the survivors' arrays (order kept)."""
    arrs = {"x": _f64(x).copy(), "y": _f64(y).copy(), "z": _f64(z).copy(),
            "diameter": _f32(diam).copy(), "volume": _f64(vol).copy()}
    m = lib().orc_apoptosis(len(x), arrs["x"], arrs["y"], arrs["z"], arrs["diameter"],
                            arrs["volume"], probability_threshold(p_apoptosis), seed & 0xFFFFFFFF,
                            run & 0xFFFFFFFF, step & 0xFFFFFFFF)
    return {k: v[:m].copy() for k, v in arrs.items()}


def brownian(x, y, z, sigma, seed, run, step):
    """Brownian migration after the mechanical update (reading R13); returns new x, y, z."""
    x, y, z = _f64(x).copy(), _f64(y).copy(), _f64(z).copy()
    lib().orc_brownian(len(x), x, y, z, float(sigma), seed & 0xFFFFFFFF, run & 0xFFFFFFFF,
                       step & 0xFFFFFFFF)
    return x, y, z


def chemotaxis(x, y, z, sx, sy, sz, grid_values, origin, voxel, chi):
    """Chemotaxis after the update (reading R15): returns x, y, z moved by chi * grad c, the grid
    gradient at the voxel of the step-start centres (sx, sy, sz); grid shape (nz, ny, nx)."""
    nz, ny, nx = grid_values.shape
    x, y, z = _f64(x).copy(), _f64(y).copy(), _f64(z).copy()
    lib().orc_chemotaxis(len(x), x, y, z, _f64(sx), _f64(sy), _f64(sz),
                         np.ascontiguousarray(grid_values, np.float64).reshape(-1),
                         np.array([nx, ny, nz], np.int64), _f64(origin), float(voxel), float(chi))
    return x, y, z


def secrete(x, y, z, grid_values, origin, voxel, amount):
    """Secretion (reading R8), in place on the FP64 grid (shape (nz, ny, nx))."""
    nz, ny, nx = grid_values.shape
    dims = np.array([nx, ny, nz], np.int64)
    flat = grid_values.reshape(-1)
    assert flat.base is grid_values or flat is grid_values or flat.flags.c_contiguous
    lib().orc_secrete(len(x), _f64(x), _f64(y), _f64(z), flat, dims, _f64(origin), voxel, amount)


def ftcs(u, lam, mu_dt):
    """One FTCS step (reading R9) of an FP64 grid of shape (nz, ny, nx).  Returns (u', mass)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    nz, ny, nx = u.shape
    out = np.empty_like(u)
    mass = lib().orc_ftcs(np.array([nx, ny, nz], np.int64), u.reshape(-1), out.reshape(-1), lam,
                          mu_dt)
    return out, mass


def ftcs_coefficients(diffusion_coeff, dt_diffusion, voxel, decay):
    """lambda = D dt / h^2 and mu dt, evaluated once in FP64 (reading R9)."""
    return (diffusion_coeff * dt_diffusion) / (voxel * voxel), decay * dt_diffusion


# ------------------------------------------------------------------------------------------------
# SIR (paper Sec. "Epidemiology use case"; reading R10)
# ------------------------------------------------------------------------------------------------
SIR_UNITS_PER_UM = 1024  # int32 fixed point, 2^-10 um


def sir_units(v_um: float) -> int:
    return int(round(v_um * SIR_UNITS_PER_UM))


def probability_threshold(p: float) -> int:
    """Event iff a uniform 32-bit word w < floor(p * 2^32) (reading R10)."""
    if not (0.0 <= p <= 1.0):
        raise ValueError("probability out of range")
    return int(math.floor(p * 4294967296.0))


def sir_step(X, Y, Z, state, L, nb, r, s, p_infect, p_recover, seed, run, step):
    """One synchronous SIR step of one run; positions are int32 lattice units."""
    n = len(X)
    nX, nY, nZ = (np.zeros(n, np.int32) for _ in range(3))
    nst = np.zeros(n, np.uint8)
    ninf = np.zeros(n, np.uint32)
    box = np.zeros(n, np.uint32)
    counts = np.zeros(3, np.uint32)
    rc = lib().orc_sir_step(n, np.ascontiguousarray(X, np.int32), np.ascontiguousarray(Y, np.int32),
                            np.ascontiguousarray(Z, np.int32), np.ascontiguousarray(state, np.uint8),
                            L, nb, r, s, probability_threshold(p_infect),
                            probability_threshold(p_recover), seed & 0xFFFFFFFF, run & 0xFFFFFFFF,
                            step & 0xFFFFFFFF, nX, nY, nZ, nst, ninf, box, counts)
    if rc:
        raise ValueError("orc_sir_step rejected the input (%d)" % rc)
    return {"X": nX, "Y": nY, "Z": nZ, "state": nst, "infected_neighbours": ninf, "box_id": box,
            "counts": counts}


# ------------------------------------------------------------------------------------------------
# One simulation, in the order of reading R11: behaviours (growth, division) -> grid rebuild and
# mechanics -> secretion -> diffusion (paper Sec. "Simulation concepts": agent operations run for
# every agent each step, standalone operations once per step).
# ------------------------------------------------------------------------------------------------
class OracleSim:
    """Mirror of one library simulation handle, driven by the same parameter dictionary."""

    def __init__(self, params: dict):
        self.p = dict(params)
        self.kind = self.p.get("kind", "mechanics")
        self.step_index = int(self.p.get("first_step", 0))
        self.n = 0
        self.x = np.zeros(0)
        self.y = np.zeros(0)
        self.z = np.zeros(0)
        self.diameter = np.zeros(0, np.float32)
        self.volume = np.zeros(0)
        self.state = np.zeros(0, np.uint8)
        self.X = self.Y = self.Z = np.zeros(0, np.int32)
        self.neighbour_count = np.zeros(0, np.uint32)
        self.box_id = np.zeros(0, np.uint32)
        self.last_grid = None
        self.sir_counts = np.zeros(3, np.uint32)
        self.grid = None
        self.mass = 0.0
        if self.p.get("diffusion_enabled"):
            nx, ny, nz = self.p["grid_n"]
            self.grid = np.zeros((nz, ny, nx))

    # -- initialisation (paper: "place agents in space, set their attributes") ------------------
    def add_agents(self, x, y, z, diameter=None, volume=None, sir_state=None):
        x, y, z = _f64(x), _f64(y), _f64(z)
        if self.kind == "sir":
            X = np.rint(x * SIR_UNITS_PER_UM).astype(np.int32)
            Y = np.rint(y * SIR_UNITS_PER_UM).astype(np.int32)
            Z = np.rint(z * SIR_UNITS_PER_UM).astype(np.int32)
            self.X = np.concatenate([self.X, X])
            self.Y = np.concatenate([self.Y, Y])
            self.Z = np.concatenate([self.Z, Z])
            st = np.zeros(len(x), np.uint8) if sir_state is None else np.asarray(sir_state, np.uint8)
            self.state = np.concatenate([self.state, st])
        else:
            d = _f32(diameter)
            self.x = np.concatenate([self.x, x])
            self.y = np.concatenate([self.y, y])
            self.z = np.concatenate([self.z, z])
            self.diameter = np.concatenate([self.diameter, d])
            if volume is None:
                dd = d.astype(np.float64)
                volume = (0.5235987755982988 * dd) * dd * dd
            self.volume = np.concatenate([self.volume, _f64(volume)])
        self.n += len(x)

    def set_grid(self, values):
        nx, ny, nz = self.p["grid_n"]
        self.grid = np.asarray(values, np.float32).astype(np.float64).reshape(nz, ny, nx).copy()
        self.mass = float(self.grid.sum())

    # -- execution ------------------------------------------------------------------------------
    def _mech_one(self):
        p = self.p
        if p.get("p_apoptosis", 0.0) > 0.0 and self.n:
            r = apoptosis(self.x, self.y, self.z, self.diameter, self.volume, p["p_apoptosis"],
                          p.get("seed", 0), p.get("run_id", 0), self.step_index)
            self.x, self.y, self.z = r["x"], r["y"], r["z"]
            self.diameter, self.volume = r["diameter"], r["volume"]
            self.n = len(self.x)
        if p.get("growth_enabled"):
            r = grow_divide(self.x, self.y, self.z, self.diameter, self.volume, p["growth_volume"],
                            p["division_volume"], p["division_offset_frac"], p.get("seed", 0),
                            p.get("run_id", 0), self.step_index)
            self.x, self.y, self.z = r["x"], r["y"], r["z"]
            self.diameter, self.volume = r["diameter"], r["volume"]
            self.n = len(self.x)
        if self.n:
            x0, y0, z0 = self.x, self.y, self.z
            r = mech_step(self.x, self.y, self.z, self.diameter, p["dt"], p["repulsion"],
                          p["attraction"], p["max_displacement"], p.get("interaction_radius", 0.0),
                          p.get("box_length", 0.0))
            self.x, self.y, self.z = r["x"], r["y"], r["z"]
            self.neighbour_count, self.box_id, self.last_grid = (r["neighbour_count"], r["box_id"],
                                                                 r["grid"])
            if p.get("brownian_sigma", 0.0) > 0.0:
                self.x, self.y, self.z = brownian(self.x, self.y, self.z, p["brownian_sigma"],
                                                  p.get("seed", 0), p.get("run_id", 0),
                                                  self.step_index)
            if p.get("chemotaxis", 0.0) and self.grid is not None:
                self.x, self.y, self.z = chemotaxis(self.x, self.y, self.z, x0, y0, z0, self.grid,
                                                    p["grid_origin"], p["voxel"], p["chemotaxis"])
        if p.get("diffusion_enabled"):
            if p.get("secretion", 0.0):
                secrete(self.x, self.y, self.z, self.grid, p["grid_origin"], p["voxel"],
                        p["secretion"])
            self._diffuse_one()

    def _diffuse_one(self):
        p = self.p
        lam, mu_dt = ftcs_coefficients(p["diffusion_coeff"], p["dt_diffusion"], p["voxel"],
                                       p["decay"])
        self.grid, self.mass = ftcs(self.grid, lam, mu_dt)

    def _sir_one(self):
        p = self.p
        r = sir_step(self.X, self.Y, self.Z, self.state, sir_units(p["sir_domain"]),
                     int(p["sir_boxes"]), sir_units(p["sir_radius"]), sir_units(p["sir_step"]),
                     p["p_infect"], p["p_recover"], p.get("seed", 0), p.get("run_id", 0),
                     self.step_index)
        self.X, self.Y, self.Z, self.state = r["X"], r["Y"], r["Z"], r["state"]
        self.neighbour_count, self.box_id = r["infected_neighbours"], r["box_id"]
        self.sir_counts = r["counts"]

    def step(self, n=1):
        for _ in range(n):
            if self.kind == "sir":
                self._sir_one()
            else:
                self._mech_one()
            self.step_index += 1

    def diffusion_step(self, n=1):
        for _ in range(n):
            self._diffuse_one()

    def get_state(self):
        s = {"n": self.n, "step": self.step_index, "neighbour_count": self.neighbour_count,
             "box_id": self.box_id}
        if self.kind == "sir":
            s.update(x=self.X / SIR_UNITS_PER_UM, y=self.Y / SIR_UNITS_PER_UM,
                     z=self.Z / SIR_UNITS_PER_UM, sir_state=self.state,
                     sir_counts=self.sir_counts)
        else:
            s.update(x=self.x, y=self.y, z=self.z, diameter=self.diameter, volume=self.volume)
        if self.grid is not None:
            s["grid"] = self.grid
            s["mass_total"] = self.mass
        return s
