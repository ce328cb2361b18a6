"""Thin ctypes binding of the ugkwp C-ABI (include/ugkwp.h).

Functions carry the C names and only marshal arguments: every step of the
method runs in the CUDA library ``libugkwp.so``.  There is no CPU fallback: if
the library cannot be built or loaded, or a call needs a GPU that is absent,
the call raises.  ``Simulation`` bundles the calls the way a user strings them
together, with the device workspace and the stream taken from PyTorch.
"""
import ctypes
import os

import numpy as np

from . import build_lib

# ------------------------------------------------------------- constants
OK = 0
E_ARG, E_MESH, E_CUDA, E_WORKSPACE, E_CAPACITY = -1, -2, -3, -4, -5
E_TRACK_LIMIT, E_FIXED_OVERFLOW, E_NONFINITE, E_STATE, E_UNSUPPORTED = -7, -8, -9, -10, -11
BC_DIFFUSE_WALL, BC_SPECULAR, BC_FARFIELD, BC_OUTFLOW = 1, 2, 3, 4
BC_TYPES = {"wall": BC_DIFFUSE_WALL, "specular": BC_SPECULAR, "farfield": BC_FARFIELD, "inflow": BC_FARFIELD,
            "outflow": BC_OUTFLOW}
FP64, MIXED = 0, 1
PRECISION = {"fp64": FP64, "mixed": MIXED}
W, WP, WH, PRIM, WBAR = 0, 1, 2, 3, 4
LAST = {"dt": 0, "tau": 1, "rho_h": 2, "n_sam": 3, "m_sam": 4, "flux": 5, "pflux": 6, "surv_mass": 7,
        "surv_count": 8, "grad_W": 9, "grad_rho_h": 10}


class UgkwpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ugkwp error {code}: {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tets", ctypes.c_int32), ("n_bfaces", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("xyz", ctypes.c_void_p), ("tets", ctypes.c_void_p),
                ("bfaces", ctypes.c_void_p), ("bface_tags", ctypes.c_void_p)]


class Bc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("reserved", ctypes.c_int32), ("T_w", ctypes.c_double),
                ("U_w", ctypes.c_double * 3), ("W_in", ctypes.c_double * 5)]


class Params(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("mu_ref", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("omega", ctypes.c_double), ("Pr", ctypes.c_double), ("CFL", ctypes.c_double),
                ("C2", ctypes.c_double), ("venkat_K", ctypes.c_double), ("order", ctypes.c_int32),
                ("N_ref", ctypes.c_int32), ("N_min", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_crossings", ctypes.c_int32), ("n_bc", ctypes.c_int32), ("sampling", ctypes.c_int32),
                ("K", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("particle_capacity", ctypes.c_int64), ("bc", Bc * 16)]


class Sizes(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_size_t), ("n_cells", ctypes.c_int64), ("n_faces", ctypes.c_int64),
                ("n_bfaces", ctypes.c_int64)]


SAMPLING = {"maxwell": 0, "energy_matched": 1, "gp1": 2}


class LaunchCfg(ctypes.Structure):
    _fields_ = [("particle_blocks", ctypes.c_int32), ("wave_blocks", ctypes.c_int32),
                ("track_threads", ctypes.c_int32), ("smem_carveout", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("step", ctypes.c_int64),
                ("n_particles", ctypes.c_int64), ("n_tracked", ctypes.c_int64), ("n_sampled", ctypes.c_int64),
                ("n_collided", ctypes.c_int64), ("n_exited", ctypes.c_int64), ("n_lost", ctypes.c_int64),
                ("n_crossings", ctypes.c_int64), ("n_wall_hits", ctypes.c_int64), ("n_moves_total", ctypes.c_int64),
                ("n_movers", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class State(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("step", ctypes.c_int64), ("t", ctypes.c_double),
                ("exps", ctypes.c_int32 * 5), ("reserved", ctypes.c_int32), ("W", ctypes.c_void_p),
                ("id", ctypes.c_void_p), ("cell", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("m", ctypes.c_void_p), ("e", ctypes.c_void_p)]


class StateNative(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("step", ctypes.c_int64), ("t", ctypes.c_double),
                ("exps", ctypes.c_int32 * 5), ("real_size", ctypes.c_int32), ("W", ctypes.c_void_p),
                ("id", ctypes.c_void_p), ("cell", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("m", ctypes.c_void_p), ("e", ctypes.c_void_p)]


class AdjointReq(ctypes.Structure):
    _fields_ = [("functional", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("wall_tags", ctypes.c_void_p),
                ("n_wall_tags", ctypes.c_int32), ("reserved_", ctypes.c_int32), ("theta", ctypes.c_void_p),
                ("d_workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


KERNELS = ["reset", "cell_prep", "sample_count", "scan", "scatter", "sample", "track", "flux", "update", "movers", "gradients", "flux_o2"]

EXPORTED = ["ugkwp_gks_steps", "ugkwp_average", "ugkwp_average_time", "ugkwp_kn_gll", "ugkwp_adjoint_query", "ugkwp_get_launch_cfg", "ugkwp_set_launch_cfg", "ugkwp_autotune", "ugkwp_batch_create",
            "ugkwp_batch_step", "ugkwp_batch_sync", "ugkwp_batch_autotune", "ugkwp_batch_free",
            "ugkwp_time_step_noalloc", "ugkwp_timing_enable", "ugkwp_timing_read", "ugkwp_mesh_load", "ugkwp_mesh_free", "ugkwp_query_sizes", "ugkwp_init", "ugkwp_free", "ugkwp_step",
            "ugkwp_sync", "ugkwp_moments", "ugkwp_state_info", "ugkwp_export_state", "ugkwp_import_state",
            "ugkwp_export_state_native", "ugkwp_import_state_native",
            "ugkwp_last", "ugkwp_adjoint_wave", "ugkwp_last_error"]

_LIB = None


def library_path() -> str:
    return build_lib.LIB


def lib():
    """Load libugkwp.so (building it in-tree first if it is missing or stale)."""
    global _LIB
    if _LIB is None:
        path = build_lib.build()
        L = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        P = ctypes.POINTER
        sig = {
            "ugkwp_mesh_load": [P(MeshDesc), P(vp)],
            "ugkwp_mesh_free": [vp],
            "ugkwp_query_sizes": [vp, P(Params), P(Sizes)],
            "ugkwp_init": [vp, P(Params), vp, vp, sz, vp, P(vp)],
            "ugkwp_free": [vp],
            "ugkwp_step": [vp, i32, P(Stats)],
            "ugkwp_sync": [vp],
            "ugkwp_moments": [vp, i32, vp, i32],
            "ugkwp_state_info": [vp, P(State)],
            "ugkwp_export_state": [vp, P(State)],
            "ugkwp_import_state": [vp, P(State)],
            "ugkwp_export_state_native": [vp, P(StateNative)],
            "ugkwp_import_state_native": [vp, P(StateNative)],
            "ugkwp_last": [vp, i32, vp],
            "ugkwp_adjoint_wave": [vp, P(AdjointReq), vp],
            "ugkwp_adjoint_query": [vp, i32, P(sz)],
            "ugkwp_last_error": [ctypes.c_char_p, sz],
            "ugkwp_timing_enable": [vp, i32],
            "ugkwp_timing_read": [vp, vp, vp],
            "ugkwp_time_step_noalloc": [vp, vp, vp, i32, ctypes.c_double, ctypes.c_double, vp, vp],
            "ugkwp_get_launch_cfg": [vp, P(LaunchCfg)],
            "ugkwp_gks_steps": [vp, i32, i32, P(Stats)],
            "ugkwp_average": [vp, i32],
            "ugkwp_average_time": [vp, P(ctypes.c_double)],
            "ugkwp_kn_gll": [vp, vp],
            "ugkwp_set_launch_cfg": [vp, P(LaunchCfg)],
            "ugkwp_autotune": [vp, i32, P(LaunchCfg)],
            "ugkwp_batch_create": [vp, i32, vp, P(vp)],
            "ugkwp_batch_step": [vp, i32],
            "ugkwp_batch_sync": [vp],
            "ugkwp_batch_autotune": [vp, i32, P(LaunchCfg)],
            "ugkwp_batch_free": [vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(rc):
    if rc != OK:
        buf = ctypes.create_string_buffer(1024)
        lib().ugkwp_last_error(buf, 1024)
        raise UgkwpError(rc, buf.value.decode(errors="replace"))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def make_params(p: dict) -> Params:
    o = Params()
    for k in ("R", "mu_ref", "T_ref", "omega", "CFL", "C2"):
        setattr(o, k, float(p[k]))
    o.Pr = float(p.get("Pr", 0.0))
    o.venkat_K = float(p.get("venkat_K", 0.0))
    o.order = int(p.get("order", 1))
    o.N_ref = int(p["N_ref"])
    o.N_min = int(p.get("N_min", 0))
    o.precision = PRECISION[p.get("precision", "fp64")]
    o.max_crossings = int(p.get("max_crossings", 1000))
    o.seed = int(p["seed"])
    o.particle_capacity = int(p["particle_capacity"])
    o.n_bc = len(p["bc"])
    o.sampling = SAMPLING[p.get("sampling", "maxwell")]
    o.K = int(p.get("K", 0))
    for k, b in enumerate(p["bc"]):
        c = o.bc[k]
        c.type = BC_TYPES[b["type"]]
        c.T_w = float(b.get("T_w", 0.0))
        for j, v in enumerate(b.get("U_w", (0.0, 0.0, 0.0))):
            c.U_w[j] = float(v)
        for j, v in enumerate(b.get("W_in", (0.0,) * 5)):
            c.W_in[j] = float(v)
    return o


# ------------------------------------------------------------ C-ABI calls
class Mesh:
    """Owner of a ugkwp_mesh handle and of the host arrays it was built from."""

    def __init__(self, mesh: dict):
        self.nodes = np.ascontiguousarray(mesh["nodes"], dtype=np.float64)
        self.tets = np.ascontiguousarray(mesh["tets"], dtype=np.int32)
        self.bfaces = np.ascontiguousarray(mesh["bfaces"], dtype=np.int32)
        self.btags = np.ascontiguousarray(mesh["btags"], dtype=np.int32)
        d = MeshDesc(self.nodes.shape[0], self.tets.shape[0], self.bfaces.shape[0], 0,
                     self.nodes.ctypes.data, self.tets.ctypes.data, self.bfaces.ctypes.data, self.btags.ctypes.data)
        h = ctypes.c_void_p()
        _check(lib().ugkwp_mesh_load(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.ugkwp_mesh_free(self.handle)
            self.handle = None


def ugkwp_mesh_load(mesh: dict) -> Mesh:
    return Mesh(mesh)


def ugkwp_query_sizes(mesh: Mesh, params: dict) -> Sizes:
    P = make_params(params)
    s = Sizes()
    _check(lib().ugkwp_query_sizes(mesh.handle, ctypes.byref(P), ctypes.byref(s)))
    return s


def ugkwp_init(mesh: Mesh, params: dict, W0, d_workspace: int, workspace_bytes: int, stream: int = 0):
    P = make_params(params)
    W0 = np.ascontiguousarray(W0, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib().ugkwp_init(mesh.handle, ctypes.byref(P), _ptr(W0), ctypes.c_void_p(d_workspace),
                            workspace_bytes, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def ugkwp_free(sim):
    _check(lib().ugkwp_free(sim))


def ugkwp_step(sim, n_steps: int = 1, stats: bool = False):
    st = Stats() if stats else None
    _check(lib().ugkwp_step(sim, int(n_steps), ctypes.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def ugkwp_gks_steps(sim, n_steps: int = 1, local_dt: bool = False, stats: bool = False):
    st = Stats() if stats else None
    _check(lib().ugkwp_gks_steps(sim, int(n_steps), 1 if local_dt else 0,
                                 ctypes.byref(st) if st is not None else None))
    return st.as_dict() if st is not None else None


def ugkwp_sync(sim):
    _check(lib().ugkwp_sync(sim))


def ugkwp_moments(sim, which: int, out_ptr: int, out_on_device: bool):
    _check(lib().ugkwp_moments(sim, int(which), ctypes.c_void_p(out_ptr), 1 if out_on_device else 0))


def ugkwp_state_info(sim) -> State:
    st = State()
    _check(lib().ugkwp_state_info(sim, ctypes.byref(st)))
    return st


def ugkwp_export_state(sim, n_cells: int) -> dict:
    info = ugkwp_state_info(sim)
    n = info.n_particles
    out = {"W": np.empty((5, n_cells)), "id": np.empty(n, dtype=np.uint64), "cell": np.empty(n, dtype=np.int32),
           "x": np.empty((3, n)), "u": np.empty((3, n)), "m": np.empty(n), "e": np.empty(n)}
    st = State()
    st.n_particles = n
    for k in ("W", "id", "cell", "x", "u", "m", "e"):
        setattr(st, k, out[k].ctypes.data)
    _check(lib().ugkwp_export_state(sim, ctypes.byref(st)))
    out.update(step=int(st.step), t=float(st.t), exps=np.array(list(st.exps), dtype=np.int64))
    return out


def ugkwp_import_state(sim, state: dict):
    arrs = {"W": np.ascontiguousarray(state["W"], dtype=np.float64),
            "id": np.ascontiguousarray(state["id"], dtype=np.uint64),
            "cell": np.ascontiguousarray(state["cell"], dtype=np.int32),
            "x": np.ascontiguousarray(state["x"], dtype=np.float64),
            "u": np.ascontiguousarray(state["u"], dtype=np.float64),
            "m": np.ascontiguousarray(state["m"], dtype=np.float64)}
    if state.get("e") is not None:
        arrs["e"] = np.ascontiguousarray(state["e"], dtype=np.float64)
    st = State()
    st.n_particles = arrs["id"].size
    st.step = int(state["step"])
    st.t = float(state["t"])
    for q in range(5):
        st.exps[q] = int(state["exps"][q])
    for k, a in arrs.items():
        setattr(st, k, a.ctypes.data)
    _check(lib().ugkwp_import_state(sim, ctypes.byref(st)))


def ugkwp_export_state_native(sim, n_cells: int) -> dict:
    """The native state image (see include/ugkwp.h): x, u, e in the particle
    precision (float32 in MIXED, x the offsets from the tets' anchors)."""
    probe = StateNative()
    probe.n_particles = -1  # too small on purpose: fills the scalar fields only
    rc = lib().ugkwp_export_state_native(sim, ctypes.byref(probe))
    if rc not in (0, E_ARG):
        _check(rc)
    n = probe.n_particles
    dt = np.float32 if probe.real_size == 4 else np.float64
    out = {"W": np.empty((5, n_cells)), "id": np.empty(n, dtype=np.uint64), "cell": np.empty(n, dtype=np.int32),
           "x": np.empty((3, n), dtype=dt), "u": np.empty((3, n), dtype=dt), "m": np.empty(n),
           "e": np.empty(n, dtype=dt)}
    st = StateNative()
    st.n_particles = n
    for k in ("W", "id", "cell", "x", "u", "m", "e"):
        setattr(st, k, out[k].ctypes.data)
    _check(lib().ugkwp_export_state_native(sim, ctypes.byref(st)))
    out.update(step=int(st.step), t=float(st.t), exps=np.array(list(st.exps), dtype=np.int64),
               real_size=int(st.real_size))
    return out


def ugkwp_import_state_native(sim, state: dict):
    dt = np.float32 if int(state["real_size"]) == 4 else np.float64
    arrs = {"W": np.ascontiguousarray(state["W"], dtype=np.float64),
            "id": np.ascontiguousarray(state["id"], dtype=np.uint64),
            "cell": np.ascontiguousarray(state["cell"], dtype=np.int32),
            "x": np.ascontiguousarray(state["x"], dtype=dt),
            "u": np.ascontiguousarray(state["u"], dtype=dt),
            "m": np.ascontiguousarray(state["m"], dtype=np.float64)}
    if state.get("e") is not None:
        arrs["e"] = np.ascontiguousarray(state["e"], dtype=dt)
    st = StateNative()
    st.n_particles = arrs["id"].size
    st.step = int(state["step"])
    st.t = float(state["t"])
    st.real_size = int(state["real_size"])
    for q in range(5):
        st.exps[q] = int(state["exps"][q])
    for k, a in arrs.items():
        setattr(st, k, a.ctypes.data)
    _check(lib().ugkwp_import_state_native(sim, ctypes.byref(st)))


def ugkwp_last(sim, which: str, n_cells: int, n_faces: int):
    code = LAST[which]
    shape, dt = {0: ((1,), np.float64), 1: ((n_cells,), np.float64), 2: ((n_cells,), np.float64),
                 3: ((n_cells,), np.int64), 4: ((n_cells,), np.float64), 5: ((5, n_faces), np.float64),
                 6: ((5, n_cells), np.int64), 7: ((n_cells,), np.int64), 8: ((n_cells,), np.int64),
                 9: ((5, 3, n_cells), np.float64), 10: ((3, n_cells), np.float64)}[code]
    out = np.empty(shape, dtype=dt)
    _check(lib().ugkwp_last(sim, code, out.ctypes.data))
    return float(out[0]) if code == 0 else out


def ugkwp_adjoint_query(sim, n_steps: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().ugkwp_adjoint_query(sim, int(n_steps), ctypes.byref(b)))
    return int(b.value)


def ugkwp_adjoint_wave(sim, functional: int = 0, n_steps: int = 1, wall_tags=(), theta=None, d_workspace: int = 0,
                       workspace_bytes: int = 0):
    """[J, dJ/drho_inf, dJ/dU_inf, dJ/dT_w] of the frozen-particle wave map over
    the next n_steps steps (which the call takes); see include/ugkwp.h."""
    tags = np.ascontiguousarray(wall_tags, dtype=np.int32)
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    req = AdjointReq(int(functional), int(n_steps), tags.ctypes.data if tags.size else None, tags.size, 0,
                     th.ctypes.data if th is not None else None, d_workspace or None, int(workspace_bytes))
    out = np.zeros(4)
    _check(lib().ugkwp_adjoint_wave(sim, ctypes.byref(req), out.ctypes.data))
    return out


def ugkwp_timing_enable(sim, enable: bool = True):
    _check(lib().ugkwp_timing_enable(sim, 1 if enable else 0))


def ugkwp_timing_read(sim):
    """(ms per kernel class, launches per kernel class) as dicts keyed by KERNELS."""
    ms = np.zeros(len(KERNELS))
    n = np.zeros(len(KERNELS), dtype=np.int64)
    _check(lib().ugkwp_timing_read(sim, ms.ctypes.data, n.ctypes.data))
    return dict(zip(KERNELS, ms.tolist())), dict(zip(KERNELS, (int(v) for v in n)))


NOALLOC_MAX_CELLS = 1 << 24


def ugkwp_time_step_noalloc(d_W: int, d_vol: int, d_dS: int, n_cells: int, R: float, CFL: float, d_dt: int,
                            stream: int = 0):
    """Time step from caller-owned device arrays with no device allocation
    (for callers that cannot allocate; see include/ugkwp.h)."""
    _check(lib().ugkwp_time_step_noalloc(ctypes.c_void_p(d_W), ctypes.c_void_p(d_vol), ctypes.c_void_p(d_dS),
                                         int(n_cells), float(R), float(CFL), ctypes.c_void_p(d_dt),
                                         ctypes.c_void_p(stream)))


def ugkwp_average(sim, start: bool = True):
    _check(lib().ugkwp_average(sim, 1 if start else 0))


def ugkwp_average_time(sim) -> float:
    t = ctypes.c_double()
    _check(lib().ugkwp_average_time(sim, ctypes.byref(t)))
    return t.value


def ugkwp_kn_gll(sim, n_cells: int) -> np.ndarray:
    out = np.empty(n_cells)
    _check(lib().ugkwp_kn_gll(sim, out.ctypes.data))
    return out


def ugkwp_get_launch_cfg(sim) -> dict:
    c = LaunchCfg()
    _check(lib().ugkwp_get_launch_cfg(sim, ctypes.byref(c)))
    return c.as_dict()


def ugkwp_set_launch_cfg(sim, particle_blocks: int, wave_blocks: int, track_threads: int = None,
                         smem_carveout: int = None):
    """Set the launch configuration; fields left None keep their current values."""
    cur = ugkwp_get_launch_cfg(sim)
    c = LaunchCfg(int(particle_blocks), int(wave_blocks),
                  int(cur["track_threads"] if track_threads is None else track_threads),
                  int(cur["smem_carveout"] if smem_carveout is None else smem_carveout))
    _check(lib().ugkwp_set_launch_cfg(sim, ctypes.byref(c)))


def ugkwp_autotune(sim, steps_per_trial: int = 2) -> dict:
    c = LaunchCfg()
    _check(lib().ugkwp_autotune(sim, int(steps_per_trial), ctypes.byref(c)))
    return c.as_dict()


def ugkwp_batch_create(handles, stream: int):
    arr = (ctypes.c_void_p * len(handles))(*handles)
    out = ctypes.c_void_p()
    _check(lib().ugkwp_batch_create(arr, len(handles), ctypes.c_void_p(stream), ctypes.byref(out)))
    return out


def ugkwp_batch_step(batch, n: int):
    _check(lib().ugkwp_batch_step(batch, int(n)))


def ugkwp_batch_sync(batch):
    _check(lib().ugkwp_batch_sync(batch))


def ugkwp_batch_autotune(batch, steps_per_trial: int = 2) -> dict:
    c = LaunchCfg()
    _check(lib().ugkwp_batch_autotune(batch, int(steps_per_trial), ctypes.byref(c)))
    return c.as_dict()


def ugkwp_batch_free(batch):
    _check(lib().ugkwp_batch_free(batch))


# ------------------------------------------------------------ convenience
class Simulation:
    """A UGKWP simulation on one GPU: workspace from the PyTorch allocator,
    work enqueued on a PyTorch stream (the current one by default; a stream of
    its own, e.g. torch.cuda.Stream(), steps faster than the legacy default
    stream, with which the step's concurrent kernels serialise in part)."""

    def __init__(self, mesh: dict, W0, params: dict, device: str = "cuda", stream=None):
        import torch
        self.params = dict(params)
        self.mesh = ugkwp_mesh_load(mesh)
        sizes = ugkwp_query_sizes(self.mesh, params)
        self.n_cells, self.n_faces = int(sizes.n_cells), int(sizes.n_faces)
        self.n_bfaces = int(sizes.n_bfaces)
        self.workspace_bytes = int(sizes.workspace_bytes)
        self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=device)
        base = self._ws.data_ptr()
        self.d_workspace = (base + 255) // 256 * 256
        self.device = self._ws.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.handle = ugkwp_init(self.mesh, params, W0, self.d_workspace, self.workspace_bytes,
                                 self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            ugkwp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1, stats: bool = False):
        return ugkwp_step(self.handle, n, stats)

    def gks_steps(self, n: int = 1, local_dt: bool = False, stats: bool = False):
        """n start-up steps of the gas-kinetic scheme (no particles)."""
        return ugkwp_gks_steps(self.handle, n, local_dt, stats)

    def sync(self):
        ugkwp_sync(self.handle)

    def moments(self, which: int = W, out=None):
        """[5, n_cells] float64: a torch tensor on the device if `out` is one,
        else a numpy array (synchronising)."""
        if out is not None:
            ugkwp_moments(self.handle, which, out.data_ptr(), True)
            return out
        host = np.empty((5, self.n_cells))
        ugkwp_moments(self.handle, which, host.ctypes.data, False)
        return host

    def state(self):
        return ugkwp_export_state(self.handle, self.n_cells)

    def set_state(self, st: dict):
        ugkwp_import_state(self.handle, st)

    def state_native(self):
        """The native image (checkpoint of this mesh and precision)."""
        return ugkwp_export_state_native(self.handle, self.n_cells)

    def set_state_native(self, st: dict):
        ugkwp_import_state_native(self.handle, st)

    def last(self, which: str):
        return ugkwp_last(self.handle, which, self.n_cells, self.n_faces)

    def adjoint(self, functional: int, n_steps: int, wall_tags, theta=None):
        """[J, dJ/dtheta] of the frozen-particle wave map over the next n_steps
        steps (taken by the call); the scratch comes from the PyTorch allocator."""
        import torch
        nb = ugkwp_adjoint_query(self.handle, n_steps)
        ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        base = (ws.data_ptr() + 255) // 256 * 256
        out = ugkwp_adjoint_wave(self.handle, functional, n_steps, wall_tags, theta, base, nb)
        del ws
        return out


class Batch:
    """Independent simulations stepped together, one CUDA graph per step pair
    launched on `stream` (a new PyTorch stream by default).  Members keep their
    own results; read them after sync()."""

    def __init__(self, sims, stream=None):
        import torch
        self.sims = list(sims)
        dev = self.sims[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.handle = ugkwp_batch_create([s.handle for s in self.sims], self.stream.cuda_stream)

    def step(self, n: int = 1):
        ugkwp_batch_step(self.handle, n)

    def sync(self):
        ugkwp_batch_sync(self.handle)

    def autotune(self, steps_per_trial: int = 2) -> dict:
        return ugkwp_batch_autotune(self.handle, steps_per_trial)

    def close(self):
        if getattr(self, "handle", None):
            ugkwp_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wall_functional(theta, sim: Simulation, functional: int, n_steps: int, wall_tags):
    """J(theta) as a differentiable PyTorch scalar: the forward runs the
    adjoint call (taking n_steps steps of `sim`), the backward returns its
    hand-written reverse-sweep gradient."""
    import torch

    class _WallFunctional(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            out = sim.adjoint(functional, n_steps, wall_tags, th.detach().double().cpu().numpy())
            ctx.save_for_backward(torch.tensor(out[1:], dtype=th.dtype, device=th.device))
            return torch.tensor(out[0], dtype=th.dtype, device=th.device)

        @staticmethod
        def backward(ctx, gJ):
            (g,) = ctx.saved_tensors
            return gJ * g

    return _WallFunctional.apply(theta)
