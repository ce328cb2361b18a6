"""Python handle on the CPU oracle of the UGKWP step (arXiv 2007.13091, Sec. 2).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package; the product package
``paper_2007_13091_gb300`` never does, and this package never imports it.

Inputs (mesh, initial state, parameters) come as plain dicts and arrays from
the seeded workload generators; nothing here reads the product's code.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

BC_TYPES = {"wall": 1, "specular": 2, "inflow": 3, "farfield": 3, "outflow": 4}
PRECISION = {"fp64": 0, "mixed": 1}


class OrcBc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("pad_", ctypes.c_int32), ("T_w", ctypes.c_double),
                ("U_w", ctypes.c_double * 3), ("W_in", ctypes.c_double * 5)]


class OrcParams(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("mu_ref", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("omega", ctypes.c_double), ("CFL", ctypes.c_double), ("C2", ctypes.c_double),
                ("venkat_K", ctypes.c_double), ("Pr", ctypes.c_double), ("order", ctypes.c_int32), ("N_ref", ctypes.c_int32), ("N_min", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_crossings", ctypes.c_int32),
                ("n_bc", ctypes.c_int32), ("sampling", ctypes.c_int32), ("K", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("bc", OrcBc * 16)]


_LIB = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i32, i64, u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        vp, cp = ctypes.c_void_p, ctypes.c_char_p
        L.orc_math_d.argtypes = [ctypes.c_int, vp, vp, i64]
        L.orc_math_logf.argtypes = [vp, vp, i64]
        L.orc_philox32.argtypes = [vp, vp, vp]
        L.orc_math_sincos2pi_f.argtypes = [vp, vp, vp, i64]
        L.orc_philox.argtypes = [vp, vp, vp]
        L.orc_qcoef.argtypes = [d, d, vp]
        L.orc_maxwell_moments.argtypes = [vp, d, vp, ctypes.c_int, i32, vp, vp]
        L.orc_face_flux.argtypes = [P(OrcParams), ctypes.c_int, vp, d, vp, d, vp, d, d, P(OrcBc), i32, vp]
        L.orc_create.argtypes = [P(OrcParams), i32, vp, i32, vp, i32, vp, vp, vp, cp, i32]
        L.orc_create.restype = vp
        L.orc_free.argtypes = [vp]
        L.orc_step.argtypes = [vp, cp, i32]
        L.orc_gks_step.argtypes = [vp, i32, cp, i32]
        L.orc_sizes.argtypes = [vp, vp]
        L.orc_geometry.argtypes = [vp, ctypes.c_int, vp]
        L.orc_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_set_state.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, d, vp, cp, i32]
        L.orc_last.argtypes = [vp, ctypes.c_int, vp]
        L.orc_track_one.argtypes = [vp, u64, i32, vp, vp, vp, d, d, i64, vp, vp]
        L.orc_prepare.argtypes = [vp, cp, i32]
        L.orc_gradients.argtypes = [vp, ctypes.c_int, vp, vp]
        L.orc_slope_moment.argtypes = [vp, d, ctypes.c_int, i32, vp, ctypes.c_int, vp]
        L.orc_micro_slope.argtypes = [vp, d, i32, vp, vp]
        L.orc_face_flux_o2.argtypes = [P(OrcParams), vp, d, vp, vp, vp, vp, d, vp, vp, vp, vp, d, i32, vp]
        L.orc_frozen_objective.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, vp, i32, vp]
        L.orc_frozen_value.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, vp, i32, vp]
        L.orc_frozen_o2_value.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, vp, i32, vp, i32, vp]
        L.orc_sample_cell.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp]
        L.orc_sample_cell.restype = i64
        L.orc_gp_coefficients.argtypes = [vp, i32, vp]
        L.orc_gp_draw.argtypes = [i32, u64, u64, vp, u64, i64, vp]
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_bc(b: dict) -> OrcBc:
    c = OrcBc()
    c.type = BC_TYPES[b["type"]]
    c.T_w = float(b.get("T_w", 0.0))
    for k, v in enumerate(b.get("U_w", (0.0, 0.0, 0.0))):
        c.U_w[k] = float(v)
    for k, v in enumerate(b.get("W_in", (0.0,) * 5)):
        c.W_in[k] = float(v)
    return c


SAMPLING = {"maxwell": 0, "energy_matched": 1, "gp1": 2}


def make_params(p: dict) -> OrcParams:
    o = OrcParams()
    for k in ("R", "mu_ref", "T_ref", "omega", "CFL", "C2"):
        setattr(o, k, float(p[k]))
    o.venkat_K = float(p.get("venkat_K", 5.0))
    o.Pr = float(p.get("Pr", 0.0))
    o.order = int(p.get("order", 1))
    o.N_ref = int(p["N_ref"])
    o.N_min = int(p.get("N_min", 0))
    o.precision = PRECISION[p.get("precision", "fp64")]
    o.max_crossings = int(p.get("max_crossings", 1000))
    o.sampling = SAMPLING[p.get("sampling", "maxwell")]
    o.K = int(p.get("K", 0))
    o.seed = int(p["seed"])
    o.n_bc = len(p["bc"])
    for k, b in enumerate(p["bc"]):
        o.bc[k] = make_bc(b)
    return o


# ------------------------------------------------------------------ pins API
def math_d(which: str, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    code = {"exp": 0, "log": 1, "sin2pi": 2, "cos2pi": 3}[which]
    lib().orc_math_d(code, _ptr(x), _ptr(y), x.size)
    return y


def logf(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().orc_math_logf(_ptr(x), _ptr(y), x.size)
    return y


def sincos2pi_f(x):
    """(sin 2 pi x, cos 2 pi x) in binary32, as the mixed-mode particles use them."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    sn = np.empty_like(x)
    cs = np.empty_like(x)
    lib().orc_math_sincos2pi_f(_ptr(x), _ptr(sn), _ptr(cs), x.size)
    return sn, cs


def philox32(ctr, key):
    """Philox4x32-10 of one counter (4 x uint32) and key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox32(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def qcoef(dt: float, tau: float):
    q = np.empty(7)
    lib().orc_qcoef(float(dt), float(tau), _ptr(q))
    return q


def maxwell_moments(U, lam, n, half, K=0):
    U = np.ascontiguousarray(U, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    H = np.empty(5)
    G = np.empty(5)
    lib().orc_maxwell_moments(_ptr(U), float(lam), _ptr(n), int(half), int(K), _ptr(H), _ptr(G))
    return H, G


def face_flux(params: dict, kind: str, WL, rhohL, WR, rhohR, n, dt, tau_wall=0.0, bc=None, gks=False):
    """kind: 'interior' or a boundary type name; WR is ignored for boundaries.
    gks: the flux of a step without particles (whole free transport in the wave)."""
    P = make_params(params)
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR if WR is not None else WL, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    F = np.empty(5)
    kcode = 0 if kind == "interior" else BC_TYPES[kind]
    if bc is None and kind != "interior":
        bc = {"type": kind}
    bcs = make_bc(bc) if bc is not None else None
    rc = lib().orc_face_flux(ctypes.byref(P), kcode, _ptr(WL), float(rhohL), _ptr(WR), float(rhohR),
                             _ptr(n), float(dt), float(tau_wall),
                             ctypes.byref(bcs) if bcs is not None else None, int(bool(gks)), _ptr(F))
    if rc:
        raise ValueError("orc_face_flux failed")
    return F


def slope_moment(U, lam, half, a, d, K=0):
    """int u_n u_d (a . psi) psi g du for a unit-density Maxwellian in a face
    frame (components of U and a along n, t1, t2)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty(5)
    lib().orc_slope_moment(_ptr(U), float(lam), int(half), int(K), _ptr(a), int(d), _ptr(out))
    return out


def micro_slope(U, lam, b, K=0):
    U = np.ascontiguousarray(U, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    a = np.empty(5)
    lib().orc_micro_slope(_ptr(U), float(lam), int(K), _ptr(b), _ptr(a))
    return a


def face_flux_o2(params, WL, rhohL, gWL, gHL, dxL, WR, rhohR, gWR, gHR, dxR, n, dt, gks=False):
    """Second-order flux of one interior face; gW are [5][3] gradients."""
    P = make_params(params)
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (WL, gWL, gHL, dxL, WR, gWR, gHR, dxR, n)]
    F = np.empty(5)
    lib().orc_face_flux_o2(ctypes.byref(P), _ptr(arrs[0]), float(rhohL), _ptr(arrs[1]), _ptr(arrs[2]),
                           _ptr(arrs[3]), _ptr(arrs[4]), float(rhohR), _ptr(arrs[5]), _ptr(arrs[6]),
                           _ptr(arrs[7]), _ptr(arrs[8]), float(dt), int(bool(gks)), _ptr(F))
    return F


def gp_draw(coef, n, id0=0, step=1, seed=1, precision="fp64"):
    """n first-order g_p draws X [3, n] for the acceptance polynomial `coef`."""
    c = np.ascontiguousarray(coef, dtype=np.float64)
    X = np.empty((n, 3))
    lib().orc_gp_draw(PRECISION[precision], int(seed), int(step), _ptr(c), int(id0), int(n), _ptr(X))
    return X.T.copy()


# ------------------------------------------------------------- simulation
class OracleSim:
    """One oracle simulation: mesh + parameters + state, stepped on the CPU."""

    def __init__(self, mesh: dict, W0, params: dict):
        L = lib()
        self.params = params
        self._P = make_params(params)
        nodes = np.ascontiguousarray(mesh["nodes"], dtype=np.float64)
        tets = np.ascontiguousarray(mesh["tets"], dtype=np.int32)
        bf = np.ascontiguousarray(mesh["bfaces"], dtype=np.int32)
        bt = np.ascontiguousarray(mesh["btags"], dtype=np.int32)
        W0 = np.ascontiguousarray(W0, dtype=np.float64)
        if W0.shape != (5, tets.shape[0]):
            raise ValueError("W0 must be [5, n_tets]")
        err = ctypes.create_string_buffer(512)
        h = L.orc_create(ctypes.byref(self._P), nodes.shape[0], _ptr(nodes), tets.shape[0], _ptr(tets),
                         bf.shape[0], _ptr(bf), _ptr(bt), _ptr(W0), err, 512)
        if not h:
            raise ValueError("oracle: " + err.value.decode())
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    def sizes(self):
        out = np.zeros(5, dtype=np.int64)
        lib().orc_sizes(self._h, _ptr(out))
        return {"n_cells": int(out[0]), "n_faces": int(out[1]), "n_bfaces": int(out[2]),
                "n_particles": int(out[3]), "step": int(out[4])}

    def step(self, n: int = 1):
        err = ctypes.create_string_buffer(512)
        for _ in range(n):
            rc = lib().orc_step(self._h, err, 512)
            if rc:
                raise RuntimeError(f"oracle step failed ({rc}): {err.value.decode()}")

    def gks_step(self, n: int = 1, local: bool = False):
        """n steps of the gas-kinetic scheme (no particles), with the global or
        local time steps."""
        err = ctypes.create_string_buffer(512)
        for _ in range(n):
            rc = lib().orc_gks_step(self._h, int(bool(local)), err, 512)
            if rc:
                raise RuntimeError(f"oracle GKS step failed ({rc}): {err.value.decode()}")

    def geometry(self, which: str):
        s = self.sizes()
        nc, nf = s["n_cells"], s["n_faces"]
        code, shape = {"vol": (0, (nc,)), "centroid": (1, (3, nc)), "face_normal": (2, (3, nf)),
                       "face_area": (3, (nf,)), "face_owner": (4, (nf,)), "face_nbr": (5, (nf,)),
                       "dS": (6, (3, nc)), "face_d": (7, (nf,))}[which]
        out = np.empty(shape)
        lib().orc_geometry(self._h, code, _ptr(out))
        return out

    def state(self):
        s = self.sizes()
        nc, n = s["n_cells"], s["n_particles"]
        W = np.empty((5, nc))
        pid = np.empty(n, dtype=np.uint64)
        cell = np.empty(n, dtype=np.int32)
        x = np.empty((3, n))
        u = np.empty((3, n))
        m = np.empty(n)
        e = np.empty(n)
        scal = np.empty(6, dtype=np.int64)
        t = ctypes.c_double()
        lib().orc_get_state(self._h, _ptr(W), _ptr(pid), _ptr(cell), _ptr(x), _ptr(u), _ptr(m),
                            _ptr(scal), ctypes.byref(t), _ptr(e))
        return {"W": W, "id": pid, "cell": cell, "x": x, "u": u, "m": m, "e": e,
                "step": int(scal[0]), "exps": scal[1:].copy(), "t": t.value}

    def set_state(self, st: dict):
        W = np.ascontiguousarray(st["W"], dtype=np.float64)
        pid = np.ascontiguousarray(st["id"], dtype=np.uint64)
        cell = np.ascontiguousarray(st["cell"], dtype=np.int32)
        x = np.ascontiguousarray(st["x"], dtype=np.float64)
        u = np.ascontiguousarray(st["u"], dtype=np.float64)
        m = np.ascontiguousarray(st["m"], dtype=np.float64)
        scal = np.ascontiguousarray([st["step"], *st["exps"]], dtype=np.int64)
        e = st.get("e")
        e = None if e is None else np.ascontiguousarray(e, dtype=np.float64)
        err = ctypes.create_string_buffer(512)
        rc = lib().orc_set_state(self._h, _ptr(W), pid.size, _ptr(pid), _ptr(cell), _ptr(x), _ptr(u),
                                 _ptr(m), _ptr(scal), float(st["t"]), _ptr(e) if e is not None else None, err, 512)
        if rc:
            raise ValueError("oracle set_state: " + err.value.decode())

    def last(self, which: str):
        s = self.sizes()
        nc, nf = s["n_cells"], s["n_faces"]
        code, shape, dt = {"dt": (0, (1,), np.float64), "tau": (1, (nc,), np.float64),
                           "rho_h": (2, (nc,), np.float64), "n_sam": (3, (nc,), np.int64),
                           "m_sam": (4, (nc,), np.float64), "flux": (5, (5, nf), np.float64),
                           "pflux": (6, (5, nc), np.int64), "surv_mass": (7, (nc,), np.int64),
                           "surv_count": (8, (nc,), np.int64), "counters": (9, (7,), np.int64)}[which]
        out = np.empty(shape, dtype=dt)
        lib().orc_last(self._h, code, _ptr(out))
        if which == "dt":
            return float(out[0])
        if which == "counters":
            keys = ["n_tracked", "n_collided", "n_exited", "n_lost", "n_crossings", "n_wall_hits", "n_sampled"]
            return dict(zip(keys, (int(v) for v in out)))
        return out

    def record_frozen(self, K):
        """Take K steps, recording what the frozen-particle wave map needs:
        (W0, dt[K], rho_p[K][nc], pflux[K][5][nc] scaled to conservative units)."""
        st = self.state()
        W0 = st["W"].copy()
        e = st["exps"]
        nc = W0.shape[1]
        vol = self.geometry("vol")
        dt, rho_p, pf = [], [], []
        for _ in range(K):
            W = self.state()["W"]
            self.step()
            dt.append(self.last("dt"))
            rho_p.append(W[0] - self.last("rho_h"))
            q = self.last("pflux").astype(np.float64)
            pf.append(np.stack([np.ldexp(q[c], int(e[c])) for c in range(5)]))
        return W0, np.array(dt), np.array(rho_p).reshape(K, nc), np.array(pf).reshape(K, 5, nc)

    def frozen_objective(self, frozen, theta, functional=0, tags=(), grad=True):
        """J (and dJ/dtheta by dual numbers) of the frozen-particle wave map."""
        W0, dt, rho_p, pf = (np.ascontiguousarray(a, dtype=np.float64) for a in frozen)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        tg = np.ascontiguousarray(tags, dtype=np.int32)
        out = np.zeros(4)
        fn = lib().orc_frozen_objective if grad else lib().orc_frozen_value
        rc = fn(self._h, len(dt), _ptr(W0), _ptr(dt), _ptr(rho_p), _ptr(pf), _ptr(th), int(functional),
                _ptr(tg) if tg.size else None, tg.size, _ptr(out))
        if rc:
            raise RuntimeError("oracle frozen objective failed")
        return out if grad else float(out[0])

    def frozen_o2(self, frozen, theta, functional=0, tags=(), phi=None):
        """J of the second-order frozen-particle wave map and the limiter values
        phi [K][6][nc]: computed at theta (and returned) when phi is None, else
        taken as given (the limiter frozen)."""
        W0, dt, rho_p, pf = (np.ascontiguousarray(a, dtype=np.float64) for a in frozen)
        nc = W0.shape[1]
        th = np.ascontiguousarray(theta, dtype=np.float64)
        tg = np.ascontiguousarray(tags, dtype=np.int32)
        record = phi is None
        ph = np.zeros((len(dt), 6, nc)) if record else np.ascontiguousarray(phi, dtype=np.float64).copy()
        out = np.zeros(1)
        rc = lib().orc_frozen_o2_value(self._h, len(dt), _ptr(W0), _ptr(dt), _ptr(rho_p), _ptr(pf), _ptr(th),
                                       int(functional), _ptr(tg) if tg.size else None, tg.size, _ptr(ph),
                                       int(record), _ptr(out))
        if rc:
            raise RuntimeError("oracle second-order frozen map failed")
        return float(out[0]), ph

    def frozen_o2_gradient(self, frozen, theta, functional=0, tags=(), rel_step=1e-5):
        """[J, dJ/dtheta] of the second-order frozen map: the limiter frozen at
        theta, derivatives by central differences with steps rel_step * theta."""
        th = np.asarray(theta, dtype=np.float64)
        J, phi = self.frozen_o2(frozen, th, functional, tags)
        out = [J]
        for k in range(3):
            h = rel_step * th[k]
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            out.append((self.frozen_o2(frozen, tp, functional, tags, phi)[0] -
                        self.frozen_o2(frozen, tm, functional, tags, phi)[0]) / (2.0 * h))
        return np.array(out)

    def prepare(self):
        """Primitives, tau, rho^h, dt and sampling counts of the current state
        (readable through last()), without stepping."""
        err = ctypes.create_string_buffer(512)
        rc = lib().orc_prepare(self._h, err, 512)
        if rc:
            raise RuntimeError(f"oracle prepare failed ({rc}): {err.value.decode()}")

    def sample_cell(self, cell):
        """The particles `cell` samples at the current step (after prepare())."""
        n = lib().orc_sample_cell(self._h, int(cell), 0, None, None, None, None, None)
        pid = np.empty(n, dtype=np.uint64)
        x = np.empty((n, 3))
        u = np.empty((n, 3))
        m = np.empty(n)
        e = np.empty(n)
        lib().orc_sample_cell(self._h, int(cell), n, _ptr(pid), _ptr(x), _ptr(u), _ptr(m), _ptr(e))
        return {"id": pid, "x": x.T.copy(), "u": u.T.copy(), "m": m, "e": e}

    def gp_coefficients(self, cell):
        """First-order g_p sampling: the cell's acceptance polynomial and bound
        [a0, L(3), Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, C(3), M] (after prepare())."""
        out = np.empty(14)
        if lib().orc_gp_coefficients(self._h, int(cell), _ptr(out)):
            raise ValueError("no first-order g_p coefficients (sampling 'gp1' and prepare() needed)")
        return out

    def gradients(self, limited=True):
        """Least-squares gradients of W [5, 3, nc] and rho^h [3, nc] of the current
        state (limited with Venkatakrishnan's limiter if `limited`)."""
        nc = self.sizes()["n_cells"]
        gW = np.empty((5, 3, nc))
        gH = np.empty((3, nc))
        rc = lib().orc_gradients(self._h, 1 if limited else 0, _ptr(gW), _ptr(gH))
        if rc:
            raise RuntimeError("oracle gradients failed")
        return gW, gH

    def track_one(self, pid, cell, x, u, tau_cell, dt, step, e=0.0):
        io_x = np.ascontiguousarray(x, dtype=np.float64).copy()
        io_u = np.ascontiguousarray(u, dtype=np.float64).copy()
        io_e = ctypes.c_double(float(e))
        c_out = ctypes.c_int32()
        nc = ctypes.c_int32()
        st = lib().orc_track_one(self._h, int(pid), int(cell), _ptr(io_x), _ptr(io_u), ctypes.byref(io_e),
                                 float(tau_cell), float(dt), int(step), ctypes.byref(c_out), ctypes.byref(nc))
        return {"status": int(st), "cell": int(c_out.value), "x": io_x, "u": io_u, "e": io_e.value,
                "ncross": int(nc.value)}
