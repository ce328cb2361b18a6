"""Pins of the oracle's second-order reconstruction and flux (Sec. 2.1, 2.3).

* least-squares gradients reproduce linear fields exactly (jittered mesh);
* Venkatakrishnan's limiter keeps face values within the neighbour extrema
  (epsilon = 0) and leaves gradients untouched as epsilon grows;
* slope moments int u_n u_d (a.psi) psi g and the micro-slope solve of the
  moment system against direct quadrature;
* the Chapman-Enskog limit (tau << dt): shear stress -mu dw/dx dt and heat
  flux -5/2 R mu dT/dx dt with mu = tau p (BGK, Pr = 1);
* zero gradients give the first-order flux; at equal resolution the
  second-order scheme is closer to the exact Sod solution;
* Prandtl-number fix: for any uniform velocity and pressure with a
  temperature gradient, the energy flux of the equilibrium part is exactly
  q2 (5/2) p R dT/dn / Pr (the Chapman-Enskog heat flux of the BGK model with
  the conductivity scaled by 1/Pr), and shear alone is left untouched.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import workloads as wl
from tests import riemann_exact

PARAMS = {"R": 1.0, "mu_ref": 0.05, "T_ref": 1.0, "omega": 0.81, "CFL": 0.5, "C2": 0.0, "order": 2,
          "venkat_K": 5.0, "N_ref": 10, "seed": 1, "bc": []}


def _interior_cells(tets, bfaces):
    bnodes = set(np.unique(bfaces).tolist())
    return np.array([i for i, t in enumerate(tets) if not (set(t.tolist()) & bnodes)])


def test_lsq_gradient_exact_for_linear_fields():
    cfg = wl.uniform_box(n=(4, 4, 4), jitter_amount=0.25, seed=3, Kn=1e-9, bc_type="outflow")
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    cen = nodes[tets].mean(1)
    G = np.array([[0.1, -0.2, 0.05], [0.02, 0.01, -0.03], [-0.01, 0.03, 0.02], [0.0, 0.01, 0.01], [0.3, 0.1, -0.2]])
    base = np.array([1.0, 0.1, -0.05, 0.02, 2.0])
    W0 = base[:, None] + G @ cen.T
    params = dict(cfg["params"], order=2)
    s = oracle.OracleSim(cfg["mesh"], W0, params)
    gW, gH = s.gradients(limited=False)
    inner = _interior_cells(tets, cfg["mesh"]["bfaces"])
    assert len(inner) > 20
    for q in range(5):
        for d in range(3):
            np.testing.assert_allclose(gW[q, d, inner], G[q, d], rtol=0, atol=1e-12)
    np.testing.assert_allclose(gH[:, inner], np.broadcast_to(G[0][:, None], gH[:, inner].shape), atol=1e-12)


def test_limiter_bounds_and_relaxation():
    cfg = wl.uniform_box(n=(4, 4, 4), jitter_amount=0.2, seed=4, Kn=1e-9, bc_type="outflow")
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    cen = nodes[tets].mean(1)
    rng = np.random.default_rng(5)
    W0 = np.array([1.0, 0.0, 0.0, 0.0, 1.5])[:, None] * np.ones(len(tets))
    W0[0] += 0.2 * rng.random(len(tets))      # rough density field
    W0[4] += 0.3 * np.sin(4 * cen[:, 0])
    s0 = oracle.OracleSim(cfg["mesh"], W0, dict(cfg["params"], order=2, venkat_K=0.0))
    gW, _ = s0.gradients(limited=True)
    own = s0.geometry("face_owner").astype(int)
    nb = s0.geometry("face_nbr").astype(int)
    # neighbour extrema and face centroids per cell
    nc = len(tets)
    vmax = W0.copy()
    vmin = W0.copy()
    for f in range(len(own)):
        if nb[f] >= 0:
            a, b = own[f], nb[f]
            vmax[:, a] = np.maximum(vmax[:, a], W0[:, b]); vmin[:, a] = np.minimum(vmin[:, a], W0[:, b])
            vmax[:, b] = np.maximum(vmax[:, b], W0[:, a]); vmin[:, b] = np.minimum(vmin[:, b], W0[:, a])
    inner = _interior_cells(tets, cfg["mesh"]["bfaces"])
    faces = [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]
    for i in inner:
        for k in range(4):
            xf = nodes[tets[i][faces[k]]].mean(0)
            for q in (0, 4):
                v = W0[q, i] + gW[q, :, i] @ (xf - cen[i])
                assert vmin[q, i] - 1e-12 <= v <= vmax[q, i] + 1e-12
    # a large epsilon switches the limiter off
    s1 = oracle.OracleSim(cfg["mesh"], W0, dict(cfg["params"], order=2, venkat_K=1e6))
    g1, _ = s1.gradients(limited=True)
    g2, _ = s1.gradients(limited=False)
    np.testing.assert_allclose(g1, g2, rtol=1e-6, atol=1e-12)


def _quad_frame(U, lam, half, fun):
    """int fun(u, v, w) g du dv dw for the unit Maxwellian in a face frame:
    Gauss-Hermite in v, w (exact for the polynomial weights), adaptive in u."""
    from scipy.integrate import quad
    xg, wg = np.polynomial.hermite.hermgauss(8)
    s = 1.0 / math.sqrt(lam)
    lo, hi = {1: (0.0, np.inf), -1: (-np.inf, 0.0), 0: (-np.inf, np.inf)}[half]
    tot = np.zeros(5)
    for xa, wa in zip(xg, wg):
        for xb, wb in zip(xg, wg):
            v, w = U[1] + s * xa, U[2] + s * xb
            for k in range(5):
                def integrand(u):
                    return math.sqrt(lam / math.pi) * math.exp(-lam * (u - U[0]) ** 2) * fun(u, v, w)[k]
                tot[k] += wa * wb / math.pi * quad(integrand, lo, hi, epsabs=1e-14, epsrel=1e-12)[0]
    return tot


def _psi(u, v, w):
    return np.array([1.0, u, v, w, 0.5 * (u * u + v * v + w * w)])


@pytest.mark.parametrize("half", [1, -1, 0])
def test_slope_moments_against_quadrature(half):
    rng = np.random.default_rng(20 + half)
    U = rng.normal(size=3) * 0.7
    lam = rng.uniform(0.4, 1.5)
    a = rng.normal(size=5)
    for d in range(3):
        got = oracle.slope_moment(U, lam, half, a, d)
        ref = _quad_frame(U, lam, half, lambda u, v, w: u * (u, v, w)[d] * (a @ _psi(u, v, w)) * _psi(u, v, w))
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-11)


def test_micro_slope_solves_the_moment_system():
    rng = np.random.default_rng(8)
    U = rng.normal(size=3)
    lam = 0.8
    M = np.zeros((5, 5))
    for c in range(5):
        e = np.zeros(5); e[c] = 1.0
        M[:, c] = _quad_frame(U, lam, 0, lambda u, v, w: _psi(u, v, w) * (e @ _psi(u, v, w)))
    b = rng.normal(size=5)
    np.testing.assert_allclose(oracle.micro_slope(U, lam, b), np.linalg.solve(M, b), rtol=1e-9, atol=1e-10)


def _W(rho, U, p):
    U = np.asarray(U, float)
    return np.concatenate([[rho], rho * U, [0.5 * rho * U.dot(U) + 1.5 * p]])


def test_navier_stokes_shear_stress_limit():
    rho, p, gam = 1.0, 1.0, 0.05
    dt = 1.0
    tau = 1e-3 * dt
    params = dict(PARAMS, mu_ref=tau * p)  # T = T_ref = 1: tau = mu_ref / p
    W = _W(rho, (0.0, 0.0, 0.0), p)
    gW = np.zeros((5, 3)); gW[3, 0] = rho * gam  # d(rho w)/dx
    z = np.zeros(3)
    F = oracle.face_flux_o2(params, W, rho, gW, gW[0], z, W, rho, gW, gW[0], z, [1.0, 0.0, 0.0], dt)
    assert F[3] == pytest.approx(-tau * p * gam * dt, rel=3e-3)
    assert abs(F[0]) < 1e-12 and abs(F[4]) < 1e-12


def test_navier_stokes_heat_flux_limit():
    rho, T, gam = 1.0, 1.0, 0.04
    p = rho * T
    dt = 1.0
    tau = 1e-3 * dt
    params = dict(PARAMS, mu_ref=tau * p)
    W = _W(rho, (0.0, 0.0, 0.0), p)
    gW = np.zeros((5, 3)); gW[0, 0] = -rho * gam / T  # constant pressure, dT/dx = gam
    z = np.zeros(3)
    F = oracle.face_flux_o2(params, W, rho, gW, gW[0], z, W, rho, gW, gW[0], z, [1.0, 0.0, 0.0], dt)
    mu = tau * p
    assert F[4] == pytest.approx(-2.5 * 1.0 * mu * gam * dt, rel=3e-3)


@pytest.mark.parametrize("tau", [1e-4, 1e-2, 1.0])
def test_prandtl_fix_heat_flux_closed_form(tau):
    """rho^h = 0 leaves the equilibrium part alone.  With p and U uniform and T
    varying, g_t = -(U.grad) g, and the heat flux relative to U0 of
    q2 u.g_x + q3 g_t is q2 (5/2) p R dT/dn whatever U (the odd moments drop);
    the fix multiplies it by 1/Pr and changes nothing else."""
    rng = np.random.default_rng(int(1e4 * tau) + 3)
    Rg, rho, T = 1.0, 1.3, 0.9
    p = rho * Rg * T
    dt = 0.01
    n = rng.normal(size=3); n /= np.linalg.norm(n)
    U = rng.normal(size=3) * 0.4
    gT = rng.normal(size=3) * 0.05
    grho = -rho * gT / T  # uniform pressure
    gW = np.zeros((5, 3))
    gW[0] = grho
    for c in range(3):
        gW[1 + c] = U[c] * grho
    gW[4] = 0.5 * U.dot(U) * grho
    W = _W(rho, U, p)
    z = np.zeros(3)
    params = dict(PARAMS, R=Rg, mu_ref=tau * p / T ** PARAMS["omega"])
    q2 = oracle.qcoef(dt, tau)[1]
    ref = None
    for Pr in (1.0, 2.0 / 3.0, 0.72):
        F = oracle.face_flux_o2(dict(params, Pr=Pr), W, 0.0, gW, z, z, W, 0.0, gW, z, z, n, dt)
        if ref is None:
            ref = F
            continue
        np.testing.assert_array_equal(F[:4], ref[:4])
        assert F[4] - ref[4] == pytest.approx((1.0 / Pr - 1.0) * q2 * 2.5 * p * Rg * gT.dot(n), rel=1e-9)
    # at rest the whole energy flux is the heat flux
    W0 = _W(rho, (0.0, 0.0, 0.0), p)
    g0 = np.zeros((5, 3)); g0[0] = grho
    for Pr in (1.0, 2.0 / 3.0):
        F = oracle.face_flux_o2(dict(params, Pr=Pr), W0, 0.0, g0, z, z, W0, 0.0, g0, z, z, n, dt)
        assert F[4] == pytest.approx(q2 * 2.5 * p * Rg * gT.dot(n) / Pr, rel=1e-11)


def test_prandtl_fix_leaves_shear_and_uniform_states():
    rho, p, gam, dt = 1.0, 1.0, 0.05, 0.01
    W = _W(rho, (0.0, 0.0, 0.0), p)
    gW = np.zeros((5, 3)); gW[3, 0] = rho * gam  # d(rho w)/dx: shear, no heat flux
    z = np.zeros(3)
    n = [1.0, 0.0, 0.0]
    a = oracle.face_flux_o2(dict(PARAMS, Pr=1.0), W, rho, gW, gW[0], z, W, rho, gW, gW[0], z, n, dt)
    b = oracle.face_flux_o2(dict(PARAMS, Pr=2.0 / 3.0), W, rho, gW, gW[0], z, W, rho, gW, gW[0], z, n, dt)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-18)
    WL = _W(1.0, (0.3, -0.1, 0.2), 0.9)
    WR = _W(0.4, (0.1, 0.2, -0.1), 0.5)
    z5 = np.zeros((5, 3))
    a = oracle.face_flux_o2(dict(PARAMS, Pr=1.0), WL, 0.6, z5, z, z, WR, 0.3, z5, z, z, n, dt)
    b = oracle.face_flux_o2(dict(PARAMS, Pr=0.5), WL, 0.6, z5, z, z, WR, 0.3, z5, z, z, n, dt)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-18)


def test_zero_gradients_reduce_to_first_order():
    WL = _W(1.0, (0.3, -0.1, 0.2), 0.9)
    WR = _W(0.4, (0.1, 0.2, -0.1), 0.5)
    n = np.array([0.36, 0.48, 0.8])
    z5 = np.zeros((5, 3)); z3 = np.zeros(3)
    F2 = oracle.face_flux_o2(PARAMS, WL, 0.6, z5, z3, z3, WR, 0.3, z5, z3, z3, n, 2e-3)
    F1 = oracle.face_flux(dict(PARAMS, order=1), "interior", WL, 0.6, WR, 0.3, n, 2e-3)
    np.testing.assert_allclose(F2, F1, rtol=1e-12, atol=1e-16)


def test_second_order_sod_is_more_accurate():
    errs = {}
    nx = 100
    for order in (1, 2):
        cfg = wl.shock_tube(nx=nx, ny=1, nz=1, Kn=1e-8, width=1.0 / nx)
        cfg["params"]["order"] = order
        cfg["params"]["C2"] = 1.0
        s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
        while s.state()["t"] < 0.1:
            s.step()
        st = s.state()
        nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
        vol = s.geometry("vol")
        slab = np.minimum((nodes[tets].mean(1)[:, 0] * nx).astype(int), nx - 1)
        rho = np.bincount(slab, st["W"][0] * vol, nx) / np.bincount(slab, vol, nx)
        ex = riemann_exact.density((np.arange(nx) + 0.5) / nx, st["t"], (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
        errs[order] = np.mean(np.abs(rho - ex))
    assert errs[2] < 0.8 * errs[1], errs
