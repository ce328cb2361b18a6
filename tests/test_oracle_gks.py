"""Pins of the oracle's gas-kinetic (GKS) start-up step: the method without
particles (Sec. 3.2), used for the initial fields of the steady cases (Sec. 4.3, 4.4),
with the global time step or local time steps.

* free-molecular limit (tau -> infinity): the GKS flux is dt times the upwind
  Maxwellian flux int_{u.n>0} u.n psi g_L + int_{u.n<0} u.n psi g_R, checked
  against direct quadrature, first and second order (zero slopes);
* continuum limit (e^{-dt/tau} = 0, nothing is sampled): a GKS step is the
  method's own step, bit for bit, at first and second order, walls included;
* closed specular box: mass and energy are conserved to rounding;
* local time steps: a uniform flow on a jittered mesh stays uniform, and where
  every cell has the same local step the result is the global step's;
* a state holding particles is refused.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import workloads as wl


def _W(rho, U, p):
    U = np.asarray(U, float)
    return np.concatenate([[rho], rho * U, [0.5 * rho * U.dot(U) + 1.5 * p]])


def _half_flux_quad(W, n, half, R=1.0):
    """int_{half} u.n psi g du for the Maxwellian of W, by quadrature:
    Gauss-Hermite across the face, adaptive along n."""
    from scipy.integrate import quad
    rho = W[0]
    U = W[1:4] / rho
    p = (W[4] - 0.5 * rho * U.dot(U)) / 1.5
    lam = rho / (2.0 * p)
    n = np.asarray(n, float) / np.linalg.norm(n)
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    t1 = np.cross(n, a); t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    Un, U1, U2 = U.dot(n), U.dot(t1), U.dot(t2)
    xg, wg = np.polynomial.hermite.hermgauss(10)
    s = 1.0 / math.sqrt(lam)
    lo, hi = (0.0, np.inf) if half > 0 else (-np.inf, 0.0)
    out = np.zeros(5)
    for xa, wa in zip(xg, wg):
        for xb, wb in zip(xg, wg):
            v, w = U1 + s * xa, U2 + s * xb
            for k in range(5):
                def f(u, k=k):
                    vel = u * n + v * t1 + w * t2
                    psi = (1.0, vel[0], vel[1], vel[2], 0.5 * vel.dot(vel))[k]
                    return math.sqrt(lam / math.pi) * math.exp(-lam * (u - Un) ** 2) * u * psi
                out[k] += rho * wa * wb / math.pi * quad(f, lo, hi, epsabs=1e-15, epsrel=1e-12)[0]
    return out


PARAMS = {"R": 1.0, "mu_ref": 1e12, "T_ref": 1.0, "omega": 0.81, "CFL": 0.5, "C2": 0.0, "order": 1,
          "venkat_K": 5.0, "N_ref": 10, "seed": 1, "bc": []}


def test_gks_flux_free_molecular_limit():
    WL = _W(1.2, (0.3, -0.2, 0.1), 0.9)
    WR = _W(0.5, (-0.1, 0.25, 0.05), 0.4)
    n = np.array([0.48, -0.6, 0.64])
    dt = 0.02
    ref = dt * (_half_flux_quad(WL, n, +1) + _half_flux_quad(WR, n, -1))
    F1 = oracle.face_flux(PARAMS, "interior", WL, WL[0], WR, WR[0], n, dt, gks=True)
    np.testing.assert_allclose(F1, ref, rtol=1e-9, atol=1e-15)
    z5, z3 = np.zeros((5, 3)), np.zeros(3)
    F2 = oracle.face_flux_o2(dict(PARAMS, order=2), WL, WL[0], z5, z3, z3, WR, WR[0], z5, z3, z3, n, dt,
                             gks=True)
    np.testing.assert_allclose(F2, ref, rtol=1e-9, atol=1e-15)
    # with particles the free transport is theirs: the wave flux vanishes
    F0 = oracle.face_flux(PARAMS, "interior", WL, WL[0], WR, WR[0], n, dt)
    assert np.max(np.abs(F0)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("order", [1, 2])
def test_gks_step_is_the_method_without_particles(order):
    cfg = wl.cavity(n=3, Kn=1e-9, N_ref=8, precision="fp64", order=order)
    a = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    b = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    for _ in range(3):
        a.step()
        b.gks_step()
        assert a.sizes()["n_particles"] == 0
        sa, sb = a.state(), b.state()
        np.testing.assert_array_equal(sa["W"], sb["W"])
        assert sa["t"] == sb["t"]


@pytest.mark.parametrize("order", [1, 2])
def test_gks_conserves_mass_and_energy_in_a_closed_box(order):
    cfg = wl.uniform_box(n=(3, 3, 3), jitter_amount=0.2, seed=9, Kn=0.05, bc_type="specular")
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    cen = nodes[tets].mean(1)
    rho = 1.0 + 0.3 * np.sin(3.0 * cen[:, 0]) * np.cos(2.0 * cen[:, 1])
    U = 0.2 * np.stack([np.sin(2 * cen[:, 2]), np.cos(3 * cen[:, 0]), 0.5 * cen[:, 1]])
    p = 1.0 + 0.2 * np.cos(4.0 * cen[:, 2])
    W0 = np.concatenate([rho[None], rho * U, (0.5 * rho * (U * U).sum(0) + 1.5 * p)[None]])
    s = oracle.OracleSim(cfg["mesh"], W0, dict(cfg["params"], order=order))
    vol = s.geometry("vol")
    tot0 = (s.state()["W"] * vol).sum(1)
    s.gks_step(4)
    tot = (s.state()["W"] * vol).sum(1)
    np.testing.assert_allclose(tot[[0, 4]], tot0[[0, 4]], rtol=1e-13)
    assert not np.allclose(s.state()["W"], W0)


def test_gks_local_steps_keep_a_uniform_flow():
    cfg = wl.uniform_box(n=(3, 3, 3), jitter_amount=0.25, seed=11, U=(0.3, -0.2, 0.1), Kn=0.05,
                         bc_type="farfield")
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], dict(cfg["params"], order=2))
    s.gks_step(3, local=True)
    st = s.state()
    np.testing.assert_allclose(st["W"], cfg["W0"], rtol=1e-13, atol=1e-14)
    assert st["t"] == 0.0  # pseudo-time iterations


def test_gks_local_steps_with_equal_cell_steps_are_the_global_step():
    # congruent tets of one cube pattern, uniform T and U = 0: every cell has
    # the same local step, while rho (and p) vary
    cfg = wl.uniform_box(n=(3, 3, 3), Kn=0.05, bc_type="specular")
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    cen = nodes[tets].mean(1)
    rho = 1.0 + 0.25 * np.sin(3.0 * cen[:, 0] + cen[:, 2])
    W0 = np.concatenate([rho[None], np.zeros((3, len(tets))), (1.5 * rho)[None]])
    a = oracle.OracleSim(cfg["mesh"], W0, dict(cfg["params"], order=2))
    vol, dS = a.geometry("vol"), a.geometry("dS")
    r = vol / dS.sum(0)
    assert np.ptp(r) <= 1e-14 * r.max()
    b = oracle.OracleSim(cfg["mesh"], W0, dict(cfg["params"], order=2))
    a.gks_step()  # one step: after it T is no longer uniform
    b.gks_step(local=True)
    np.testing.assert_allclose(b.state()["W"], a.state()["W"], rtol=1e-13, atol=1e-15)


def test_gks_refuses_a_state_with_particles():
    cfg = wl.uniform_box(n=(2, 2, 2), Kn=1.0, N_ref=4)
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    s.step()
    assert s.sizes()["n_particles"] > 0
    with pytest.raises(RuntimeError, match="without particles"):
        s.gks_step()
