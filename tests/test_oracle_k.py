"""Pins of the oracle with K internal degrees of freedom (rho E = rho |U|^2/2 +
(3+K)/2 p; particles carry an internal energy e, phi = m (1, u, (|u|^2 + e)/2);
Sec. 2.2 names the internal energy of a particle and its sampling from T and K).

* a uniform state: the particle-free (GKS) flux is dt times the Euler flux
  with gamma = (K+5)/(K+3), orders 1 and 2;
* slope moments <u_n u_d (a.psi) psi> and the micro-slope solve with xi, against
  quadrature in (u, v, w) and scipy's chi-square moments of |xi|^2;
* Chapman-Enskog limit: heat flux -(K+5)/2 R mu dT/dx dt (c_p = (K+5)/2 R);
* continuum limit: the Sod profile converges to the exact Riemann solution
  with gamma = 7/5 (K = 2, the paper's diatomic Sod case);
* sampled internal energies and diffuse-wall re-emitted ones are R T chi^2_K
  (both precisions); a closed box with particles conserves mass exactly and
  energy to rounding.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import workloads as wl
from tests import riemann_exact

PARAMS = {"R": 1.0, "mu_ref": 1e-3, "T_ref": 1.0, "omega": 0.81, "CFL": 0.5, "C2": 0.0, "order": 1,
          "venkat_K": 5.0, "N_ref": 10, "seed": 1, "bc": []}


def _W(rho, U, p, K):
    U = np.asarray(U, float)
    return np.concatenate([[rho], rho * U, [0.5 * rho * U.dot(U) + (3 + K) / 2.0 * p]])


@pytest.mark.parametrize("K", [1, 2, 5])
def test_uniform_state_gks_flux_is_euler(K):
    rho, U, p = 1.3, np.array([0.3, -0.2, 0.4]), 0.8
    W = _W(rho, U, p, K)
    n = np.array([0.36, 0.48, 0.8])
    dt = 0.01
    E = W[4]
    Fe = np.concatenate([[rho * U @ n], rho * (U @ n) * U + p * n, [(U @ n) * (E + p)]])
    params = dict(PARAMS, K=K)
    F1 = oracle.face_flux(params, "interior", W, rho, W, rho, n, dt, gks=True)
    np.testing.assert_allclose(F1, dt * Fe, rtol=1e-12, atol=1e-15)
    z5, z3 = np.zeros((5, 3)), np.zeros(3)
    F2 = oracle.face_flux_o2(dict(params, order=2), W, rho, z5, z3, z3, W, rho, z5, z3, z3, n, dt, gks=True)
    np.testing.assert_allclose(F2, dt * Fe, rtol=1e-12, atol=1e-15)


def _quad_k(U, lam, half, K, fun):
    """int fun(u, v, w, s) g du dv dw over the unit Maxwellian, averaged over
    s = |xi|^2 with <s^j> from scipy's chi-square moments (fun is at most
    quadratic in s: evaluated at s = 0, 1, 2 and combined exactly)."""
    from scipy import stats
    from scipy.integrate import quad
    xg, wg = np.polynomial.hermite.hermgauss(8)
    sd = 1.0 / math.sqrt(lam)
    lo, hi = {1: (0.0, np.inf), -1: (-np.inf, 0.0), 0: (-np.inf, np.inf)}[half]
    th = 1.0 / (2.0 * lam)
    m1 = stats.chi2(K).moment(1) * th
    m2 = stats.chi2(K).moment(2) * th * th
    tot = np.zeros(5)
    for xa, wa in zip(xg, wg):
        for xb, wb in zip(xg, wg):
            v, w = U[1] + sd * xa, U[2] + sd * xb
            for k in range(5):
                def integrand(u):
                    f0, f1, f2 = (fun(u, v, w, s)[k] for s in (0.0, 1.0, 2.0))
                    c2 = 0.5 * (f2 - 2.0 * f1 + f0)
                    c1 = f1 - f0 - c2
                    return math.sqrt(lam / math.pi) * math.exp(-lam * (u - U[0]) ** 2) * (f0 + c1 * m1 + c2 * m2)
                tot[k] += wa * wb / math.pi * quad(integrand, lo, hi, epsabs=1e-14, epsrel=1e-12)[0]
    return tot


def _psi(u, v, w, s):
    return np.array([1.0, u, v, w, 0.5 * (u * u + v * v + w * w + s)])


@pytest.mark.parametrize("half", [1, 0])
def test_slope_moments_with_internal_energy(half):
    K = 2
    rng = np.random.default_rng(31 + half)
    U = rng.normal(size=3) * 0.6
    lam = 0.7
    a = rng.normal(size=5)
    for d in range(3):
        got = oracle.slope_moment(U, lam, half, a, d, K=K)
        ref = _quad_k(U, lam, half, K, lambda u, v, w, s: u * (u, v, w)[d] * (a @ _psi(u, v, w, s)) * _psi(u, v, w, s))
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-11)


def test_micro_slope_with_internal_energy():
    K = 3
    rng = np.random.default_rng(9)
    U = rng.normal(size=3)
    lam = 0.9
    M = np.zeros((5, 5))
    for c in range(5):
        e = np.zeros(5); e[c] = 1.0
        M[:, c] = _quad_k(U, lam, 0, K, lambda u, v, w, s: _psi(u, v, w, s) * (e @ _psi(u, v, w, s)))
    b = rng.normal(size=5)
    np.testing.assert_allclose(oracle.micro_slope(U, lam, b, K=K), np.linalg.solve(M, b), rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("K", [0, 2])
def test_navier_stokes_heat_flux_with_internal_energy(K):
    rho, T, gam = 1.0, 1.0, 0.04
    p = rho * T
    dt = 1.0
    tau = 1e-3 * dt
    params = dict(PARAMS, order=2, mu_ref=tau * p, K=K)
    W = _W(rho, (0.0, 0.0, 0.0), p, K)
    gW = np.zeros((5, 3)); gW[0, 0] = -rho * gam / T  # uniform pressure, dT/dx = gam
    z = np.zeros(3)
    F = oracle.face_flux_o2(params, W, rho, gW, gW[0], z, W, rho, gW, gW[0], z, [1.0, 0.0, 0.0], dt)
    assert F[4] == pytest.approx(-(K + 5) / 2.0 * tau * p * gam * dt, rel=3e-3)


def test_continuum_sod_with_internal_energy():
    K = 2
    errs = []
    for nx in (50, 100, 200):
        cfg = wl.shock_tube(nx=nx, ny=1, nz=1, Kn=1e-8, width=1.0 / nx, K=K)
        s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
        while s.state()["t"] < 0.1:
            s.step()
        assert s.sizes()["n_particles"] == 0
        st = s.state()
        nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
        vol = s.geometry("vol")
        slab = np.minimum((nodes[tets].mean(1)[:, 0] * nx).astype(int), nx - 1)
        rho = np.bincount(slab, st["W"][0] * vol, nx) / np.bincount(slab, vol, nx)
        xc = (np.arange(nx) + 0.5) / nx
        ex = riemann_exact.density(xc, st["t"], (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g=1.4)
        errs.append(np.mean(np.abs(rho - ex)))
        if nx == 200:
            wrong = riemann_exact.density(xc, st["t"], (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g=5.0 / 3.0)
            assert np.mean(np.abs(rho - wrong)) > 2.0 * errs[-1]
    assert errs[1] < 0.8 * errs[0] and errs[2] < 0.8 * errs[1]
    assert errs[2] < 0.008


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("K", [2, 5])
def test_sampled_internal_energy_is_chi_square(precision, K):
    from scipy import stats
    T = 1.7
    cfg = wl.uniform_box(n=(2, 2, 2), Kn=1.0, N_ref=4000, p=T, precision=precision, K=K)
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    s.prepare()
    smp = s.state()
    e = np.concatenate([_cell_e(s, c) for c in range(3)])
    assert e.size > 5000
    assert stats.kstest(e / T, stats.chi2(K).cdf).pvalue > 1e-4
    assert stats.kstest(e / T, stats.chi2(K + 1).cdf).pvalue < 1e-6


def _cell_e(s, cell):
    """Internal energies of the particles `cell` samples: one oracle step from a
    particle-free state, then the survivors' and the cell's e (Kn large: no
    collisions, positions only move)."""
    return s.sample_cell(cell)["e"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wall_reemission_internal_energy(precision):
    from scipy import stats
    K, T_w = 2, 2.0
    cfg = wl.uniform_box(n=(2, 2, 2), bc_type="wall", T_w=T_w, precision=precision, Kn=1e6, K=K)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    cen = nodes[tets].mean(1)
    c = int(np.argmin(cen[:, 0] + 10 * np.abs(cen[:, 1] - 0.25) + 10 * np.abs(cen[:, 2] - 0.25)))
    x = cen[c].astype(np.float32).astype(np.float64)
    speed = 16.0
    dt = float(np.float32(x[0] / speed * (1 + 1e-4)))
    es = []
    for k in range(3000):
        pid = (5 << 40) | (1 << 16) | k
        out = s.track_one(pid=pid, cell=c, x=x, u=[-speed, 0.0, 0.0], tau_cell=1.0, dt=dt, step=5, e=0.25)
        assert out["status"] == 0
        es.append(out["e"])
    es = np.array(es)
    assert stats.kstest(es / T_w, stats.chi2(K).cdf).pvalue > 1e-4
    # a particle that meets no wall keeps its internal energy
    out = s.track_one(pid=7, cell=c, x=x, u=[0.0, 0.0, 0.0], tau_cell=1.0, dt=dt, step=5, e=0.25)
    assert out["e"] == pytest.approx(0.25, rel=1e-7)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_closed_box_conservation_with_internal_energy(precision):
    K = 2
    cfg = wl.uniform_box(n=(4, 3, 3), Kn=0.03, N_ref=30, bc_type="specular", precision=precision,
                         jitter_amount=0.15, seed=4, K=K)
    W0 = cfg["W0"].copy()
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    left = nodes[tets].mean(1)[:, 0] < 0.5
    W0[:, left] *= 2.0
    W0[1, :] = 0.2 * W0[0]
    W0[4] += 0.5 * 0.04 * W0[0]
    s = oracle.OracleSim(cfg["mesh"], W0, cfg["params"])
    vol = s.geometry("vol")
    M0, E0 = (W0[0] * vol).sum(), (W0[4] * vol).sum()
    for _ in range(8):
        s.step()
        assert s.last("pflux")[0].sum() == 0
        W = s.state()["W"]
        assert abs((W[0] * vol).sum() - M0) < 1e-13 * M0
        assert abs((W[4] * vol).sum() - E0) < 1e-12 * E0
    st = s.state()
    assert st["id"].size > 1000 and np.all(st["e"] > 0.0)
