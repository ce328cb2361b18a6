"""Pins of the oracle's first-order g_p sampling (option, Sec. 2.2).

The hydrodynamic particles are drawn from g_p = g - c (u.grad g + g_t),
c = tau - dt e^{-dt/tau} / (1 - e^{-dt/tau}); with X = (u - U)/sqrt(RT) the
acceptance weight is 1 + phi(X), phi = a0 + L.X + X^T Q X + (C.X)|X|^2.

* conservation: g_p has the moments of g, i.e. E[phi] = E[phi X] = E[phi |X|^2]
  = 0 for X ~ N(0, I): a0 = 0, tr Q = 0, L + 5 C = 0;
* the non-equilibrium moments are the Navier-Stokes (BGK) ones with c in
  place of tau: pressure tensor p (I + 2Q) with Q = -(c/2)(grad U + grad U^T -
  2/3 div U I), heat flux 5 rho (RT)^{3/2} C = -(5/2) R c p grad T, for
  arbitrary gradients of rho, U and p (the density and pressure gradients
  must cancel through g_t);
* the sampler draws what the polynomial prescribes: mean, covariance I + 2Q,
  E[X |X|^2] = 10 C and the exact CDF of a marginal (both precisions); a
  cell's particles are U + sqrt(RT) X of the sampler with its coefficients;
* zero gradients give plain N(0, I) draws; large gradients are limited to the
  bound M = 2; first-order g_p needs the second-order reconstruction.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import workloads as wl


def _linear_state(grad_scale=1.0, n=(5, 4, 4), seed=3, N_ref=20, Kn=0.05, U0=(0.2, -0.1, 0.05)):
    cfg = wl.uniform_box(n=n, Kn=Kn, bc_type="outflow", N_ref=N_ref)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    cen = nodes[tets].mean(1)
    rng = np.random.default_rng(seed)
    gr, gU, gp = (rng.normal(size=3) * 0.1 * grad_scale, rng.normal(size=(3, 3)) * 0.1 * grad_scale,
                  rng.normal(size=3) * 0.1 * grad_scale)
    x = cen - cen.mean(0)
    rho = 1.0 + x @ gr
    U = np.asarray(U0)[:, None] + gU @ x.T
    p = 1.0 + x @ gp
    W0 = np.concatenate([rho[None], rho * U, (0.5 * rho * (U * U).sum(0) + 1.5 * p)[None]])
    params = dict(cfg["params"], order=2, venkat_K=1e6, sampling="gp1")
    return cfg, W0, params


def _interior(cfg):
    tets, bf = cfg["mesh"]["tets"], cfg["mesh"]["bfaces"]
    bn = set(np.unique(bf).tolist())
    return [i for i, t in enumerate(tets) if not (set(t.tolist()) & bn)]


def _ns_expectation(W, gW, R, c):
    """Q and C that the Navier-Stokes stress and heat flux give with c for tau."""
    rho, mom, E = W[0], W[1:4], W[4]
    U = mom / rho
    p = (E - 0.5 * rho * U @ U) / 1.5
    T = p / (rho * R)
    grho, gm, gE = gW[0], gW[1:4], gW[4]          # [3] (d), [3 (j), 3 (d)], [3]
    dU = (gm - np.outer(U, grho)) / rho            # dU[j, d] = d U_j / d x_d
    dp = (2.0 / 3.0) * (gE - U @ gm + 0.5 * (U @ U) * grho)
    dT = (dp - R * T * grho) / (rho * R)
    S = dU + dU.T - (2.0 / 3.0) * np.trace(dU) * np.eye(3)
    Q = -0.5 * c * S
    sig = math.sqrt(R * T)
    C = -0.5 * c * R * dT / sig
    return Q, C


def _temperature_wave(N_ref=20, amp=0.8):
    """Uniform pressure, T = 1 + amp sin(4 pi x) on 12 cells along x: a smooth
    profile steep enough per cell for the bound of the correction to exceed 1."""
    cfg = wl.uniform_box(n=(12, 2, 2), Kn=5.0, bc_type="specular", N_ref=N_ref)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    x = nodes[tets].mean(1)[:, 0]
    T = 1.0 + amp * np.sin(4.0 * math.pi * x)
    rho = 1.0 / T
    W0 = np.concatenate([rho[None], np.zeros((3, len(tets))), np.full((1, len(tets)), 1.5)])
    return cfg, W0, dict(cfg["params"], order=2, venkat_K=1e6, sampling="gp1")


def _coef_parts(co):
    a0, L = co[0], co[1:4]
    Q = np.array([[co[4], co[7], co[8]], [co[7], co[5], co[9]], [co[8], co[9], co[6]]])
    return a0, L, Q, co[10:13], co[13]


@pytest.mark.parametrize("Kn", [1e-3, 0.05, 5.0])
def test_gp_coefficients_conserve_and_give_navier_stokes_moments(Kn):
    cfg, W0, params = _linear_state(Kn=Kn)
    s = oracle.OracleSim(cfg["mesh"], W0, params)
    s.prepare()
    gW, _ = s.gradients(limited=True)
    dt = s.last("dt")
    tau = s.last("tau")
    R = params["R"]
    for i in _interior(cfg)[:12]:
        a0, L, Q, C, M = _coef_parts(s.gp_coefficients(i))
        assert M < 2.0  # not limited
        e = math.exp(-dt / tau[i])
        c = tau[i] - dt * e / (1.0 - e)
        Qe, Ce = _ns_expectation(s.state()["W"][:, i], gW[:, :, i], R, c)
        scale = max(np.abs(Qe).max(), 1e-300)
        assert abs(a0) <= 1e-11 * scale and abs(np.trace(Q)) <= 1e-11 * scale
        np.testing.assert_allclose(L, -5.0 * C, rtol=1e-9, atol=1e-12 * scale)
        np.testing.assert_allclose(Q, Qe, rtol=1e-8, atol=1e-11 * scale)
        np.testing.assert_allclose(C, Ce, rtol=1e-8, atol=1e-11 * scale)


def _coef(Q, C):
    L = -5.0 * np.asarray(C)
    co = np.concatenate([[0.0], L, [Q[0][0], Q[1][1], Q[2][2], Q[0][1], Q[0][2], Q[1][2]], C])
    Phi = 5 * np.linalg.norm(L) + 25 * np.sqrt((np.asarray(Q) ** 2).sum()) + 125 * np.linalg.norm(C)
    assert Phi <= 1.0
    return np.concatenate([co, [1.0 + Phi]])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gp_draws_follow_the_target(precision):
    """The sampler on its own: for phi = X^T Q X + (C.X)(|X|^2 - 5) (tr Q = 0)
    the draws have E[X] = 0, E[X X^T] = I + 2Q, E[X |X|^2] = 10 C, and the
    marginal of X_1 has the CDF Phi(x) - N(x)(Q11 x + C1 (x^2 - 1))."""
    from scipy import stats
    Q = np.array([[0.008, 0.010, 0.0], [0.010, -0.003, 0.002], [0.0, 0.002, -0.005]])
    C = np.array([0.0025, -0.0015, 0.0008])
    n = 1_500_000
    X = oracle.gp_draw(_coef(Q, C), n, id0=7 << 16, step=3, seed=11, precision=precision)
    zm = X.mean(1) * math.sqrt(n)
    cov = X @ X.T / n
    zc = (cov - np.eye(3) - 2.0 * Q) * math.sqrt(n) / np.sqrt(np.ones((3, 3)) + np.eye(3))
    h = (X * (X * X).sum(0)).mean(1)
    zh = (h - 10.0 * C) * math.sqrt(n / 35.0)
    assert np.abs(zm).max() < 4.5 and np.abs(zc).max() < 4.5 and np.abs(zh).max() < 4.5, (zm, zc, zh)
    # the Maxwellian is rejected by the same statistics
    assert np.abs(2.0 * Q * math.sqrt(n)).max() > 20 and np.abs(10.0 * C * math.sqrt(n / 35.0)).max() > 4.5

    def cdf(x):
        return stats.norm.cdf(x) - stats.norm.pdf(x) * (Q[0, 0] * x + C[0] * (x * x - 1.0))
    assert stats.kstest(X[0], cdf).pvalue > 1e-3
    assert stats.kstest(X[0], "norm").pvalue < 1e-4


def test_gp_cell_samples_use_the_cell_coefficients():
    cfg, W0, params = _temperature_wave(N_ref=200)
    s = oracle.OracleSim(cfg["mesh"], W0, params)
    s.prepare()
    i = 7
    co = s.gp_coefficients(i)
    assert np.abs(co[10:13]).max() > 1e-3
    smp = s.sample_cell(i)
    st = s.state()
    Wc = st["W"][:, i]
    U = Wc[1:4] / Wc[0]
    T = (Wc[4] - 0.5 * Wc[0] * U @ U) / (1.5 * Wc[0])
    order = np.argsort(smp["id"])
    ids = smp["id"][order]
    assert np.array_equal(ids, ids[0] + np.arange(ids.size, dtype=np.uint64))
    X = oracle.gp_draw(co, ids.size, id0=int(ids[0]), step=st["step"], seed=params["seed"])
    np.testing.assert_array_equal(smp["u"][:, order], U[:, None] + math.sqrt(T) * X)


def test_gp_without_gradients_is_the_maxwellian():
    from scipy import stats
    cfg = wl.uniform_box(n=(3, 3, 3), Kn=0.05, bc_type="outflow", N_ref=4000, U=(0.1, 0.2, -0.3))
    params = dict(cfg["params"], order=2, sampling="gp1")
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], params)
    s.prepare()
    co = s.gp_coefficients(5)
    np.testing.assert_allclose(co[:13], 0.0, atol=1e-12)
    assert co[13] == pytest.approx(1.0, abs=1e-12)
    smp = s.sample_cell(5)
    X = (smp["u"] - np.array([0.1, 0.2, -0.3])[:, None])  # R T = 1
    for d in range(3):
        assert stats.kstest(X[d], "norm").pvalue > 1e-3
    # particles are drawn on their own: no +/- pairs
    assert not np.allclose(X[:, 0::2], -X[:, 1::2])


def test_gp_large_gradients_are_limited():
    cfg, W0, params = _temperature_wave()
    s = oracle.OracleSim(cfg["mesh"], W0, params)
    s.prepare()
    Ms = np.array([s.gp_coefficients(k)[13] for k in range(len(cfg["mesh"]["tets"]))])
    assert (Ms == 2.0).any() and (Ms < 2.0).any()
    i = int(np.argmax(Ms))
    a0, L, Q, C, M = _coef_parts(s.gp_coefficients(i))
    assert M == 2.0
    bound = abs(a0) + 5 * np.linalg.norm(L) + 25 * np.sqrt((Q * Q).sum()) + 125 * np.linalg.norm(C)
    assert bound == pytest.approx(1.0, rel=1e-12)
    assert s.sample_cell(i)["id"].size > 0


def test_gp_needs_second_order():
    cfg = wl.uniform_box(n=(2, 2, 2))
    with pytest.raises(ValueError, match="order 2"):
        oracle.OracleSim(cfg["mesh"], cfg["W0"], dict(cfg["params"], order=1, sampling="gp1"))
