"""Pins of the oracle's wave-flux building blocks (Sec. 2.1, 2.3, 2.4 (e)).

* q1..q5 against numerical integration (40 digits) of the printed c1..c5 over
  [0, dt]; the collisional-wave coefficients a4, a5 against the integral that
  defines F^{fr,wave} (UGKS free transport minus the DVM part carried by the
  sampled particles); the printed limits dt >> tau and dt << tau.
* Half- and full-range Maxwellian moments against direct quadrature in an
  independently chosen velocity frame.
* Whole-face fluxes of uniform states against the closed-form Euler flux, and
  the wall / specular / far-field variants against their defining properties.
"""
import math

import numpy as np
import pytest

import oracle

PARAMS = {"R": 1.0, "mu_ref": 0.05, "T_ref": 1.0, "omega": 0.81, "CFL": 0.5, "C2": 0.0,
          "order": 1, "N_ref": 10, "seed": 1, "bc": []}


def _q_reference(dt, tau):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    dt, tau = mpmath.mpf(dt), mpmath.mpf(tau)
    E = mpmath.exp(-dt / tau)
    c = [lambda t: 1 - mpmath.exp(-t / tau),
         lambda t: t * mpmath.exp(-t / tau) - tau * (1 - mpmath.exp(-t / tau)),
         lambda t: t - tau * (1 - mpmath.exp(-t / tau)),
         lambda t: mpmath.exp(-t / tau),
         lambda t: -t * mpmath.exp(-t / tau),
         lambda t: mpmath.exp(-t / tau) - E,          # c4 minus the particle part
         lambda t: -t * mpmath.exp(-t / tau) + t * E]  # c5 minus the particle part
    return [float(mpmath.quad(f, [0, dt])) for f in c]


@pytest.mark.parametrize("ratio", [1e-6, 1e-3, 0.05, 0.5, 0.99, 1.01, 3.0, 40.0, 1e3, 1e6, 1e9])
def test_qcoef_equals_time_integrals_of_c(ratio):
    dt = 2.5e-3
    tau = ratio * dt
    got = oracle.qcoef(dt, tau)
    ref = _q_reference(dt, tau)
    scale = [dt, dt * dt, dt * dt, dt, dt * dt, dt, dt * dt]
    for g, r, s in zip(got, ref, scale):
        assert abs(g - r) <= 1e-13 * abs(r) + 1e-15 * s, (ratio, g, r)


def test_qcoef_printed_limits():
    dt = 1.0
    q = oracle.qcoef(dt, 1e-9)  # dt >> tau: q1 -> dt, q3 -> dt^2/2
    assert q[0] == pytest.approx(dt, rel=1e-8) and q[2] == pytest.approx(dt * dt / 2, rel=1e-8)
    assert abs(q[3]) < 1e-8 and abs(q[4]) < 1e-8
    q = oracle.qcoef(dt, 1e9)  # dt << tau: q4 -> dt, q5 -> -dt^2/2
    assert q[3] == pytest.approx(dt, rel=1e-8) and q[4] == pytest.approx(-dt * dt / 2, rel=1e-8)
    assert abs(q[0]) < 1e-8 and abs(q[2]) < 1e-8
    # the collisional-wave free-transport coefficients vanish in both limits
    for tau in (1e-9, 1e9):
        q = oracle.qcoef(dt, tau)
        assert abs(q[5]) < 1e-8 and abs(q[6]) < 1e-8


def _quad_moments(U, lam, n, half):
    """int_{half} g psi du and int_{half} (u.n) g psi du for a unit-density Maxwellian,
    by Gauss-Hermite in two tangential directions (exact for the polynomial
    weights) and adaptive quadrature in the normal one."""
    from scipy.integrate import quad
    U = np.asarray(U, float)
    n = np.asarray(n, float) / np.linalg.norm(n)
    # an orthonormal frame chosen differently from the oracle's
    a = np.array([0.3, -0.7, 0.64])
    t1 = a - a.dot(n) * n
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    xg, wg = np.polynomial.hermite.hermgauss(6)  # exact: tangential weights are quadratic
    s = 1.0 / math.sqrt(lam)
    Un, U1, U2 = U.dot(n), U.dot(t1), U.dot(t2)
    H = np.zeros(5)
    G = np.zeros(5)
    lo, hi = {1: (0.0, np.inf), -1: (-np.inf, 0.0), 0: (-np.inf, np.inf)}[half]
    for i, (xa, wa) in enumerate(zip(xg, wg)):
        for j, (xb, wb) in enumerate(zip(xg, wg)):
            va, vb = U1 + s * xa, U2 + s * xb
            w2 = wa * wb / math.pi

            def comp(un, k, flux):
                u = un * n + va * t1 + vb * t2
                psi = [1.0, u[0], u[1], u[2], 0.5 * u.dot(u)][k]
                g = math.sqrt(lam / math.pi) * math.exp(-lam * (un - Un) ** 2)
                return g * psi * (un if flux else 1.0)
            for k in range(5):
                for flux, acc in ((False, H), (True, G)):
                    if half == 0:
                        v = quad(comp, -np.inf, np.inf, args=(k, flux), epsabs=1e-14, epsrel=1e-13)[0]
                    else:
                        v = quad(comp, lo, hi, args=(k, flux), epsabs=1e-14, epsrel=1e-13)[0]
                    acc[k] += w2 * v
    return H, G


@pytest.mark.parametrize("case", range(4))
def test_maxwell_moments_against_quadrature(case):
    rng = np.random.default_rng(100 + case)
    U = rng.normal(size=3) * [0.3, 1.0, 2.0][case % 3]
    lam = rng.uniform(0.3, 2.0)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    for half in (1, -1, 0):
        H, G = oracle.maxwell_moments(U, lam, n, half)
        Hq, Gq = _quad_moments(U, lam, n, half)
        np.testing.assert_allclose(H, Hq, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(G, Gq, rtol=1e-10, atol=1e-12)


def _euler_flux(W, n):
    rho = W[0]
    U = W[1:4] / rho
    p = (W[4] - 0.5 * rho * U.dot(U)) / 1.5
    Un = U.dot(n)
    return np.concatenate([[rho * Un], rho * Un * U + p * n, [Un * (W[4] + p)]]), p


def _W(rho, U, p):
    U = np.asarray(U, float)
    return np.concatenate([[rho], rho * U, [0.5 * rho * U.dot(U) + 1.5 * p]])


@pytest.mark.parametrize("U", [(0, 0, 0), (0.3, -0.2, 0.5), (2.5, 0.1, -0.4)])
@pytest.mark.parametrize("frac_h", [1.0, 0.37, 0.0])
def test_uniform_state_flux_is_scaled_euler_flux(U, frac_h):
    """Equal left/right states: W0 = W, and both F^eq and F^{fr,wave} reduce to
    multiples of the Euler flux: F = (q1 + a4 rho^h/rho) F_Euler(W)."""
    rho, p = 1.3, 0.8
    W = _W(rho, U, p)
    n = np.array([0.48, -0.6, 0.64])
    dt = 1e-3
    F = oracle.face_flux(PARAMS, "interior", W, frac_h * rho, W, frac_h * rho, n, dt)
    FE, _ = _euler_flux(W, n)
    T = p / rho
    tau = PARAMS["mu_ref"] * T ** PARAMS["omega"] / p
    q = oracle.qcoef(dt, tau)
    np.testing.assert_allclose(F, (q[0] + q[5] * frac_h) * FE, rtol=1e-12, atol=1e-16)


def test_flux_antisymmetry_and_upwinding():
    """Swapping sides and flipping the normal negates the flux; a supersonic
    state from the left is pure upwind."""
    WL = _W(1.0, (0.2, 0.1, 0.0), 1.0)
    WR = _W(0.125, (-0.1, 0.0, 0.3), 0.1)
    n = np.array([0.0, 0.6, 0.8])
    dt = 2e-3
    F1 = oracle.face_flux(PARAMS, "interior", WL, 0.7, WR, 0.1, n, dt)
    F2 = oracle.face_flux(PARAMS, "interior", WR, 0.1, WL, 0.7, -n, dt)
    np.testing.assert_allclose(F1, -F2, rtol=1e-13, atol=1e-17)
    Ws = _W(1.0, 10.0 * n, 1.0)   # Mach ~7.7 along n, into a near vacuum
    Wv = _W(1e-14, (0, 0, 0), 1e-14)
    F = oracle.face_flux(PARAMS, "interior", Ws, 1.0, Wv, 1e-14, n, dt)
    FE, _ = _euler_flux(Ws, n)
    q = oracle.qcoef(dt, PARAMS["mu_ref"] / 1.0)
    np.testing.assert_allclose(F, (q[0] + q[5]) * FE, rtol=1e-9)


@pytest.mark.parametrize("frac_h", [1.0, 0.4])
def test_diffuse_wall_flux(frac_h):
    """Zero net mass flux of the wave; at rest and at the wall temperature the
    energy flux vanishes and the normal momentum flux is (q1 + a4 rho^h/rho) p."""
    rho, p = 0.9, 0.9
    W = _W(rho, (0, 0, 0), p)
    n = np.array([0.0, 0.0, 1.0])
    dt, tau = 1e-3, 4e-3
    bc = {"type": "wall", "T_w": 1.0, "U_w": (0.0, 0.0, 0.0)}
    F = oracle.face_flux(PARAMS, "wall", W, frac_h * rho, None, 0, n, dt, tau_wall=tau, bc=bc)
    q = oracle.qcoef(dt, tau)
    assert abs(F[0]) < 1e-16
    assert abs(F[4]) < 1e-15
    np.testing.assert_allclose(F[1:4], (q[0] + q[5] * frac_h) * p * n, rtol=1e-12, atol=1e-17)
    # a hot gas loses energy to a cold wall, a moving wall drags the gas
    Wh = _W(rho, (0, 0, 0), 2 * p)
    Fh = oracle.face_flux(PARAMS, "wall", Wh, rho, None, 0, n, dt, tau_wall=tau, bc=bc)
    assert Fh[4] > 0 and abs(Fh[0]) < 1e-15
    bcm = {"type": "wall", "T_w": 1.0, "U_w": (0.5, 0.0, 0.0)}
    Fm = oracle.face_flux(PARAMS, "wall", W, rho, None, 0, n, dt, tau_wall=tau, bc=bcm)
    assert Fm[1] < 0  # x-momentum flows from the wall (outside, along -n) into the gas


def test_specular_and_far_field():
    W = _W(1.1, (0.3, -0.2, 0.4), 0.7)
    n = np.array([0.6, 0.0, 0.8])
    dt = 1e-3
    F = oracle.face_flux(PARAMS, "specular", W, 0.5, None, 0, n, dt)
    assert F[0] == 0.0 and F[4] == 0.0
    assert np.allclose(np.cross(F[1:4], n), 0.0, atol=1e-18)
    assert F[1:4].dot(n) > 0
    # outflow of a uniform state at rest: the ghost is all-hydro, so
    # F = q1 F_E + a4 rho^h G+ + q4 rho G- ; mass part in closed form
    W0 = _W(1.0, (0, 0, 0), 1.0)
    Fo = oracle.face_flux(PARAMS, "outflow", W0, 0.3, None, 0, n, dt)
    lam = 1.0 / 2.0
    q = oracle.qcoef(dt, PARAMS["mu_ref"] / 1.0)
    half = 1.0 / (2.0 * math.sqrt(math.pi * lam))
    assert Fo[0] == pytest.approx(q[5] * 0.3 * half - q[3] * 1.0 * half, rel=1e-12)
    # inflow with the ghost equal to the interior state gives the same flux
    bc = {"type": "inflow", "W_in": tuple(W0)}
    Fi = oracle.face_flux(PARAMS, "inflow", W0, 0.3, None, 0, n, dt, bc=bc)
    np.testing.assert_allclose(Fi, Fo, rtol=1e-14, atol=1e-18)
