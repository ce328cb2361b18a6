"""Pins of the oracle's frozen-particle wave map and its reference gradient.

With the particle part of each step frozen (the recorded time steps, particle
densities and particle fluxes), a wall functional J(theta) of the wave fluxes
is a smooth function of theta = (rho_inf, U_inf, T_w).  The oracle evaluates
it generically in the scalar type: in binary64 it reproduces the wall fluxes
of the oracle's own steps, and its forward-mode dual-number derivative agrees
with central finite differences of the binary64 map.

At second order (limited least-squares reconstruction at interior faces) the
map is evaluated in binary64 with the limiter values either computed or given;
with them frozen at theta0 the map is smooth in theta and its reference
gradient is taken by central differences.  Pins: it reproduces the wall fluxes
of the oracle's second-order steps at theta0 and, from a run whose far field
and wall hold another theta, at that theta (the theta-dependent ghosts of the
reconstruction included); with every limiter value 0 it is the first-order
map, derivatives included; where the limiter is inactive, freezing it changes
no derivative; the central differences converge as h^2.
"""
import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import workloads as wl

K = 3


@pytest.fixture(scope="module")
def recorded():
    cfg = wl.wall_channel()
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    s.step(2)
    s0 = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    s0.step(2)
    fr = s0.record_frozen(K)
    return cfg, s, fr


def _theta0():
    return np.array([1.0, 0.5 * np.sqrt(5.0 / 3.0), 1.0])


def test_frozen_map_reproduces_the_steps(recorded):
    """At theta0 the frozen map's wall functional equals the sum of the wall
    fluxes of the oracle's own steps (same states, same fluxes)."""
    cfg, s, fr = recorded
    area = s.geometry("face_area")
    nb = s.geometry("face_nbr").astype(int)
    fc = s.geometry("face_normal")  # [3][nf]
    J = {0: 0.0, 1: 0.0}
    for k in range(K):
        s.step()
        F = s.last("flux")
        # a boundary face is a wall face iff its outward normal is along y or z
        bnd = nb < 0
        wall = bnd & (np.abs(fc[0]) < 0.5)
        J[0] += float((F[1, wall] * area[wall]).sum())
        J[1] += float((F[4, wall] * area[wall]).sum())
    for fun in (0, 1):
        got = s.frozen_objective(fr, _theta0(), functional=fun, tags=[1], grad=False)
        assert got == pytest.approx(J[fun], rel=1e-12, abs=1e-16)


@pytest.mark.parametrize("functional", [0, 1])
def test_dual_gradient_matches_central_differences(recorded, functional):
    cfg, s, fr = recorded
    th = _theta0()
    out = s.frozen_objective(fr, th, functional=functional, tags=[1])
    assert out[0] == pytest.approx(s.frozen_objective(fr, th, functional, [1], grad=False), rel=1e-14)
    for k in range(3):
        h = 1e-5 * th[k]
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (s.frozen_objective(fr, tp, functional, [1], grad=False) -
              s.frozen_objective(fr, tm, functional, [1], grad=False)) / (2 * h)
        scale = max(abs(out[1 + k]), 1e-3 * np.abs(out[1:]).max())
        assert abs(out[1 + k] - fd) <= 1e-6 * scale, (k, out[1 + k], fd)
    # every parameter matters within three steps in this channel
    assert np.all(np.abs(out[1:]) > 0)


def _wall_sums(s, steps):
    area = s.geometry("face_area")
    nb = s.geometry("face_nbr").astype(int)
    fc = s.geometry("face_normal")
    wall = (nb < 0) & (np.abs(fc[0]) < 0.5)
    J = {0: 0.0, 1: 0.0}
    for _ in range(steps):
        s.step()
        F = s.last("flux")
        J[0] += float((F[1, wall] * area[wall]).sum())
        J[1] += float((F[4, wall] * area[wall]).sum())
    return J


def _channel_o2(theta=None, **kw):
    """The channel at second order; with theta, its far field and walls hold
    (rho_inf, U_inf, T_w) = theta (the far-field temperature unchanged)."""
    cfg = wl.wall_channel(order=2, **kw)
    if theta is not None:
        rho, U, Tw = theta
        cfg["params"]["bc"][0]["W_in"] = tuple(float(v) for v in wl.conservative(
            np.array(rho), np.array([U, 0.0, 0.0]), np.array(rho)))
        cfg["params"]["bc"][1]["T_w"] = float(Tw)
    return cfg


@pytest.fixture(scope="module")
def recorded_o2():
    cfg = _channel_o2()
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    s.step(2)
    return cfg, s, s.record_frozen(K)


@pytest.mark.parametrize("theta", [None, (1.15, 0.8, 1.4)])
def test_o2_frozen_map_reproduces_the_steps(theta):
    """The second-order map with the particle data of a run whose far field and
    walls hold theta gives, at theta, the wall fluxes of that run's steps,
    evaluated on a simulation set up with theta0."""
    th = _theta0() if theta is None else np.array(theta)
    run = _channel_o2(theta)
    a = oracle.OracleSim(run["mesh"], run["W0"], run["params"])
    a.step(2)
    b = oracle.OracleSim(run["mesh"], run["W0"], run["params"])
    b.step(2)
    fr = b.record_frozen(K)
    J = _wall_sums(a, K)
    base = _channel_o2()
    s = oracle.OracleSim(base["mesh"], base["W0"], base["params"])
    for fun in (0, 1):
        got, phi = s.frozen_o2(fr, th, functional=fun, tags=[1])
        assert got == pytest.approx(J[fun], rel=1e-12, abs=1e-16)
        assert s.frozen_o2(fr, th, functional=fun, tags=[1], phi=phi)[0] == got
    # the limiter is active in these steps
    assert phi.min() < 0.9 and phi.max() > 0.999


def test_o2_map_with_zero_limiter_is_the_first_order_map(recorded_o2):
    cfg, s, fr = recorded_o2
    o1 = dict(cfg["params"], order=1)
    s1 = oracle.OracleSim(cfg["mesh"], cfg["W0"], o1)
    th = _theta0()
    zero = np.zeros((K, 6, len(cfg["mesh"]["tets"])))
    for fun in (0, 1):
        ref = s1.frozen_objective(fr, th, functional=fun, tags=[1])
        assert s.frozen_o2(fr, th, fun, [1], phi=zero)[0] == pytest.approx(ref[0], rel=1e-12)
        for k in range(3):
            h = 1e-5 * th[k]
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd = (s.frozen_o2(fr, tp, fun, [1], phi=zero)[0] - s.frozen_o2(fr, tm, fun, [1], phi=zero)[0]) / (2 * h)
            assert abs(fd - ref[1 + k]) <= 1e-6 * max(abs(ref[1 + k]), 1e-3 * np.abs(ref[1:]).max()), (k, fd, ref)


def test_o2_inactive_limiter_freezing_changes_no_derivative():
    cfg = _channel_o2()
    cfg["params"]["venkat_K"] = 1e4
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    s.step(2)
    fr = s.record_frozen(K)
    th = _theta0()
    J, phi = s.frozen_o2(fr, th, 0, [1])
    assert phi.min() > 1.0 - 1e-8
    frozen = s.frozen_o2_gradient(fr, th, 0, [1])
    for k in range(3):
        h = 1e-5 * th[k]
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        live = (s.frozen_o2(fr, tp, 0, [1])[0] - s.frozen_o2(fr, tm, 0, [1])[0]) / (2 * h)
        assert live == pytest.approx(frozen[1 + k], rel=1e-7, abs=1e-9 * np.abs(frozen[1:]).max())


def test_o2_central_differences_converge(recorded_o2):
    cfg, s, fr = recorded_o2
    th = _theta0()
    g = [s.frozen_o2_gradient(fr, th, 1, [1], rel_step=r)[1:] for r in (4e-3, 2e-3, 1e-5)]
    e1, e2 = np.abs(g[0] - g[2]), np.abs(g[1] - g[2])
    assert np.all(e2 < 0.35 * e1), (e1, e2)  # error ~ h^2 (ratio 1/4)
    assert np.all(np.abs(g[2]) > 0)
