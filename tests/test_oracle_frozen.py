"""Pins of the oracle's frozen-particle wave map and its reference gradient.

With the particle part of each step frozen (the recorded time steps, particle
densities and particle fluxes), a wall functional J(theta) of the wave fluxes
is a smooth function of theta = (rho_inf, U_inf, T_w).  The oracle evaluates
it generically in the scalar type: in binary64 it reproduces the wall fluxes
of the oracle's own steps, and its forward-mode dual-number derivative agrees
with central finite differences of the binary64 map.
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
