"""Time averaging (Sec. 2.4 (c)) and the gradient-length local Knudsen number
on the GPU.

* W-bar after averaged steps equals sum dt^n W^n / sum dt^n formed on the host
  from the states and time steps read after each step, and graph-replayed
  steps give the same average as single steps;
* Kn_GLL = l |grad rho| / rho agrees with the value formed from the oracle's
  unlimited least-squares gradient of rho and the VHS mean free path.
"""
import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import ugkwp, workloads as wl

pytestmark = pytest.mark.gpu


def test_time_average_matches_its_definition():
    import torch
    cfg = wl.cavity(n=6, N_ref=60, precision="mixed", order=2)
    a = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    b = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    a.step(3)
    b.step(3)
    with pytest.raises(ugkwp.UgkwpError):
        a.moments(ugkwp.WBAR)          # nothing averaged yet
    ugkwp.ugkwp_average(a.handle, True)
    ugkwp.ugkwp_average(b.handle, True)
    S, T = 0.0, 0.0
    for _ in range(5):
        a.step(1)
        dt = a.last("dt")
        S = S + dt * a.moments(ugkwp.W)
        T += dt
    b.step(5)                          # two graph-replayed pairs and one step
    Wa, Wb = a.moments(ugkwp.WBAR), b.moments(ugkwp.WBAR)
    np.testing.assert_allclose(Wa, S / T, rtol=1e-14, atol=0)
    np.testing.assert_array_equal(Wa, Wb)
    assert ugkwp.ugkwp_average_time(a.handle) == pytest.approx(T, rel=1e-15)
    ugkwp.ugkwp_average(a.handle, False)   # stop: the sums stay
    a.step(2)
    np.testing.assert_array_equal(a.moments(ugkwp.WBAR), Wa)


@pytest.mark.parametrize("bc", ["specular", "farfield"])
def test_kn_gll_matches_oracle_gradient(bc):
    cfg = wl.cube_flow(h0=0.5, growth=2.0, N_ref=20, precision="mixed", Kn=0.1) if bc == "farfield" else \
        wl.shock_tube(nx=40, ny=2, nz=2, precision="mixed")
    o = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    o.step(2)
    st = o.state()
    g = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    g.set_state(st)
    kn = ugkwp.ugkwp_kn_gll(g.handle, g.n_cells)
    o.prepare()
    gW, _ = o.gradients(limited=False)
    W = st["W"]
    rho = W[0]
    U2 = (W[1:4] ** 2).sum(0) / rho ** 2
    p = (W[4] - 0.5 * rho * U2) / 1.5
    P = cfg["params"]
    T = p / (rho * P["R"])
    mu = P["mu_ref"] * (T / P["T_ref"]) ** P["omega"]
    w = P["omega"]
    lmfp = 2 * (5 - 2 * w) * (7 - 2 * w) / 15 * mu / (rho * np.sqrt(2 * np.pi * P["R"] * T))
    ref = lmfp * np.linalg.norm(gW[0], axis=0) / rho
    np.testing.assert_allclose(kn, ref, rtol=1e-9, atol=1e-12 * ref.max())
    assert ref.max() > 0
