"""Hand-written adjoint of the frozen-particle wave map on the GPU.

From a common state, the GPU call (K real steps recorded, frozen forward,
reverse sweep) is compared with the oracle's reference (its own K steps
recorded, the same map evaluated on forward-mode dual numbers), with central
finite differences of the GPU's own frozen map, and through the PyTorch
autograd wrapper.
"""
import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import ugkwp, workloads as wl

pytestmark = pytest.mark.gpu

K = 3


def _theta0():
    return np.array([1.0, 0.5 * np.sqrt(5.0 / 3.0), 1.0])


def _setup(precision):
    import torch
    cfg = wl.wall_channel(precision=precision)
    g = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    g.step(2)
    return cfg, g, g.state()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("functional", [0, 1])
def test_adjoint_matches_oracle_reference(precision, functional):
    cfg, g, st = _setup(precision)
    out = g.adjoint(functional, K, [1])
    o = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    o.set_state(st)
    ref = o.frozen_objective(o.record_frozen(K), _theta0(), functional=functional, tags=[1])
    assert out[0] == pytest.approx(ref[0], rel=1e-10)
    scale = np.abs(ref[1:]).max()
    for k in range(3):
        assert abs(out[1 + k] - ref[1 + k]) <= 1e-6 * max(abs(ref[1 + k]), 1e-3 * scale), (k, out, ref)


def test_adjoint_matches_gpu_finite_differences():
    cfg, g, st = _setup("fp64")
    th = _theta0()
    g.set_state(st)
    out = g.adjoint(0, K, [1], th)
    for k in range(3):
        h = 1e-5 * th[k]
        J = []
        for sgn in (1.0, -1.0):
            t = th.copy()
            t[k] += sgn * h
            g.set_state(st)  # the same recorded particle data for every evaluation
            J.append(g.adjoint(0, K, [1], t)[0])
        fd = (J[0] - J[1]) / (2 * h)
        assert abs(out[1 + k] - fd) <= 1e-6 * max(abs(out[1 + k]), 1e-3 * np.abs(out[1:]).max()), (k, out, fd)


def test_autograd_wrapper_and_order2_refusal():
    import torch
    cfg, g, st = _setup("mixed")
    theta = torch.tensor(_theta0(), dtype=torch.float64, requires_grad=True)
    J = ugkwp.wall_functional(theta, g, 1, K, [1])
    J.backward()
    g.set_state(st)
    out = g.adjoint(1, K, [1], _theta0())
    assert float(J.detach()) == pytest.approx(out[0], rel=1e-12)
    np.testing.assert_allclose(theta.grad.numpy(), out[1:], rtol=1e-12)
    o2 = wl.wall_channel(precision="mixed", order=2)
    g2 = ugkwp.Simulation(o2["mesh"], o2["W0"], o2["params"])
    with pytest.raises(ugkwp.UgkwpError) as e:
        g2.adjoint(0, 1, [1])
    assert e.value.code == ugkwp.E_UNSUPPORTED
