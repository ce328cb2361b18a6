"""The allocation-free time step against the regular path.

ugkwp_time_step_noalloc serves callers that cannot allocate device memory
(their host application owns the GPU's memory, or allocation is not allowed
where they run): it reads device arrays the caller already has and keeps its
scratch in static device memory inside the library.  Its result must match the
time step that ugkwp_step computed from the same state (read back with
ugkwp_last), within the tolerance of the parity tests, on two calls in a row
that share the static scratch.
"""
import numpy as np
import pytest

from paper_2007_13091_gb300 import ugkwp, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _volumes_and_projected_areas(nodes, tets):
    p = nodes[tets]
    vol = np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0])) / 6.0
    dS = np.zeros((3, len(tets)))
    for k in range(4):
        a, b, c = (p[:, j] for j in range(4) if j != k)
        S = 0.5 * np.cross(b - a, c - a)  # area vector of the face opposite node k
        dS += 0.5 * np.abs(S).T
    return vol, dS


@pytest.mark.parametrize("case", ["shock_tube", "cavity"])
def test_noalloc_time_step_matches_step(case):
    import torch

    cfg = wl.shock_tube(nx=30, ny=2, nz=2, N_ref=20) if case == "shock_tube" else \
        wl.cavity(n=6, N_ref=20, precision="mixed")
    sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    vol, dS = _volumes_and_projected_areas(cfg["mesh"]["nodes"], cfg["mesh"]["tets"])
    d_vol = torch.tensor(vol, device="cuda", dtype=torch.float64)
    d_dS = torch.tensor(dS, device="cuda", dtype=torch.float64).contiguous()
    d_dt = torch.empty(1, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        sim.step(1)
        Wn = sim.moments(ugkwp.W)             # state the next step starts from
        sim.step(1)
        dt_ref = sim.last("dt")               # the step's own time step from Wn
        d_W = torch.tensor(Wn, device="cuda", dtype=torch.float64).contiguous()
        d_dt.fill_(float("nan"))
        ugkwp.ugkwp_time_step_noalloc(d_W.data_ptr(), d_vol.data_ptr(), d_dS.data_ptr(), sim.n_cells,
                                      cfg["params"]["R"], cfg["params"]["CFL"], d_dt.data_ptr(), stream)
        torch.cuda.synchronize()
        dt = float(d_dt.item())
        assert abs(dt - dt_ref) <= TOL * dt_ref, (call, dt, dt_ref)
    sim.close()


def test_noalloc_rejects_oversized_input():
    with pytest.raises(ugkwp.UgkwpError) as e:
        ugkwp.ugkwp_time_step_noalloc(1 << 20, 1 << 20, 1 << 20, ugkwp.NOALLOC_MAX_CELLS + 1, 1.0, 0.5, 1 << 20)
    assert e.value.code == ugkwp.E_ARG
