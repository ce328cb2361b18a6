"""The allocation-free time step against the oracle and the regular path.

ugkwp_time_step_noalloc serves callers that cannot allocate device memory
(their host application owns the GPU's memory, or allocation is not allowed
where they run): it reads device arrays the caller already has and keeps its
scratch in static device memory inside the library.  Given the same W, cell
volumes and projected areas, its result must equal the time step the oracle
takes from that state bit for bit, and so the one ugkwp_step takes from it.
The meshes run large, small, large in one process, two calls each, so that a
small call reads the shared scratch after a large call left more slots behind.
"""
import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import ugkwp, workloads as wl

pytestmark = pytest.mark.gpu


def _cases():
    # N_ref 60: at lower N_ref the sampling noise drives rarefied cells of the
    # cavity to negative pressure within a few steps
    return [("cavity 12^3 (10,368 cells)", wl.cavity(n=12, N_ref=60, precision="mixed")),
            ("shock tube 30x2x2 (720 cells)", wl.shock_tube(nx=30, ny=2, nz=2, N_ref=60)),
            ("cavity 12^3 again", wl.cavity(n=12, N_ref=60, precision="mixed"))]


def test_noalloc_time_step_equals_oracle_and_step():
    import torch

    d_dt = torch.empty(1, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream().cuda_stream
    for name, cfg in _cases():
        osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
        gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
        vol = osim.geometry("vol")
        dS = osim.geometry("dS")
        d_vol = torch.tensor(vol, device="cuda", dtype=torch.float64)
        d_dS = torch.tensor(dS, device="cuda", dtype=torch.float64).contiguous()
        for call in range(2):
            osim.step(1)
            st = osim.state()                      # the state the next step starts from
            osim.step(1)
            dt_ref = osim.last("dt")               # the oracle's time step from st["W"]
            gsim.set_state(st)
            gsim.step(1)
            assert gsim.last("dt") == dt_ref, (name, call)
            d_W = torch.tensor(st["W"], device="cuda", dtype=torch.float64).contiguous()
            d_dt.fill_(float("nan"))
            ugkwp.ugkwp_time_step_noalloc(d_W.data_ptr(), d_vol.data_ptr(), d_dS.data_ptr(), gsim.n_cells,
                                          cfg["params"]["R"], cfg["params"]["CFL"], d_dt.data_ptr(), stream)
            torch.cuda.synchronize()
            dt = float(d_dt.item())
            assert dt == dt_ref, (name, call, dt, dt_ref)
        gsim.close()


def test_noalloc_rejects_oversized_input():
    with pytest.raises(ugkwp.UgkwpError) as e:
        ugkwp.ugkwp_time_step_noalloc(1 << 20, 1 << 20, 1 << 20, ugkwp.NOALLOC_MAX_CELLS + 1, 1.0, 0.5, 1 << 20)
    assert e.value.code == ugkwp.E_ARG
