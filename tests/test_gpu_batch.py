"""Batched stepping, launch configurations and the autotuner on the GPU.

A batch captures every member's step pair into one CUDA graph; the members
must end bit for bit where they end when stepped alone (their kernels, random
streams and fixed-point sums are their own), and each member's batched step
must match the oracle's step teacher-forced from the same state.  Grid sizes
chosen by hand or by the autotuner change only the speed.
"""
import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import ugkwp, workloads as wl
from tests.test_gpu_parity import assert_particles_equal, compare_step

pytestmark = pytest.mark.gpu


def _members():
    return [
        wl.shock_tube(nx=40, ny=2, nz=2, precision="mixed", U=0.8),
        wl.cavity(n=6, N_ref=60, precision="mixed", order=2),
        wl.uniform_box(n=(3, 3, 3), Kn=0.5, N_ref=30, bc_type="specular", precision="fp64"),
        wl.cube_flow(h0=0.5, growth=2.0, N_ref=40, precision="mixed", Kn=0.1, order=2),
    ]


def _sim(cfg, stream=None):
    return ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=stream)


def _assert_same(a, b):
    sa, sb = a.state(), b.state()
    assert sa["step"] == sb["step"]
    np.testing.assert_array_equal(sa["W"], sb["W"])
    assert_particles_equal(sa, sb)


def test_batch_equals_members_stepped_alone():
    import torch
    cfgs = _members()
    batched = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    alone = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    b = ugkwp.Batch(batched)
    b.step(5)  # two graph-replayed pairs and one directly enqueued step
    b.sync()
    for s in alone:
        s.step(5)
    for x, y in zip(batched, alone):
        _assert_same(x, y)
    # a member stepped on its own after a sync continues consistently
    batched[1].step(2)
    alone[1].step(2)
    _assert_same(batched[1], alone[1])
    b.close()


def test_batched_step_matches_oracle():
    """One batched step of each member from the oracle's state, against the
    oracle's own step (teacher forcing, the single-simulation protocol)."""
    import torch
    cfgs = [wl.shock_tube(precision="fp64"), wl.cavity(n=6, N_ref=40, precision="mixed", order=2)]
    osims = [oracle.OracleSim(c["mesh"], c["W0"], c["params"]) for c in cfgs]
    gsims = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    for o, g in zip(osims, gsims):
        o.step(3)
        g.set_state(o.state())
    b = ugkwp.Batch(gsims)
    b.step(1)
    b.sync()
    for o, g in zip(osims, gsims):
        o.step()
        compare_step(g, o)
    b.close()


# tracking blocks (threads per tile) and carveouts that must give the results
# of the default configuration bit for bit
SHAPES = [(128, 58), (256, -1), (256, 86)]


@pytest.mark.parametrize("precision,K", [("mixed", 0), ("fp64", 0), ("mixed", 2)])
def test_launch_cfg_changes_only_speed(precision, K):
    """Odd grid sizes, tracking tiles of 128 or 256 particles and carveouts:
    the same states bit for bit as the default configuration."""
    import torch
    cfg = wl.cavity(n=6, N_ref=60, precision=precision, order=2, K=K)
    c = _sim(cfg, torch.cuda.Stream())
    c.step(4)
    for threads, carve in SHAPES:
        a = _sim(cfg, torch.cuda.Stream())
        d = ugkwp.ugkwp_get_launch_cfg(a.handle)
        assert d["particle_blocks"] > 0 and d["wave_blocks"] > 0
        ugkwp.ugkwp_set_launch_cfg(a.handle, 7, 3, threads, carve)   # odd grids on purpose
        assert ugkwp.ugkwp_get_launch_cfg(a.handle) == {"particle_blocks": 7, "wave_blocks": 3, "track_threads": threads,
                                                       "smem_carveout": carve}
        a.step(4)
        _assert_same(a, c)
        a.close()
    with pytest.raises(ugkwp.UgkwpError):
        ugkwp.ugkwp_set_launch_cfg(c.handle, 0, 1)
    for bad in ((8, 8, 64, -1), (8, 8, 128, 101), (8, 8, 128, -2)):
        with pytest.raises(ugkwp.UgkwpError):
            ugkwp.ugkwp_set_launch_cfg(c.handle, *bad)


def test_autotuner_picks_a_candidate_and_keeps_results():
    import torch
    cfg = wl.cavity(n=6, N_ref=60, precision="mixed", order=2)
    a, c = _sim(cfg, torch.cuda.Stream()), _sim(cfg, torch.cuda.Stream())
    best = ugkwp.ugkwp_autotune(a.handle, 2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert best["particle_blocks"] % sms == 0 and best["wave_blocks"] % sms == 0
    assert best["track_threads"] in (128, 256) and best["smem_carveout"] in (-1, 58)
    assert ugkwp.ugkwp_get_launch_cfg(a.handle) == best
    n = a.step(0, stats=True)["step"]
    # 4 block x carveout trials, then 5 grid trials at order 2; 2 warm-up + 2 timed steps each
    assert n == 9 * 4
    c.step(n)
    _assert_same(a, c)


def test_batch_autotune_and_member_errors():
    import torch
    cfgs = [wl.shock_tube(nx=40, ny=2, nz=2, precision="mixed", U=0.8, N_ref=100), _members()[1]]
    for c in cfgs:  # 38 steps: keep the tube physical (N_ref 100, energy-matched sampling)
        c["params"]["sampling"] = "energy_matched"
    sims = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    b = ugkwp.Batch(sims)
    best = b.autotune(2)
    assert best["particle_blocks"] > 0
    b.step(2)
    b.sync()
    b.close()
    # a member that overflows its particle capacity is reported by index
    bad = wl.shock_tube(nx=20, ny=2, nz=2)
    bad["params"]["particle_capacity"] = 1000
    sims2 = [_sim(cfgs[0], torch.cuda.Stream()), _sim(bad, torch.cuda.Stream())]
    b2 = ugkwp.Batch(sims2)
    b2.step(1)
    with pytest.raises(ugkwp.UgkwpError, match="batch member 1"):
        b2.sync()
    b2.close()


def test_fused_chunks_equal_members_stepped_alone():
    """Fifteen members of one kind (MIXED, second order): two fused chunks
    (13 and 2 members), each kernel one launch per chunk.  Uneven sizes and
    Knudsen numbers; every member ends bit for bit where it ends alone, after
    a graph-replayed pair and a direct step."""
    import torch
    cfgs = []
    for k in range(15):
        if k % 2:
            cfgs.append(wl.cavity(n=4 + k % 4, N_ref=40 + 5 * k, Kn=0.02 * (1 + k), precision="mixed", order=2,
                                  seed=100 + k))
        else:
            cfgs.append(wl.shock_tube(nx=12 + 3 * k, ny=2, nz=2, precision="mixed", order=2, U=0.1 * k,
                                      Kn=10.0 ** (-3 + k / 5), N_ref=60, seed=100 + k))
    for c in cfgs:
        c["params"]["sampling"] = "energy_matched"
    batched = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    alone = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    b = ugkwp.Batch(batched)
    b.step(3)
    b.sync()
    for s in alone:
        s.step(3)
    for x, y in zip(batched, alone):
        _assert_same(x, y)
    b.close()


def test_fused_chunk_with_pair_sampling_equals_members_stepped_alone():
    """Five cavities with the printed pair sampling (Sec. 2.4 (b)), one fused
    chunk: every member ends bit for bit where it ends alone, after two
    graph-replayed pairs and a direct step."""
    import torch
    cfgs = [wl.cavity(n=5 + k, N_ref=50 + 10 * k, Kn=0.075 * (1 + k), precision="mixed", order=2, seed=200 + k)
            for k in range(5)]
    batched = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    alone = [_sim(c, torch.cuda.Stream()) for c in cfgs]
    b = ugkwp.Batch(batched)
    b.step(5)
    b.sync()
    for s in alone:
        s.step(5)
    for x, y in zip(batched, alone):
        _assert_same(x, y)
    b.close()
