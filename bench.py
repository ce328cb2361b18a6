"""Benchmark of the UGKWP step on one GB300 (one JSON line on stdout).

Workload: the lid-driven cubic cavity (24^3 hexes x 6 = 82,944 tets, argon-like
VHS gas, Kn 0.075, diffuse walls, lid Mach 0.16, 100 reference particles per
cell, ~8.3e6 particles), MIXED precision (binary32 particles, binary64 cells,
int64 fixed-point particle flux).  A step is one full UGKWP time step.

  value      particle-moves/s, device time (CUDA events on the library's stream)
  roofline   the tracking kernel (a6-a9) against the measured HBM copy bandwidth
  fp64       the same workload with binary64 particles
  field_error MIXED vs FP64 after a fixed number of steps, with the Monte-Carlo
             noise floor (two FP64 runs with different seeds)
  e2e        per step: state import from host buffers, step, W back to host
  batched    64 independent instances in one graph, MIXED and FP64; 8 copies of
             the cavity as one batch against one of them stepped alone
  adjoint    the frozen-particle wave adjoint on a channel
  gks_start_up the particle-free start-up steps, global and local time steps
  gp1_sampling the workload with first-order g_p sampling
  diatomic   the workload with K = 2 internal degrees of freedom
  cpu_baseline the CPU oracle (single thread) on a bounded sample

Multi-GPU: replicas only (each rank runs its own simulation; value = all
ranks' moves / max time).  --impl reference times the CPU oracle instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-moves/s & cell-steps/s on 1 GB300: mixed vs FP64 at fixed error"
UNIT = "particle-moves/s"
# minimum bytes the tracking kernel moves (MIXED / FP64): read the particle
# record (x, u, m, cell, id) and write it (compacted) for the next step
TRACK_BYTES_PER_MOVE = {"mixed": 44 + 44, "fp64": 68 + 68}
# per cell and step: tracking record (planes + neighbours) and tau
TRACK_BYTES_PER_CELL = {"mixed": 80 + 8, "fp64": 144 + 8}
# DRAM bytes (read + write) of the tracking phase of one step (both k_track
# launches) on this workload, from the ncu capture summarised in
# profiles/k_track_cavity24_mixed.md; set to None whenever the
# kernel changes until it is captured again
TRACK_DRAM_BYTES = {"mixed": 1229627648 + 1073300224 + 48128, "fp64": None}
# bytes the movers' flux kernel reads per mover (start and end velocity, mass,
# start cell, end cell and exit flag), MIXED / FP64
MOVER_BYTES = {"mixed": 12 + 12 + 8 + 4 + 8, "fp64": 24 + 24 + 8 + 4 + 8}
# int64 atomic additions per mover: -phi at the start cell, +phi at the end cell
MOVER_ATOMICS = 10
# binary64 pipe operations of one phi = m (1, u, |u|^2/2): MIXED 3 widenings,
# 7 products and 3 sums; FP64 the products and sums
MOVER_FP64_OPS = {"mixed": 13, "fp64": 10}
# Binary64 flops per interior face of k_face_flux_o2 (the second-order wave flux):
# ncu's executed dadd + dmul + 2 dfma per launch divided by the interior faces, on
# this workload (profiles/); None until captured for the current kernel.
# (the kernel also takes the boundary faces' first-order flux after the
# interior faces: their flops are included, counted per interior face)
FLUX_O2_FLOPS_PER_FACE = (29934208 + 80965504 + 2 * 148104192) / 162432
FLUX_O2_DRAM_BYTES = 31148800 + 512
# FP64 peak: 2 FP64 FMA lanes per clock per SM (the nominal 1.25 TFLOP/s of this
# part at 152 SMs and 2.07 GHz), 2 flops per FMA
FP64_FMA_LANES_PER_SM = 2


def guarded(fn):
    """An extra measurement; its failure is reported in its place instead of
    ending the run (the device error words of its own simulations only)."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def fp64_peak_measured(n=8192, reps=5):
    """Binary64 throughput of this GPU measured as a cuBLAS DGEMM (2 n^3 flops)
    timed with CUDA events, best of `reps` (TFLOP/s)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The cavity's particle population grows from N_ref per cell at the start (each
# rarefied cell samples at least one pair per step) until collisions balance
# it, ~2.6 N_ref per cell after ~500 steps; the timed steps start from that
# settled state, which the 2,000-step run spends most of its time in.
SPIN_UP = 500

# reconstruction order of the workload (2: least-squares gradients with
# Venkatakrishnan's limiter, the scheme of the paper's cavity; --order 1 for zero slopes)
ORDER = 2


def workload(precision, seed=None):
    from paper_2007_13091_gb300 import workloads as wl
    cfg = wl.cavity(n=24, Kn=0.075, N_ref=100, precision=precision, order=ORDER)
    if seed is not None:
        cfg["params"]["seed"] = seed
    return cfg


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, busy_fraction_min=0.0):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                if self.uuid and parts[0] != self.uuid:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def reduce_max(x, ws):
    """Maximum over the ranks (the slowest replica sets the job's time)."""
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.MAX) if ws > 1 else x


def reduce_sum(x, ws):
    """Sum over the ranks (work of all replicas)."""
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.SUM) if ws > 1 else x


def job_rates(ms, moves, cells, steps, ws):
    """Whole-job rates of independent replicas: every rank's moves and
    cell-steps over the slowest rank's time."""
    ms_max = reduce_max(ms, ws)
    return ms_max, reduce_sum(moves, ws) / (ms_max * 1e-3), reduce_sum(cells * steps, ws) / (ms_max * 1e-3)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def time_steps(sim, steps, warmup, ws, timing=True):
    """Device time of `steps` steps after `warmup` (the production path: steps
    replayed as CUDA graphs, no per-kernel events), then, if `timing`, the
    per-kernel CUDA-event durations over `steps` further steps.
    Returns (ms, moves, launches, kernel ms per step-sum, stats)."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    sim.step(warmup)
    st0 = sim.step(0, stats=True)
    _, l0 = ugkwp.ugkwp_timing_read(sim.handle)
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    sim.step(steps)
    e1.record(sim.stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    _, l1 = ugkwp.ugkwp_timing_read(sim.handle)
    st1 = sim.step(0, stats=True)
    moves = st1["n_moves_total"] - st0["n_moves_total"]
    launches = sum(l1.values()) - sum(l0.values())
    kms = None
    if timing:
        ugkwp.ugkwp_timing_enable(sim.handle, True)
        sim.step(steps)
        ugkwp.ugkwp_timing_enable(sim.handle, False)
        kms, _ = ugkwp.ugkwp_timing_read(sim.handle)
        st2 = sim.step(0, stats=True)
        kms["_moves"] = st2["n_moves_total"] - st1["n_moves_total"]
    return ms, moves, launches, kms, st1


def field_error(horizons, device):
    """Per-field relative L2 of MIXED vs FP64 after each of `horizons` steps from
    the same initial state and seed, and the FP64 seed-to-seed noise floor."""
    from paper_2007_13091_gb300 import ugkwp

    first = {}

    def prims(precision, seed):
        cfg = workload(precision, seed)
        sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device)
        out, done = {}, 0
        for h in horizons:
            sim.step(h - done)
            done = h
            P = sim.moments(ugkwp.PRIM)
            rho, U, T = P[0], P[1:4], P[4]
            out[h] = {"rho": rho, "U": U, "T": T, "p": rho * T}
            if h == 1 and seed == 2:
                st = sim.state()
                first[precision] = (st["id"], st["cell"])
        sim.close()
        return out

    a, b, c = prims("mixed", 2), prims("fp64", 2), prims("fp64", 1002)

    def rel(x, y):
        return float(np.linalg.norm(x - y) / np.linalg.norm(y))
    # velocity error relative to the lid speed scale (the cavity starts at rest)
    ulid = 0.16 * math.sqrt(5.0 / 3.0)
    uerr = lambda x, y: float(np.linalg.norm(x - y) / (ulid * math.sqrt(y.shape[1])))
    res = {}
    for h in horizons:
        err = {k: rel(a[h][k], b[h][k]) for k in ("rho", "T", "p")}
        err["U"] = uerr(a[h]["U"], b[h]["U"])
        floor = {k: rel(c[h][k], b[h][k]) for k in ("rho", "T", "p")}
        floor["U"] = uerr(c[h]["U"], b[h]["U"])
        res[str(h)] = {"mixed_vs_fp64": err, "noise_floor_fp64_seed": floor}
    out = {"horizons": list(horizons), "by_horizon": res}
    if "mixed" in first and "fp64" in first:
        # the discrete decisions behind the error: after one step from the same
        # state and seed, particles whose cell differs between the two
        # precisions, and particles that exist in one only (t_f or exit decisions)
        (ia, ca), (ib, cb) = first["mixed"], first["fp64"]
        common, ja, jb = np.intersect1d(ia, ib, assume_unique=True, return_indices=True)
        moved = int((ca[ja] != cb[jb]).sum())
        out["after_1_step_particles"] = {"fp64": int(ib.size), "mixed": int(ia.size), "common_ids": int(common.size),
                                         "cell_differs": moved, "only_in_fp64": int(ib.size - common.size),
                                         "only_in_mixed": int(ia.size - common.size),
                                         "differing_per_particle": (moved + (ib.size - common.size) +
                                                                    (ia.size - common.size)) / max(ib.size, 1)}
    return out


def field_error_averaged(device, spin=300, avg=600):
    """The steady cavity's time-averaged fields (the paper's averaging of
    Sec. 2.4 (c), over `avg` steps after `spin` steps): per-field relative L2
    of MIXED vs FP64 at the same seed, and the FP64 seed-to-seed floor of the
    same averages."""
    from paper_2007_13091_gb300 import ugkwp

    def averaged(precision, seed):
        cfg = workload(precision, seed)
        sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device)
        sim.step(spin)
        ugkwp.ugkwp_average(sim.handle, True)
        sim.step(avg)
        Wb = sim.moments(ugkwp.WBAR)
        sim.close()
        rho = Wb[0]
        U = Wb[1:4] / rho
        p = (Wb[4] - 0.5 * rho * (U * U).sum(0)) / 1.5
        return {"rho": rho, "U": U, "T": p / rho, "p": p}

    a, b, c = averaged("mixed", 2), averaged("fp64", 2), averaged("fp64", 1002)
    ulid = 0.16 * math.sqrt(5.0 / 3.0)

    def err(x, y):
        e = {k: float(np.linalg.norm(x[k] - y[k]) / np.linalg.norm(y[k])) for k in ("rho", "T", "p")}
        e["U"] = float(np.linalg.norm(x["U"] - y["U"]) / (ulid * math.sqrt(y["U"].shape[1])))
        return e
    return {"spin_up_steps": spin, "averaged_steps": avg, "mixed_vs_fp64": err(a, b),
            "noise_floor_fp64_seed": err(c, b)}


def e2e(cfg, steps, device, launch_cfg=None):
    """Per step through the C-ABI with host buffers: import the state from host
    arrays, one step, read W back to host memory (at `launch_cfg`, the launch
    configuration a user sets once, if given).  The state goes in as the
    native image (particles in the simulation's own precision, the checkpoint
    form) and, in a second loop, as the binary64 image."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device,
                           stream=torch.cuda.Stream(device=device))
    if launch_cfg is not None:
        ugkwp.ugkwp_set_launch_cfg(sim.handle, launch_cfg["particle_blocks"], launch_cfg["wave_blocks"],
                                   launch_cfg["track_threads"], launch_cfg["smem_carveout"])
    sim.step(SPIN_UP)

    def pinned(a):
        """The array in page-locked host memory (as a user feeding the GPU keeps it)."""
        b = torch.empty(max(a.nbytes, 1), dtype=torch.uint8, pin_memory=True).numpy()[:a.nbytes]
        out = b.view(a.dtype).reshape(a.shape)
        out[...] = a
        return out

    def loop(state, load):
        state = {k: (pinned(v) if isinstance(v, np.ndarray) and v.size else v) for k, v in state.items()}
        h2d = sum(state[k].nbytes for k in ("W", "id", "cell", "x", "u", "m"))
        # one untimed round: the first binary64 import allocates its device staging
        load(state)
        sim.step(1)
        torch.cuda.synchronize()
        moves = 0
        t_load = 0.0
        t0 = time.perf_counter()
        for _ in range(steps):
            a = time.perf_counter()
            load(state)
            t_load += time.perf_counter() - a
            st = sim.step(1, stats=True)
            moves += st["n_tracked"]
            sim.moments(ugkwp.W)
        t1 = time.perf_counter()
        return moves / (t1 - t0), (t1 - t0) * 1e3 / steps, h2d, state["id"].size, t_load * 1e3 / steps

    native = sim.state_native()
    wide = sim.state()
    v_nat, ms_nat, h2d_nat, n, imp_nat = loop(native, sim.set_state_native)
    v_wide, ms_wide, h2d_wide, _, imp_wide = loop(wide, sim.set_state)
    d2h = 5 * sim.n_cells * 8
    sim.close()
    return {"value": v_nat, "unit": UNIT, "h2d_bytes_per_step": int(h2d_nat), "d2h_bytes_per_step": int(d2h),
            "steps": steps, "particles": int(n), "ms_per_step": ms_nat, "import_ms_per_step": imp_nat,
            "launch_cfg": launch_cfg,
            "per_step": "ugkwp_import_state_native of the whole state from page-locked host arrays (particles "
                        "in the simulation's precision: binary32 offsets from the tets' anchors, binary32 "
                        "velocities; copied as they are and checked on the device), one step, W read back to "
                        "host memory",
            "binary64_image": {"value": v_wide, "unit": UNIT, "ms_per_step": ms_wide, "import_ms_per_step": imp_wide,
                               "h2d_bytes_per_step": int(h2d_wide), "d2h_bytes_per_step": int(d2h),
                               "per_step": "ugkwp_import_state of the binary64 image (copied as it is, checked "
                                           "and converted to the particle precision on the device), one step, "
                                           "W read back to host memory"}}


def batched(precision, steps, warmup, device):
    """The batched form: 64 independent shock tubes and cavities of 2k-60k tets,
    Kn log-uniform in [1e-4, 1], Mach in [0.1, 3], stepped as one CUDA graph per
    step pair after the batch autotuner picked the grid sizes."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl
    # capacity 4 N_ref per cell: in rarefied cells the printed pair count adds at
    # least one pair per cell and step, so the population grows by ~2 per cell
    # and step until collisions balance it
    cases = wl.batch_instances(precision=precision, order=ORDER, cap_factor=4.0)
    sims = [ugkwp.Simulation(c["mesh"], c["W0"], c["params"], device=device, stream=torch.cuda.Stream(device=device))
            for c in cases]
    b = ugkwp.Batch(sims)
    best = b.autotune(2)
    b.step(warmup)
    b.sync()
    m0 = sum(s.step(0, stats=True)["n_moves_total"] for s in sims)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    b.sync()
    ms = e0.elapsed_time(e1)
    m1 = sum(s.step(0, stats=True)["n_moves_total"] for s in sims)
    n_cells = sum(s.n_cells for s in sims)
    b.close()
    for s in sims:
        s.close()
    return {"value": (m1 - m0) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "instances": len(cases),
            "n_cells": n_cells, "particles_per_step": (m1 - m0) / steps,
            "cell_steps_per_s": n_cells * steps / (ms * 1e-3), "launch_cfg": best,
            "workload": "64 instances (even: shock tubes moving at Mach M, N_ref 50; odd: cavities with lid "
                        "Mach M, N_ref 100), 2k-60k tets each, Kn log-uniform [1e-4, 1], M uniform [0.1, 3], "
                        f"seed 4, order {ORDER}, {precision}"}


def batched_cavities(steps, warmup, device, members=8, n=24, spin_up=500):
    """The batch with the single instance's work per member: `members` copies
    of the bench's cavity (n^3 x 6 tets, Kn 0.075, N_ref 100, MIXED, the
    printed pair sampling of Sec. 2.4 (b)) with seeds 2, 3, ...; stepped as one
    batch for `spin_up` steps (the population settles), autotuned and timed.
    Beside it, member 0 stepped alone from the state the batch left it in,
    autotuned and timed the same way: the batch's moves/s over its members'
    own."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl
    cases = [wl.cavity(n=n, N_ref=100, precision="mixed", order=ORDER, seed=2 + k) for k in range(members)]
    sims = [ugkwp.Simulation(c["mesh"], c["W0"], c["params"], device=device, stream=torch.cuda.Stream(device=device))
            for c in cases]
    b = ugkwp.Batch(sims)
    b.step(spin_up)
    b.sync()
    best = b.autotune(2)
    b.step(warmup)
    b.sync()
    m0 = sum(s.step(0, stats=True)["n_moves_total"] for s in sims)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    b.sync()
    ms = e0.elapsed_time(e1)
    m1 = sum(s.step(0, stats=True)["n_moves_total"] for s in sims)
    n_cells = sum(s.n_cells for s in sims)
    b.close()
    for s in sims[1:]:
        s.close()
    solo = sims[0]
    cfg1 = ugkwp.ugkwp_autotune(solo.handle, 4)
    ms1, mv1, _, _, _ = time_steps(solo, steps, warmup, 1, timing=False)
    solo.close()
    value = (m1 - m0) / (ms * 1e-3)
    one = mv1 / (ms1 * 1e-3)
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "instances": members, "n_cells": n_cells,
            "particles_per_step": (m1 - m0) / steps, "cell_steps_per_s": n_cells * steps / (ms * 1e-3),
            "launch_cfg": best, "sampling": "pairs (printed)",
            "member_alone": {"value": one, "unit": UNIT, "ms_per_step": ms1 / steps,
                             "particles_per_step": mv1 / steps, "launch_cfg": cfg1},
            "batch_over_member_alone": value / one,
            "workload": f"{members} lid-driven cavities {n}^3 hexes x 6 = {6 * n ** 3} tets each "
                        f"({n_cells} tets in all), Kn 0.075, N_ref 100, lid Mach 0.16, order {ORDER}, MIXED, "
                        f"printed pair sampling, seeds 2-{1 + members}, timed after {spin_up} spin-up steps"}


def batched_pairs(steps, warmup, device, launch_cfg):
    """The MIXED batch with the printed pair sampling (Sec. 2.4 (b)) instead of
    the energy-matched option, timed over `steps` steps after `warmup` from the
    start with the given launch configuration (no autotuner trials, so that it
    runs before the rarefied moving tubes fail); a device error ends it and is
    reported with the steps done."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl
    cases = wl.batch_instances(precision="mixed", order=ORDER, cap_factor=4.0, sampling="maxwell")
    sims = [ugkwp.Simulation(c["mesh"], c["W0"], c["params"], device=device, stream=torch.cuda.Stream(device=device))
            for c in cases]
    for s in sims:
        ugkwp.ugkwp_set_launch_cfg(s.handle, launch_cfg["particle_blocks"], launch_cfg["wave_blocks"],
                                   launch_cfg["track_threads"], launch_cfg["smem_carveout"])
    b = ugkwp.Batch(sims)
    out = {"sampling": "pairs (printed)", "warmup": warmup}
    try:
        b.step(warmup)
        b.sync()
        m0 = sum(s.step(0, stats=True)["n_moves_total"] for s in sims)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.step(steps)
        e1.record(b.stream)
        b.sync()
        ms = e0.elapsed_time(e1)
        m1 = sum(s.step(0, stats=True)["n_moves_total"] for s in sims)
        out.update({"value": (m1 - m0) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
                    "particles_per_step": (m1 - m0) / steps})
    except ugkwp.UgkwpError as e:
        out["error"] = str(e)[:200]
    b.close()
    for s in sims:
        s.close()
    return out


def batched_field_error(device, steps=10):
    """The batch's MIXED vs FP64 field error: both batches (energy-matched, the
    bench's sampling) from the initial states and seeds, `steps` steps, per
    field relative L2 over all members' cells, with the FP64 seed-to-seed
    noise floor (every member's seed + 1)."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl

    def fields(precision, seed_shift):
        cases = wl.batch_instances(precision=precision, order=ORDER, cap_factor=4.0)
        for c in cases:
            c["params"]["seed"] += seed_shift
        sims = [ugkwp.Simulation(c["mesh"], c["W0"], c["params"], device=device,
                                 stream=torch.cuda.Stream(device=device)) for c in cases]
        b = ugkwp.Batch(sims)
        b.step(steps)
        b.sync()
        P = [s.moments(ugkwp.PRIM) for s in sims]
        b.close()
        for s in sims:
            s.close()
        P = np.concatenate(P, axis=1)
        return {"rho": P[0], "T": P[4], "p": P[0] * P[4]}

    a, b, c = fields("mixed", 0), fields("fp64", 0), fields("fp64", 1)

    def err(x, y):
        return {k: float(np.linalg.norm(x[k] - y[k]) / np.linalg.norm(y[k])) for k in ("rho", "T", "p")}
    return {"after_steps": steps, "mixed_vs_fp64": err(a, b), "noise_floor_fp64_seed": err(c, b)}


def adjoint(device, K=10):
    """The hand-written adjoint of the frozen-particle wave map (first order):
    gradient of the drag on the side walls of a channel with respect to
    (rho_inf, U_inf, T_w) over K steps; time of one call (K real steps recorded,
    frozen forward, reverse sweep)."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl
    cfg = wl.wall_channel(n=(40, 20, 20), size=(1.0, 0.5, 0.5), N_ref=60, precision="mixed")
    cfg["params"]["sampling"] = "energy_matched"
    sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=torch.cuda.Stream(device=device))
    sim.step(2)
    sim.adjoint(0, K, [1])  # warm-up
    t0 = time.perf_counter()
    out = sim.adjoint(0, K, [1])
    t1 = time.perf_counter()
    n = sim.n_cells
    sim.close()
    return {"workload": "channel 40x20x20 hexes x 6 = 96,000 tets, Mach 0.5 far field, diffuse side walls, "
                        "Kn 0.05, N_ref 60, energy-matched sampling, MIXED, first order", "n_cells": n, "steps": K,
            "ms_per_call": 1e3 * (t1 - t0), "J_and_grad": [float(v) for v in out],
            "cell_steps_per_s": n * K / (t1 - t0)}


def gp1_sampling(device, steps, warmup, launch_cfg):
    """The bench workload with first-order g_p sampling (every hydrodynamic
    particle drawn by acceptance-rejection from its cell's g_p) after 200
    spin-up steps, timed like the main line with the main line's grid sizes."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    cfg = workload("mixed")
    cfg["params"]["sampling"] = "gp1"
    sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=torch.cuda.Stream(device=device))
    ugkwp.ugkwp_set_launch_cfg(sim.handle, **launch_cfg)
    sim.step(200)
    ms, moves, _, kms, _ = time_steps(sim, steps, warmup, 1)
    sim.close()
    kms.pop("_moves", None)
    return {"value": moves / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "kernels_ms_per_step": {k: v / steps for k, v in kms.items()},
            "workload": "cavity 24^3, MIXED, order 2, sampling gp1, 200 spin-up steps"}


def diatomic(device, steps, warmup, launch_cfg):
    """The bench workload for a diatomic gas (K = 2 internal degrees of freedom:
    particles carry an internal energy, 4 more bytes per particle record in
    MIXED) after 200 spin-up steps, timed like the main line with its grid sizes."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl
    cfg = wl.cavity(n=24, Kn=0.075, N_ref=100, precision="mixed", order=ORDER, K=2)
    sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=torch.cuda.Stream(device=device))
    ugkwp.ugkwp_set_launch_cfg(sim.handle, **launch_cfg)
    sim.step(200)
    ms, moves, _, kms, _ = time_steps(sim, steps, warmup, 1)
    sim.close()
    kms.pop("_moves", None)
    return {"value": moves / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "kernels_ms_per_step": {k: v / steps for k, v in kms.items()},
            "workload": "cavity 24^3, MIXED, order 2, K = 2 (diatomic), 200 spin-up steps"}


def shock_tube(device, steps=20, warmup=3, seeds=(1, 1002), oracle_steps=20):
    """The 3D shock tube at full size (100x4x4 hexes x 6 = 9,600 tets, Sod
    states, Kn 1e-2, N_ref 50, specular side walls, CFL 0.5, first order,
    seed 1): `steps` steps in FP64 and in MIXED, device time over the whole
    run from the initial state (the workload is those 20 steps, so nothing is
    spun up; `warmup` steps of a separate simulation come first to load the
    library's kernels and graphs), the per-field relative L2 of MIXED vs FP64
    after the run with the FP64 seed-to-seed floor, and the CPU oracle over the
    same `oracle_steps` steps."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl
    out = {"workload": "3D shock tube [0,1]x[0,0.04]^2, 100x4x4 hexes x 6 = 9,600 tets, Sod states, Kn 1e-2, "
                       "N_ref 50, specular side walls, CFL 0.5, first order, seed 1", "steps": steps}
    fields = {}
    for precision, seed in (("fp64", seeds[0]), ("mixed", seeds[0]), ("fp64", seeds[1])):
        cfg = wl.shock_tube(precision=precision, seed=seed)
        stream = torch.cuda.Stream(device=device)
        w = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=stream)
        w.step(warmup)
        w.sync()
        w.close()
        sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=stream)
        st0 = sim.step(0, stats=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        st1 = sim.step(0, stats=True)
        P = sim.moments(ugkwp.PRIM)
        fields[(precision, seed)] = {"rho": P[0], "U": P[1:4], "T": P[4], "p": P[0] * P[4]}
        moves = st1["n_moves_total"] - st0["n_moves_total"]
        if seed == seeds[0]:
            out[precision] = {"value": moves / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                              "cell_steps_per_s": sim.n_cells * steps / (ms * 1e-3),
                              "particles_per_step": moves / steps}
        sim.close()
    ref, mix, other = fields[("fp64", seeds[0])], fields[("mixed", seeds[0])], fields[("fp64", seeds[1])]
    # velocity relative to the sound speed of the left state (the tube starts at rest)
    c_left = math.sqrt(5.0 / 3.0)

    def err(x, y):
        e = {k: float(np.linalg.norm(x[k] - y[k]) / np.linalg.norm(y[k])) for k in ("rho", "T", "p")}
        e["U"] = float(np.linalg.norm(x["U"] - y["U"]) / (c_left * math.sqrt(y["U"].shape[1])))
        return e
    out["field_error"] = {"after_steps": steps, "mixed_vs_fp64": err(mix, ref), "noise_floor_fp64_seed": err(other, ref),
                          "U_scale": "sound speed of the left state"}
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["cpu_baseline"] = guarded(lambda: cpu_oracle_run(wl.shock_tube(precision="fp64", seed=seeds[0]), 0,
                                                         oracle_steps, "3D shock tube 9,600 tets, FP64, the "
                                                         f"whole {oracle_steps}-step run from the initial state"))
    return out


def gks_start_up(device, steps=20, warmup=3):
    """Start-up steps of the gas-kinetic scheme (the method without particles,
    Sec. 3.2; the initial fields of the steady cases, Sec. 4.3, 4.4) on the
    cavity 24^3 at second order with the Prandtl fix at Pr = 2/3: cell-steps/s
    with the global time step and with local time steps, CUDA events on the
    simulation's stream around `steps` direct-launch steps."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl
    cfg = wl.cavity(n=24, Kn=0.075, N_ref=100, precision="mixed", order=2)
    cfg["params"]["Pr"] = 2.0 / 3.0
    stream = torch.cuda.Stream(device=device)
    sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=stream)
    n = sim.n_cells
    out = {"workload": "cavity 24^3 hexes x 6 = 82,944 tets, Kn 0.075, order 2, Pr 2/3, no particles", "n_cells": n}
    for local in (False, True):
        sim.gks_steps(warmup, local_dt=local)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.gks_steps(steps, local_dt=local)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        out["local_dt" if local else "global_dt"] = {"ms_per_step": ms / steps,
                                                      "cell_steps_per_s": n * steps / (ms * 1e-3)}
    sim.sync()
    sim.close()
    return out


def hypersonic(device, which, steps, warmup, gks_steps, spin_up=5, adjoint_K=0):
    """The hypersonic configurations at full size, MIXED, first order, with the
    paper's particle setting N_min = N_ref (Sec. 4.3, 4.4) and energy-matched
    sampling: Ma 4 past the unit cube (1,152,912 tets, Kn 0.1, N_ref 200) or
    Ma 8 past the blunt vehicle (2,770,032 tets, Kn 1e-3, T_w = 3 T_inf,
    N_ref 100).  Each starts with `gks_steps` gas-kinetic steps with local
    time steps from the free stream (the start-up of the steady cases), then
    takes `spin_up` + `warmup` steps of the method and times up to `steps`
    more, in chunks of 10, until the first device error.  With adjoint_K > 0
    each functional (drag and wall heat flux of the body, theta = the free
    stream and the wall) gets an adjoint call of adjoint_K steps on a
    simulation of its own, right after its own start-up.

    With N_ref particles per cell the method runs on the order of 100 steps on
    the cube and 50 on the vehicle after the start-up before some cell's
    pressure falls through zero (the base region behind the cube, the bow shock
    ahead of the nose); the line reports how many steps it timed and the error
    that ended them.  A vehicle adjoint call takes 46 steps: the far field, 44
    tets from the body, reaches the functional after 46."""
    import torch
    from paper_2007_13091_gb300 import ugkwp
    from paper_2007_13091_gb300 import workloads as wl

    def config():
        cfg = wl.cube_flow() if which == "cube" else wl.blunt_vehicle()
        cfg["params"]["sampling"] = "energy_matched"
        cfg["params"]["N_min"] = cfg["params"]["N_ref"]
        return cfg

    def started(cfg, stream):
        sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.gks_steps(gks_steps, local_dt=True)
        b.record(stream)
        b.synchronize()
        return sim, a.elapsed_time(b)

    t0 = time.perf_counter()
    cfg = config()
    stream = torch.cuda.Stream(device=device)
    out = {"workload": cfg["name"], "n_cells": len(cfg["mesh"]["tets"]), "N_ref": cfg["params"]["N_ref"],
           "N_min": cfg["params"]["N_min"], "Kn": cfg["params"]["Kn"], "sampling": cfg["params"]["sampling"],
           "setup_s": time.perf_counter() - t0}
    sim, ms = started(cfg, stream)
    n = sim.n_cells
    sim.sync()
    W = sim.moments(ugkwp.W)
    U = W[1:4] / W[0]
    p = (W[4] - 0.5 * W[0] * (U * U).sum(0)) / 1.5
    out["gks_start_up"] = {"steps": gks_steps, "ms_per_step": ms / gks_steps,
                           "cell_steps_per_s": n * gks_steps / (ms * 1e-3),
                           "rho_min": float(W[0].min()), "p_min": float(p.min())}
    # timed in chunks of 10 steps (graph-replayed pairs, CUDA events on the
    # stream) until `steps` steps or the first device error, which ends the
    # run and is reported with the step it came in
    sim.step(spin_up + warmup)
    m0 = sim.step(0, stats=True)["n_moves_total"]
    ms, done, err = 0.0, 0, None
    while done < steps:
        k = min(10, steps - done)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(k)
        b.record(stream)
        try:
            st = sim.step(0, stats=True)
        except ugkwp.UgkwpError as e:
            err = {"error": str(e)[:200], "in_method_steps": [spin_up + warmup + done + 1, spin_up + warmup + done + k]}
            break
        ms += a.elapsed_time(b)
        done += k
        moves = st["n_moves_total"] - m0
    out.update({"steps_timed": done, "spin_up_steps": spin_up, "warmup_steps": warmup,
                "method_steps_after_start_up": spin_up + warmup + done, "ended_by": err})
    if done:
        out.update({"value": moves / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / done,
                    "cell_steps_per_s": n * done / (ms * 1e-3), "particles_per_step": moves / done})
    sim.close()
    if adjoint_K:
        adj = {}
        for functional, name in ((0, "drag"), (1, "wall_heat_flux")):
            sim, _ = started(config(), stream)
            t1 = time.perf_counter()
            try:
                r = sim.adjoint(functional, adjoint_K, [2])
                adj[name] = {"J_and_grad": [float(v) for v in r], "ms_per_call": 1e3 * (time.perf_counter() - t1)}
            except ugkwp.UgkwpError as e:
                adj[name] = {"error": str(e)[:200]}
            sim.close()
        out["adjoint"] = {"steps": adjoint_K, "theta": "(rho_inf, U_inf, T_w) = (1, 8 sqrt(5/3), 3)",
                          "grad_order": "dJ/drho_inf, dJ/dU_inf, dJ/dT_w", **adj}
        if "ms_per_call" in adj["drag"]:
            out["adjoint"]["cell_steps_per_s"] = n * adjoint_K / (1e-3 * adj["drag"]["ms_per_call"])
    return out


def host_cores():
    """Host cores this process may run on (the oracle itself uses one)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count()


def cpu_oracle_run(cfg, untimed, steps, sample):
    """The CPU oracle (single thread) on `cfg`: `untimed` steps, then `steps`
    timed steps; particle-moves/s and cell-steps/s."""
    import oracle
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    if untimed:
        s.step(untimed)
    moves = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        s.step()
        moves += s.last("counters")["n_tracked"]
    t1 = time.perf_counter()
    n = len(cfg["mesh"]["tets"])
    return {"value": moves / (t1 - t0), "unit": UNIT, "cores": 1, "host_cores_available": host_cores(),
            "kind": "oracle", "sample": f"{sample} ({steps} timed steps, {moves} particle moves, {t1 - t0:.1f} s)",
            "cell_steps_per_s": n * steps / (t1 - t0), "n_cells": n}


def cpu_baseline(steps):
    """The CPU oracle (single thread) on the bench workload: one untimed step
    samples the particle population, then `steps` timed steps.  The oracle
    starts from the initial state, where the cavity holds ~N_ref particles per
    cell, not from the settled ~2.6 N_ref the GPU line is timed on: its rate
    is per move, which the population size hardly changes."""
    cfg = workload("mixed")
    return cpu_oracle_run(cfg, 1, steps, f"cavity 24^3x6 tets, N_ref 100, MIXED, order {ORDER}: oracle steps after "
                                         "one sampling step, from the unsettled initial population")


def cpu_not_timed(line, start_up):
    """Why a hypersonic case has no CPU line: one oracle step moves as many
    particles as the GPU line's step (minutes on one core at the cavity's
    oracle rate) after hundreds of gas-kinetic start-up steps, which does not
    fit the bench's few minutes; the oracle's rate per move is the cavity's."""
    ppm = line.get("particles_per_step") if isinstance(line, dict) else None
    return {"timed": False, "reason": f"one oracle step moves ~{ppm:.3g} particles after {start_up} gas-kinetic "
                                      "start-up steps: minutes per step on one core, beyond the bench's few minutes"
            if ppm else "the GPU line did not run", "cores": 1, "host_cores_available": host_cores()}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    steps = max(1, min(args.steps, 4))
    warm = max(1, min(args.warmup, 1))
    import oracle
    cfg = workload("mixed")
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    s.step(warm)
    moves = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        s.step()
        moves += s.last("counters")["n_tracked"]
    dt = time.perf_counter() - t0
    v = moves / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": warm, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 cells / f32 particles (oracle)", "data": "synthetic",
            "config": {"workload": "lid-driven cavity 24^3 hexes x 6 = 82944 tets, Kn 0.075, N_ref 100, MIXED",
                       "order": ORDER,
                       "sample": f"{steps} of the requested {args.steps} steps (CPU oracle, single thread)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "host_cores_available": host_cores(),
                             "kind": "oracle",
                             "sample": f"{steps} oracle steps after {warm} warm-up step(s), {moves} moves"},
            "population": "the oracle starts from the initial state (~N_ref particles per cell) and runs only "
                          f"{warm + steps} steps, while the GPU line is timed on the settled population "
                          f"(~2.6 N_ref per cell after {SPIN_UP} steps): the rate is per particle move, which "
                          "the population size hardly changes, but the two lines do not time the same steps",
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ugkwp", choices=["ugkwp", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-extras", action="store_true", help="skip FP64, field error, e2e and CPU baseline")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--order", type=int, default=2, choices=[1, 2], help="reconstruction order of the workload")
    args = ap.parse_args()
    global ORDER
    ORDER = args.order
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    device = f"cuda:{local}"
    from paper_2007_13091_gb300 import ugkwp
    ugkwp.lib()
    stream = torch.cuda.Stream(device=device)
    cfg = workload(args.precision)
    nc = len(cfg["mesh"]["tets"])
    sim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], device=device, stream=stream)
    # spin-up to the settled particle population, then the library's autotuner
    # picks the grid sizes on that state (its trial steps are untimed)
    sim.step(SPIN_UP)
    launch_cfg = ugkwp.ugkwp_autotune(sim.handle, 4)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    with ClockSampler(uuid) as clk:
        ms, moves, launches, kms, st = time_steps(sim, args.steps, args.warmup, ws)
    clocks = clk.summary()
    ms_max, value, cell_steps = job_rates(ms, moves, nc, args.steps, ws)
    peak, peak_kind = peaks()
    track_ms = kms["track"] / args.steps
    moves_per_step = moves / args.steps
    kmoves = kms.pop("_moves") / args.steps
    alg = TRACK_BYTES_PER_MOVE[args.precision] * kmoves + TRACK_BYTES_PER_CELL[args.precision] * nc
    achieved = alg / (track_ms * 1e-3) / 1e9
    roof_track = {"kernel": "k_track (a6-a9, a11: t_f draw, tet walk, fixed-point flux, removal, compaction)", "bound": "hbm",
                  "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                  "peak_kind": f"{peak_kind} HBM copy", "traffic": TRACK_DRAM_BYTES[args.precision],
                  "traffic_unit": "bytes per step, both k_track launches (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                  "algorithmic_bytes_per_launch": alg,
                  "bytes_per_move": TRACK_BYTES_PER_MOVE[args.precision],
                  "bytes_per_cell": TRACK_BYTES_PER_CELL[args.precision], "ms_per_launch": track_ms,
                  "timing": "CUDA events on the library's stream around the tracking phase of each step (its "
                            "two k_track launches: the second starts when the wave flux is done) over "
                            f"{args.steps} further steps of the same run (direct launches, wave flux "
                            "overlapping on the second stream)"}
    # the movers' flux pass (a8): bound by its arithmetic (binary64 pipe for
    # phi, integer pipes for the fixed-point conversion); its binary64 work is
    # one phi per mover and a second one per wall hit
    movers_ms = kms.get("movers", 0.0) / args.steps
    n_movers = int(st["n_movers"])
    n_wall = int(st["n_wall_hits"])
    fp64_meas = None
    roof_movers = None
    if movers_ms > 0.0:
        fp64_meas = guarded(fp64_peak_measured)
        ops = MOVER_FP64_OPS[args.precision] * (n_movers + n_wall)
        ach_ops = ops / (movers_ms * 1e-3) / 1e9
        peak_ops = fp64_meas * 1e3 / 2.0 if isinstance(fp64_meas, float) else None
        mb = MOVER_BYTES[args.precision] * n_movers
        roof_movers = {"kernel": "k_movers (a8: binary64 counting flux of the particles that changed cell, met a "
                                 "wall or left)", "bound": "alu", "achieved": ach_ops, "peak": peak_ops,
                       "unit": "Gop/s (binary64 pipe operations)", "frac": ach_ops / peak_ops if peak_ops else None,
                       "peak_kind": "measured: cuBLAS DGEMM rate on this GPU / 2 (one FMA = 2 flops per pipe slot)",
                       "traffic": None, "fp64_ops_per_phi": MOVER_FP64_OPS[args.precision],
                       "movers_per_launch": n_movers, "wall_hits_per_launch": n_wall, "ms_per_launch": movers_ms,
                       "bytes_read_per_launch": mb, "hbm_gbs": mb / (movers_ms * 1e-3) / 1e9,
                       "int64_atomics_per_s": MOVER_ATOMICS * n_movers / (movers_ms * 1e-3),
                       "timing": "CUDA events on the library's stream around each launch"}
    roof_flux = None
    if ORDER == 2 and kms.get("flux_o2", 0.0) > 0.0:
        props = torch.cuda.get_device_properties(local)
        sm_mhz = 2070.0
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                sm_mhz = float(json.load(f).get("sm_max_mhz", sm_mhz))
        except OSError:
            pass
        fp64_nominal = props.multi_processor_count * FP64_FMA_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        if fp64_meas is None:
            fp64_meas = guarded(fp64_peak_measured)
        fp64_peak = fp64_meas if isinstance(fp64_meas, float) else fp64_nominal
        flux_ms = kms["flux_o2"] / args.steps
        n_if = sim.n_faces - sim.n_bfaces
        flops = FLUX_O2_FLOPS_PER_FACE * n_if if FLUX_O2_FLOPS_PER_FACE else None
        ach = flops / (flux_ms * 1e-3) / 1e12 if flops else None
        roof_flux = {"kernel": "k_face_flux_o2 (a3-a4: second-order wave flux of the interior faces, then the "
                               "first-order flux of the boundary faces)",
                     "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": ach / fp64_peak if ach else None,
                     "peak_kind": ("measured: cuBLAS DGEMM 8192^3 on this GPU (binary64 runs on the FMA pipes; "
                                   "there is no FP64 entry in the measured peaks)"
                                   if isinstance(fp64_meas, float) else "FP64 nominal (the DGEMM probe failed)"),
                     "fp64_nominal_tflops": fp64_nominal,
                     "fp64_nominal_kind": f"{props.multi_processor_count} SMs x {FP64_FMA_LANES_PER_SM} "
                                          f"FMA lanes/clk x 2 flop x {sm_mhz:.0f} MHz",
                     "frac_of_nominal": ach / fp64_nominal if ach else None,
                     "traffic": FLUX_O2_DRAM_BYTES, "traffic_unit": "bytes per launch (ncu)",
                     "flops_per_face": FLUX_O2_FLOPS_PER_FACE, "faces_per_launch": n_if,
                     "ms_per_launch": flux_ms,
                     "timing": "CUDA events on the library's wave stream around each launch, overlapping the "
                               "particle kernels"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_max / args.steps, "field_error": None, "mixed_over_fp64": None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 particles / f64 cells / int64 flux" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": "lid-driven cavity 24^3 hexes x 6 = 82944 tets, argon-like VHS gas, Kn 0.075, "
                                  "diffuse walls, lid Mach 0.16, N_ref 100",
                      "precision": args.precision, "order": ORDER, "n_cells": nc,
                      "spin_up_steps": SPIN_UP, "particles_per_step": int(moves_per_step),
                      "l2": "inputs larger than L2 (particle SoA %.2f GB per buffer)" % (moves_per_step * 44 / 1e9),
                      "parallelism": "replicas" if ws > 1 else "single GPU"},
           "cell_steps_per_s": cell_steps,
           "roofline": roof_track,
           "roofline_track": roof_track, "roofline_movers": roof_movers, "roofline_flux_o2": roof_flux,
           "kernels_ms_per_step": {k: v / args.steps for k, v in kms.items()},
           "step_launch": "two-step CUDA graphs replayed on the caller's stream",
           "launch_cfg": launch_cfg,
           "gpu_launches": int(launches), "clocks": clocks}
    sim.close()
    if not args.no_extras and rank == 0:
        c64 = workload("fp64")
        s64 = ugkwp.Simulation(c64["mesh"], c64["W0"], c64["params"], device=device, stream=stream)
        s64.step(SPIN_UP)
        cfg64 = ugkwp.ugkwp_autotune(s64.handle, 4)
        ms64, mv64, _, k64, _ = time_steps(s64, args.steps, args.warmup, 1)
        s64.close()
        k64.pop("_moves", None)
        out["fp64"] = {"value": mv64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / args.steps,
                       "cell_steps_per_s": nc * args.steps / (ms64 * 1e-3),
                       "kernels_ms_per_step": {k: v / args.steps for k, v in k64.items()}, "launch_cfg": cfg64}
        out["mixed_over_fp64"] = out["value"] / out["fp64"]["value"]
        out["field_error"] = guarded(lambda: field_error((1, 10, 20), device))
        out["field_error_time_averaged"] = guarded(lambda: field_error_averaged(device))
        out["e2e"] = e2e(cfg, 5, device, launch_cfg)

        def both():
            r = {"mixed": batched("mixed", args.steps, args.warmup, device),
                 "fp64": batched("fp64", args.steps, args.warmup, device)}
            r["mixed_over_fp64"] = r["mixed"]["value"] / r["fp64"]["value"]
            r["mixed_pair_sampling"] = guarded(lambda: batched_pairs(20, 3, device, r["mixed"]["launch_cfg"]))
            r["field_error"] = guarded(lambda: batched_field_error(device))
            r["equal_work_cavities"] = guarded(lambda: batched_cavities(args.steps, args.warmup, device))
            return r
        out["batched"] = guarded(both)
        out["adjoint"] = guarded(lambda: adjoint(device))
        out["gks_start_up"] = guarded(lambda: gks_start_up(device))
        out["gp1_sampling"] = guarded(lambda: gp1_sampling(device, args.steps, args.warmup, launch_cfg))
        out["diatomic"] = guarded(lambda: diatomic(device, args.steps, args.warmup, launch_cfg))
        out["shock_tube"] = guarded(lambda: shock_tube(device))
        out["cube_ma4"] = guarded(lambda: hypersonic(device, "cube", 100, 3, 300, spin_up=17))
        out["blunt_vehicle"] = guarded(lambda: hypersonic(device, "vehicle", 40, 3, 1200, spin_up=2, adjoint_K=46))
        out["cpu_baseline"] = cpu_baseline(args.cpu_steps)
        out["cpu_baseline_by_config"] = {
            "cavity": out["cpu_baseline"],
            "shock_tube": out["shock_tube"].get("cpu_baseline") if isinstance(out["shock_tube"], dict) else None,
            "cube_ma4": cpu_not_timed(out["cube_ma4"], 300), "blunt_vehicle": cpu_not_timed(out["blunt_vehicle"], 1200)}
    elif rank == 0:
        out["e2e"] = None
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
