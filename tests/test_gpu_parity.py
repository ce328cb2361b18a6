"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Protocol (teacher forcing): both sides start one step from the same state
(the oracle's own state after a few oracle steps, imported into the GPU), then
  * particles (id, cell, x, u, m) are equal bit for bit,
  * fixed-point sums (particle flux F^{fr,p}, survivor mass and count) are equal,
  * dt, tau, rho^h, N_sam, m_sam are equal bit for bit,
  * the wave flux and W^{n+1} agree within 1e-12 relative L2 (FP64 arithmetic
    with different exp/erfc implementations and fused multiply-adds).
"""
import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import ugkwp, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


def field_errors(Wg, Wo):
    """Relative L2 error per conservative component: mass and energy against
    their own norm, each momentum component against the momentum scale
    rho sqrt(p/rho) (a component that is zero up to rounding, such as the
    transverse momentum of a 1D problem, has no scale of its own)."""
    Wo = np.asarray(Wo, float)
    Wg = np.asarray(Wg, float)
    rho = Wo[0]
    p = (Wo[4] - 0.5 * (Wo[1:4] ** 2).sum(0) / rho) / 1.5
    mom = np.linalg.norm(rho * np.sqrt(np.abs(p / rho)))
    scale = [np.linalg.norm(Wo[0]), mom, mom, mom, np.linalg.norm(Wo[4])]
    return [float(np.linalg.norm(Wg[q] - Wo[q]) / scale[q]) for q in range(5)]


def assert_fields_close(Wg, Wo, tol):
    err = field_errors(Wg, Wo)
    assert max(err) <= tol, err


def _sorted(st):
    o = np.argsort(st["id"], kind="stable")
    e = st.get("e")
    return {"id": st["id"][o], "cell": st["cell"][o], "x": st["x"][:, o], "u": st["u"][:, o], "m": st["m"][o],
            "e": None if e is None else np.asarray(e)[o]}


def assert_particles_equal(g, o):
    a, b = _sorted(g), _sorted(o)
    assert a["id"].size == b["id"].size, (a["id"].size, b["id"].size)
    assert np.array_equal(a["id"], b["id"])
    assert np.array_equal(a["cell"], b["cell"])
    assert np.array_equal(a["m"], b["m"])
    assert np.array_equal(a["x"], b["x"])
    assert np.array_equal(a["u"], b["u"])
    if a["e"] is not None and b["e"] is not None:
        assert np.array_equal(a["e"], b["e"])


def compare_step(gsim, osim, check_flux=True):
    g, o = gsim.state(), osim.state()
    assert g["step"] == o["step"]
    assert gsim.last("dt") == osim.last("dt")
    for k in ("tau", "rho_h", "n_sam", "m_sam"):
        assert np.array_equal(gsim.last(k), osim.last(k)), k
    for k in ("pflux", "surv_mass", "surv_count"):
        assert np.array_equal(gsim.last(k), osim.last(k)), k
    assert_particles_equal(g, o)
    if check_flux:
        Fg, Fo = gsim.last("flux"), osim.last("flux")
        for q in range(5):
            scale = max(np.linalg.norm(Fo[q]), np.linalg.norm(Fo[1:4]) * 1e-3)
            assert np.linalg.norm(Fg[q] - Fo[q]) <= TOL * scale + 1e-300, q
    assert_fields_close(g["W"], o["W"], TOL)
    assert g["t"] == pytest.approx(o["t"], rel=1e-15)


def run_teacher_forced(cfg, warm_steps, launch=None):
    """One step of each side from the oracle's state after warm_steps steps;
    launch: (particle_blocks, wave_blocks, track_threads, smem_carveout) for
    the GPU side, or None for the default configuration."""
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step(warm_steps)
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    if launch is not None:
        ugkwp.ugkwp_set_launch_cfg(gsim.handle, *launch)
    gsim.set_state(osim.state())
    g0 = gsim.state()
    assert_particles_equal(g0, osim.state())  # import/export round trip
    osim.step()
    gsim.step()
    gsim.sync()
    compare_step(gsim, osim)
    return gsim, osim


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shock_tube_first_step_from_init(precision):
    cfg = wl.shock_tube(precision=precision)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step()
    st = gsim.step(1, stats=True)
    compare_step(gsim, osim)
    c = osim.last("counters")
    assert st["n_sampled"] == c["n_sampled"] and st["n_exited"] == c["n_exited"]
    assert st["n_crossings"] == c["n_crossings"] and st["n_particles"] == osim.sizes()["n_particles"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shock_tube_teacher_forced(precision):
    gsim, osim = run_teacher_forced(wl.shock_tube(precision=precision), warm_steps=3)
    assert osim.last("counters")["n_collided"] > 0


@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tracking_tiles_teacher_forced(precision, threads):
    """The tracking kernel with 128- or 256-particle tiles against the oracle,
    on a jittered far-field mesh whose particle count leaves a ragged last
    tile, with an odd grid so that blocks take unequal numbers of tiles and
    walks that leave their first tet wait in the blocks' queues."""
    cfg = wl.cube_flow(h0=0.5, growth=2.0, N_ref=30, precision=precision, Kn=0.1)
    gsim, osim = run_teacher_forced(cfg, warm_steps=2, launch=(37, 5, threads, -1))
    n = osim.state()["id"].size
    assert n % threads != 0 and n > 50 * threads
    assert osim.last("counters")["n_crossings"] > 0


def test_tracking_tiles_internal_energy_teacher_forced():
    """Queued walks carry the particles' internal energies (K = 2)."""
    cfg = wl.cavity(n=6, N_ref=40, precision="mixed", order=1, K=2)
    run_teacher_forced(cfg, warm_steps=3, launch=(19, 3, 128, 58))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cavity_diffuse_walls_teacher_forced(precision):
    cfg = wl.cavity(n=6, N_ref=40, precision=precision)
    gsim, osim = run_teacher_forced(cfg, warm_steps=3)
    assert osim.last("counters")["n_wall_hits"] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cube_farfield_jittered_teacher_forced(precision):
    cfg = wl.cube_flow(h0=0.5, growth=2.0, N_ref=30, precision=precision, Kn=0.1)
    assert len(cfg["mesh"]["tets"]) > 1024 + 1  # several scan blocks and a ragged tail
    gsim, osim = run_teacher_forced(cfg, warm_steps=2)
    c = osim.last("counters")
    assert c["n_exited"] > 0 and c["n_wall_hits"] > 0


def _order2(cfg, K):
    cfg["params"]["order"] = 2
    cfg["params"]["venkat_K"] = K
    return cfg


def _assert_gradients_close(gsim, gW, gH):
    """Limited gradients of the last step against the oracle's: each component
    within 1e-11 of the larger of its own norm and 1e-3 of the momentum one."""
    Gg, Hg = gsim.last("grad_W"), gsim.last("grad_rho_h")
    mom = np.linalg.norm(gW[1:4])
    for q in range(5):
        scale = max(np.linalg.norm(gW[q]), 1e-3 * mom)
        assert np.linalg.norm(Gg[q] - gW[q]) <= 1e-11 * scale, q
    assert np.linalg.norm(Hg - gH) <= 1e-11 * np.linalg.norm(gH)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_order2_shock_tube_teacher_forced(precision):
    """Second-order wave flux (Sec. 2.1): least-squares gradients with
    Venkatakrishnan's limiter at interior faces, specular and far-field ghosts."""
    cfg = _order2(wl.shock_tube(precision=precision), K=1.0)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step(3)
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim.set_state(osim.state())
    osim.prepare()
    gW, gH = osim.gradients(limited=True)
    osim.step()
    gsim.step()
    compare_step(gsim, osim)
    _assert_gradients_close(gsim, gW, gH)


@pytest.mark.parametrize("K", [0.3, 5.0])
def test_order2_cube_jittered_teacher_forced(K):
    """Jittered graded tets (several blocks and a ragged tail), far field and a
    diffuse wall; K = 0.3 keeps the limiter active, K = 5 mostly relaxes it."""
    cfg = _order2(wl.cube_flow(h0=0.5, growth=2.0, N_ref=30, precision="mixed", Kn=0.1), K=K)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step(2)
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim.set_state(osim.state())
    osim.prepare()
    gW, gH = osim.gradients(limited=True)
    ref, _ = osim.gradients(limited=False)
    osim.step()
    gsim.step()
    compare_step(gsim, osim)
    _assert_gradients_close(gsim, gW, gH)
    if K < 1.0:  # the limiter acts on a share of the cells
        assert np.mean(np.abs(gW - ref).max(axis=(0, 1)) > 1e-6 * np.abs(ref).max()) > 0.05


def test_order2_cavity_teacher_forced():
    cfg = _order2(wl.cavity(n=6, N_ref=40, precision="mixed"), K=5.0)
    gsim, osim = run_teacher_forced(cfg, warm_steps=3)
    assert osim.last("counters")["n_wall_hits"] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_matched_sampling_teacher_forced(precision):
    """Energy-matched sampling: the per-cell spread (a sequential binary64 sum over
    the cell's pairs) and every sampled particle bit for bit."""
    cfg = wl.shock_tube(precision=precision)
    cfg["params"]["sampling"] = "energy_matched"
    gsim, osim = run_teacher_forced(cfg, warm_steps=3)
    assert osim.last("counters")["n_sampled"] > 0


def test_energy_matched_sampling_cavity_order2():
    cfg = wl.cavity(n=6, N_ref=40, precision="mixed", order=2)
    cfg["params"]["sampling"] = "energy_matched"
    run_teacher_forced(cfg, warm_steps=3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gp1_sampling_teacher_forced(precision):
    """First-order g_p sampling: per-cell coefficients from the limited slopes,
    every particle drawn on its own by acceptance-rejection; the sampled
    particles bit for bit (the acceptance test runs in the particle precision
    on both sides)."""
    cfg = wl.cavity(n=6, N_ref=40, precision=precision, order=2)
    cfg["params"]["sampling"] = "gp1"
    gsim, osim = run_teacher_forced(cfg, warm_steps=3)
    assert osim.last("counters")["n_sampled"] > 0


def test_gp1_sampling_limited_wave():
    """A steep smooth temperature wave at Kn 5, where the bound of the g_p
    correction reaches 1 in some cells (the limiter scales it)."""
    import math
    cfg = wl.uniform_box(n=(12, 2, 2), Kn=5.0, bc_type="specular", N_ref=60, precision="mixed")
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    x = nodes[tets].mean(1)[:, 0]
    T = 1.0 + 0.8 * np.sin(4.0 * math.pi * x)
    W0 = np.concatenate([(1.0 / T)[None], np.zeros((3, len(tets))), np.full((1, len(tets)), 1.5)])
    cfg["W0"] = W0
    cfg["params"].update(order=2, venkat_K=1e6, sampling="gp1")
    o = oracle.OracleSim(cfg["mesh"], W0, cfg["params"])
    o.prepare()
    assert max(o.gp_coefficients(k)[13] for k in range(len(tets))) == 2.0
    gsim = ugkwp.Simulation(cfg["mesh"], W0, cfg["params"])
    o.step()
    gsim.step()
    # particles and sums bit for bit; the wave flux of this steep unlimited
    # profile is checked through the fields only
    compare_step(gsim, o, check_flux=False)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("order", [1, 2])
def test_internal_degrees_of_freedom_teacher_forced(precision, order):
    """K = 2 (diatomic): wave moments with |xi|^2, particles carrying internal
    energies (sampled, kept, re-drawn at the diffuse walls), the energy flux
    in fixed point; particles and their internal energies bit for bit."""
    cfg = wl.cavity(n=6, N_ref=40, precision=precision, order=order, K=2)
    gsim, osim = run_teacher_forced(cfg, warm_steps=3)
    c = osim.last("counters")
    assert c["n_wall_hits"] > 0 and c["n_sampled"] > 0
    assert np.all(osim.state()["e"] > 0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_internal_degrees_first_step_from_init(precision):
    """K = 2 from the common initial state, with no state import: each side
    derives its fixed-point quanta from W0 with p = (rho E - rho |U|^2/2) /
    ((3 + K)/2) (on this tube a K = 0 pressure would give the momentum
    quantum one binade too coarse), so the quanta, the first step's particles
    and its fixed-point sums are equal bit for bit."""
    cfg = wl.shock_tube(precision=precision, K=2)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    assert np.array_equal(gsim.state()["exps"], osim.state()["exps"])
    osim.step()
    gsim.step(1, stats=True)
    compare_step(gsim, osim)
    assert np.array_equal(gsim.state()["exps"], osim.state()["exps"])
    assert np.all(osim.state()["e"] > 0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_internal_degrees_of_freedom_shock_tube(precision):
    cfg = _order2(wl.shock_tube(precision=precision, K=5), K=1.0)
    run_teacher_forced(cfg, warm_steps=3)


def test_specular_box_degenerate_starts():
    """Particles placed exactly on nodes, edges and faces (teacher-forced import)."""
    cfg = wl.uniform_box(n=(3, 3, 3), Kn=0.5, N_ref=10, bc_type="specular")
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step(1)
    st = osim.state()
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    k = min(400, st["id"].size)
    P = nodes[tets[st["cell"][:k]]]
    choice = (np.arange(k) % 4)[:, None]
    st["x"][:, :k] = np.where(choice == 0, P[:, 0], np.where(choice == 1, 0.5 * (P[:, 0] + P[:, 3]),
                              np.where(choice == 2, (P[:, 1] + P[:, 2] + P[:, 3]) / 3, P.mean(1)))).T
    osim.set_state(st)
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim.set_state(st)
    osim.step()
    gsim.step()
    compare_step(gsim, osim)


def test_free_running_multi_step():
    """Five steps each side from the same initial state: fields stay within
    tolerance; particle ids and cells stay identical."""
    cfg = wl.shock_tube(precision="fp64")
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    for _ in range(5):
        osim.step()
        gsim.step()
        g, o = gsim.state(), osim.state()
        assert_fields_close(g["W"], o["W"], 1e-11)
        a, b = _sorted(g), _sorted(o)
        assert np.array_equal(a["id"], b["id"]) and np.array_equal(a["cell"], b["cell"])
        np.testing.assert_allclose(a["x"], b["x"], rtol=1e-12, atol=1e-14)


def test_no_particles_regime():
    """Near-continuum: e^{-dt/tau} below the sampling floor, no particle at all."""
    cfg = wl.shock_tube(nx=40, ny=2, nz=2, Kn=1e-9, precision="mixed")
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    for _ in range(3):
        osim.step()
        gsim.step()
        assert gsim.state()["id"].size == 0
        assert_fields_close(gsim.state()["W"], osim.state()["W"], TOL)
    gsim.set_state(osim.state())
    osim.step()
    gsim.step()
    compare_step(gsim, osim)


def test_moments_wp_wh_prim():
    cfg = wl.cavity(n=5, N_ref=30, precision="mixed")
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step(2)
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    st = osim.state()
    gsim.set_state(st)
    vol = osim.geometry("vol")
    nc = vol.size
    phi = np.stack([st["m"], st["m"] * st["u"][0], st["m"] * st["u"][1], st["m"] * st["u"][2],
                    0.5 * st["m"] * (st["u"] ** 2).sum(0)])
    WP = np.stack([np.bincount(st["cell"], phi[q], nc) for q in range(5)]) / vol
    np.testing.assert_allclose(gsim.moments(ugkwp.WP), WP, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(gsim.moments(ugkwp.WH), st["W"] - WP, rtol=1e-11, atol=1e-12)
    np.testing.assert_array_equal(gsim.moments(ugkwp.W), st["W"])
    prim = gsim.moments(ugkwp.PRIM)
    np.testing.assert_allclose(prim[0], st["W"][0], rtol=0)
    p = (st["W"][4] - 0.5 * (st["W"][1:4] ** 2).sum(0) / st["W"][0]) / 1.5
    np.testing.assert_allclose(prim[4], p / st["W"][0], rtol=1e-13)


def test_capacity_overflow_is_reported():
    cfg = wl.shock_tube(nx=20, ny=2, nz=2)
    cfg["params"]["particle_capacity"] = 1000  # far below the 240 x 50 sampled particles
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim.step()
    with pytest.raises(ugkwp.UgkwpError) as e:
        gsim.sync()
    assert e.value.code == ugkwp.E_CAPACITY


def test_crossing_limit_is_reported():
    """A planted fast particle exceeds max_crossings: both sides report it, keep
    it in place, and otherwise agree."""
    cfg = wl.shock_tube(nx=40, ny=2, nz=2, Kn=10.0)
    cfg["params"]["max_crossings"] = 20
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step()
    st = osim.state()
    k = np.argmin(np.abs(st["x"][0] - 0.3))
    st["u"][:, k] = (500.0, 3.0, 2.0)  # ~0.2 length units in one step: dozens of faces
    osim.set_state(st)
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim.set_state(st)
    with pytest.raises(RuntimeError, match="max_crossings"):
        osim.step()
    with pytest.raises(ugkwp.UgkwpError) as e:
        gsim.step(1, stats=True)
    assert e.value.code == ugkwp.E_TRACK_LIMIT
    compare_step(gsim, osim)


def _one_changed(a, i, v):
    b = np.array(a, copy=True)
    b.reshape(-1)[i] = v
    return b


@pytest.mark.parametrize("precision,K", [("mixed", 0), ("mixed", 2), ("fp64", 2)])
def test_import_rejects_bad_state(precision, K):
    """Every particle is checked on the device before the state changes: a
    rejected image names the first bad particle's problem and leaves the
    simulation where it was; a good image after it is taken as usual."""
    cfg = wl.shock_tube(nx=10, ny=2, nz=2, precision=precision, K=K)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step()
    st = osim.state()
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    gsim.step(2)
    before = gsim.state()
    n = st["cell"].size
    cases = [(dict(st, cell=_one_changed(st["cell"], n // 2, 10 ** 6).astype(np.int32)), "cell out of range"),
             (dict(st, cell=_one_changed(st["cell"], 3, -1).astype(np.int32)), "cell out of range")]
    if precision == "mixed":
        cases += [(dict(st, x=st["x"] + 1e-12), "not representable"),
                  (dict(st, u=_one_changed(st["u"], 2 * n + 5, 0.1)), "not representable")]
    if K:
        cases += [(dict(st, e=_one_changed(st["e"], 7, -1.0)), "negative internal energy"),
                  (dict(st, e=_one_changed(st["e"], 7, np.nan)), "negative internal energy")]
        if precision == "mixed":
            cases += [(dict(st, e=_one_changed(st["e"], 9, 0.1)), "internal energy not representable")]
    # the first bad particle decides the message: a bad cell after a bad position
    if precision == "mixed":
        cases += [(dict(st, x=_one_changed(st["x"], 1, 1e-9), cell=_one_changed(st["cell"], 4, -1).astype(np.int32)),
                   "not representable")]
    for bad, msg in cases:
        with pytest.raises(ugkwp.UgkwpError, match=msg) as e:
            gsim.set_state(bad)
        assert e.value.code == ugkwp.E_STATE
        after = gsim.state()
        assert after["step"] == before["step"]
        np.testing.assert_array_equal(after["W"], before["W"])
        assert_particles_equal(after, before)
    gsim.set_state(st)
    gsim.step(1)
    osim.step()
    compare_step(gsim, osim)


@pytest.mark.parametrize("precision,K", [("mixed", 0), ("mixed", 2), ("fp64", 0)])
def test_native_image_round_trip(precision, K):
    """The native image (particles in the simulation's own precision) restores
    a simulation bit for bit: a copy restored from it steps on exactly like
    the original; its velocities, cells, masses and ids are those of the
    binary64 image; a bad image is rejected and changes nothing."""
    cfg = wl.cavity(n=5, N_ref=40, precision=precision, order=2, K=K, seed=31)
    a = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    a.step(3)
    nat = a.state_native()
    wide = a.state()
    assert nat["real_size"] == (4 if precision == "mixed" else 8)
    assert nat["x"].dtype == (np.float32 if precision == "mixed" else np.float64)
    for k in ("id", "cell", "m", "W"):
        np.testing.assert_array_equal(nat[k], wide[k])
    np.testing.assert_array_equal(nat["u"].astype(np.float64), wide["u"])
    if K:
        np.testing.assert_array_equal(nat["e"].astype(np.float64), wide["e"])
    if precision == "fp64":
        np.testing.assert_array_equal(nat["x"], wide["x"])
    b = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    b.step(1)
    before = b.state()
    bad = dict(nat, cell=_one_changed(nat["cell"], 2, cfg["mesh"]["tets"].shape[0]).astype(np.int32))
    with pytest.raises(ugkwp.UgkwpError, match="cell out of range"):
        b.set_state_native(bad)
    with pytest.raises(ugkwp.UgkwpError) as e:
        b.set_state_native(dict(nat, real_size=12 - nat["real_size"]))
    assert e.value.code == ugkwp.E_ARG
    after = b.state()
    np.testing.assert_array_equal(after["W"], before["W"])
    assert_particles_equal(after, before)
    b.set_state_native(nat)
    a.step(2)
    b.step(2)
    sa, sb = a.state(), b.state()
    assert sa["step"] == sb["step"]
    np.testing.assert_array_equal(sa["W"], sb["W"])
    assert_particles_equal(sa, sb)


def test_import_of_an_image_without_particles():
    """An image with no particles is taken in both forms: the next step starts
    from W alone and samples every cell, as the first step does."""
    cfg = wl.cavity(n=4, N_ref=30, precision="mixed", order=2, seed=41)
    a = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    a.step(2)
    wide, nat = a.state(), a.state_native()
    empty_wide = dict(wide, id=wide["id"][:0], cell=wide["cell"][:0], m=wide["m"][:0], e=wide["e"][:0],
                      x=wide["x"][:, :0], u=wide["u"][:, :0])
    empty_nat = dict(nat, id=nat["id"][:0], cell=nat["cell"][:0], m=nat["m"][:0], e=nat["e"][:0],
                     x=nat["x"][:, :0], u=nat["u"][:, :0])
    b = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    c = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"])
    b.set_state(empty_wide)
    c.set_state_native(empty_nat)
    for sim in (b, c):
        st = sim.state()
        assert st["id"].size == 0 and st["step"] == wide["step"]
        np.testing.assert_array_equal(st["W"], wide["W"])
        stats = sim.step(1, stats=True)
        assert stats["n_particles"] > 0 and stats["n_sampled"] == stats["n_tracked"]
    sb, sc = b.state(), c.state()
    np.testing.assert_array_equal(sb["W"], sc["W"])
    assert_particles_equal(sb, sc)


def test_graph_replay_matches_direct_launches():
    """ugkwp_step(n >= 2) replays two-step CUDA graphs; the state must equal that
    of single-step launches bit for bit (all sums are order-independent)."""
    import torch
    cfg = wl.cavity(n=6, N_ref=30, precision="mixed")
    s_graph = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    s_direct = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    s_graph.step(6)
    for _ in range(6):
        s_direct.step(1)
    a, b = s_graph.state(), s_direct.state()
    assert a["step"] == b["step"] == 6
    np.testing.assert_array_equal(a["W"], b["W"])
    assert_particles_equal(a, b)
    # odd counts and a teacher-forced import (which drops the graphs) still agree
    s_graph.step(3)
    s_direct.step(1)
    s_direct.step(1)
    s_direct.step(1)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step(2)
    for sim in (s_graph, s_direct):
        sim.set_state(osim.state())
    s_graph.step(2)
    s_direct.step(1)
    s_direct.step(1)
    a, b = s_graph.state(), s_direct.state()
    np.testing.assert_array_equal(a["W"], b["W"])
    assert_particles_equal(a, b)


@pytest.mark.parametrize("precision", ["mixed"])
def test_cavity_full_size_teacher_forced(precision):
    """The bench workload at full size (24^3 x 6 = 82,944 tets, ~8.4e6 particles,
    second-order reconstruction) on a side stream as the bench runs it: one step from the oracle's state
    after its sampling step (graph replay equals direct launches, tested above), taken three times
    from the same state (the buffers alternate, so each reads memory the previous one wrote)."""
    import torch
    cfg = wl.cavity(n=24, N_ref=100, precision=precision, order=2)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.step(1)
    st = osim.state()
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    osim.step(1)
    for _ in range(3):
        gsim.set_state(st)
        gsim.step(1)
        compare_step(gsim, osim)
    assert osim.sizes()["n_particles"] > 8_000_000


def _tet_neighbours(tets):
    """Face-adjacent tets of every tet (-1 where the face is on the boundary)."""
    tets = np.asarray(tets, dtype=np.int64)
    nc = len(tets)
    f = np.sort(tets[:, [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]].reshape(-1, 3), axis=1)
    n = int(tets.max()) + 1
    key = (f[:, 0] * n + f[:, 1]) * n + f[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    nb = np.full(4 * nc, -1, dtype=np.int64)
    same = ks[1:] == ks[:-1]
    a, b = order[:-1][same], order[1:][same]
    nb[a] = b // 4
    nb[b] = a // 4
    return nb.reshape(nc, 4)


def test_cube_full_size_sampled():
    """Full-size Ma 4 cube (1,152,912 tets, N_ref 200, ~2.3e8 particles), first
    step from the common initial state.  All per-cell quantities of the step
    (dt, tau, rho^h, N_sam, m_sam) are compared bit for bit; for 24 random cells
    the oracle regenerates and tracks every particle born within four
    neighbour rings and reproduces the GPU's W^p of the cell exactly (fixed
    point), which covers sampling, tracking, walls and exits at full size."""
    import torch
    cfg = wl.cube_flow(precision="mixed")
    nc = len(cfg["mesh"]["tets"])
    assert nc > 1_100_000
    cfg["params"]["particle_capacity"] = int(1.3 * 200 * nc)
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    st = gsim.step(1, stats=True)
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.prepare()
    assert gsim.last("dt") == osim.last("dt")
    for k in ("tau", "rho_h", "n_sam", "m_sam"):
        assert np.array_equal(gsim.last(k), osim.last(k)), k
    assert st["n_sampled"] == int(osim.last("n_sam").sum()) > 2e8
    assert st["n_lost"] == 0
    _check_sampled_cells(gsim, osim, cfg, rng_seed=13)
    gsim.close()


def test_blunt_vehicle_full_size_sampled():
    """Full-size Ma 8 blunt vehicle (2,770,032 tets, N_ref 100, T_w = 3 T_inf,
    snapped body surface), the method's first step from the GPU's own
    gas-kinetic start-up field (300 local steps), imported into the oracle:
    per-cell dt, tau, rho^h, N_sam, m_sam bit for bit, and the GPU's W^p of 24
    random cells (and of 8 cells next to the body) reproduced exactly by the
    oracle's own sampling and tracking of the particles around them."""
    import torch
    cfg = wl.blunt_vehicle(precision="mixed")
    nc = len(cfg["mesh"]["tets"])
    assert nc > 2_700_000
    gsim = ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream())
    gsim.gks_steps(300, local_dt=True)
    st0 = gsim.state()
    assert st0["id"].size == 0
    osim = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    osim.set_state(st0)
    st = gsim.step(1, stats=True)
    osim.prepare()
    assert gsim.last("dt") == osim.last("dt")
    for k in ("tau", "rho_h", "n_sam", "m_sam"):
        assert np.array_equal(gsim.last(k), osim.last(k)), k
    assert st["n_sampled"] == int(osim.last("n_sam").sum()) > 2e8
    assert st["n_lost"] == 0
    body = _body_cells(cfg)
    _check_sampled_cells(gsim, osim, cfg, rng_seed=17, extra=np.random.default_rng(3).choice(body, 8, replace=False))
    gsim.close()


def _body_cells(cfg):
    """Tets with a face on the body (boundary tag 2)."""
    tets = np.asarray(cfg["mesh"]["tets"], dtype=np.int64)
    bf = np.sort(np.asarray(cfg["mesh"]["bfaces"], dtype=np.int64)[cfg["mesh"]["btags"] == 2], axis=1)
    n = int(tets.max()) + 1
    f = np.sort(tets[:, [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]].reshape(-1, 3), axis=1)
    key = (f[:, 0] * n + f[:, 1]) * n + f[:, 2]
    bkey = (bf[:, 0] * n + bf[:, 1]) * n + bf[:, 2]
    return np.unique(np.nonzero(np.isin(key, bkey))[0] // 4)


def _check_sampled_cells(gsim, osim, cfg, rng_seed, n_cells=24, extra=()):
    """For random cells (and `extra`), the oracle regenerates and tracks every
    particle born within four neighbour rings in the first step and
    reproduces the GPU's W^p of the cell exactly (fixed point)."""
    nc = len(cfg["mesh"]["tets"])
    WP = gsim.moments(ugkwp.WP)
    dt, tau = osim.last("dt"), osim.last("tau")
    info = ugkwp.ugkwp_state_info(gsim.handle)
    exps = [int(v) for v in info.exps]
    vol = osim.geometry("vol")
    nb = _tet_neighbours(cfg["mesh"]["tets"])
    rng = np.random.default_rng(rng_seed)
    cells = list(rng.choice(nc, n_cells, replace=False)) + [int(v) for v in extra]
    step = int(info.step) - 1
    for c in cells:
        dist = {int(c): 0}
        frontier = {int(c)}
        for r in range(1, 5):
            frontier = {int(v) for t in frontier for v in nb[t] if v >= 0} - set(dist)
            dist.update({t: r for t in frontier})
        acc = np.zeros(5, dtype=np.int64)
        for b, r in sorted(dist.items()):
            sp = osim.sample_cell(b)
            for k in range(sp["id"].size):
                out = osim.track_one(sp["id"][k], b, sp["x"][:, k], sp["u"][:, k], tau[b], dt, step)
                if out["status"] & 3 or out["cell"] != c:
                    continue
                assert r < 4, "a particle from the outermost ring reached the cell: widen the ring"
                m = sp["m"][k]
                u = out["u"]
                phi = np.array([m, m * u[0], m * u[1], m * u[2], 0.5 * (m * ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]))])
                acc += np.rint(np.ldexp(phi, -np.array(exps))).astype(np.int64)
        ref = (acc.astype(np.float64) * np.ldexp(1.0, np.array(exps))) / vol[c]
        np.testing.assert_array_equal(WP[:, c], ref)


def test_identical_simulations_stay_identical():
    """Two simulations of the same case, stepped side by side, end bit for bit
    alike: a shock tube moving at Mach 2.9 (56,154 tets, Kn 1.2e-4, second
    order, MIXED, ~2.7e6 particles, 17% of them crossing faces each step),
    40 steps at the bench's launch shape.  Guards the per-block bookkeeping of
    the tracking kernel (tiles, walk queue, output rounds) against races that
    only show as rare duplicated or dropped particles."""
    import torch
    cfg = wl.batch_instances(n=61, precision="mixed", order=2, cap_factor=4.0)[60]
    sims = [ugkwp.Simulation(cfg["mesh"], cfg["W0"], cfg["params"], stream=torch.cuda.Stream()) for _ in range(2)]
    for s in sims:
        ugkwp.ugkwp_set_launch_cfg(s.handle, 1216, 152, 128, 58)
    for _ in range(4):
        for s in sims:
            s.step(10)
        for s in sims:
            s.sync()
    a, b = sims[0].state(), sims[1].state()
    np.testing.assert_array_equal(a["W"], b["W"])
    assert_particles_equal(a, b)
    for s in sims:
        s.close()
