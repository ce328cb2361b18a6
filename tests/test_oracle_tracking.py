"""Pins of the oracle's particle streaming (Sec. 2.2: x* = x + u t_f) with
face-by-face tet tracking, against brute force:

* the end position equals the straight-line (or, with specular walls, the
  mirror-unfolded) position, and the end tet contains it;
* along the way, the tets visited agree with point location by barycentric
  coordinates at fine sub-steps;
* outflow walls absorb exactly the particles whose straight path leaves the box;
* particles started on faces, edges and vertices are tracked without loss.
"""
import numpy as np
import pytest

import oracle
from paper_2007_13091_gb300 import workloads as wl


def _locate(nodes, tets, x, tol=1e-12):
    p = nodes[tets]
    T = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2)  # [nc,3,3]
    lam = np.linalg.solve(T, (x[None, :] - p[:, 0])[..., None])[..., 0]
    bary = np.concatenate([1 - lam.sum(1, keepdims=True), lam], axis=1)
    return np.nonzero(np.all(bary >= -tol, axis=1))[0]


def _fold(y, a):
    m = np.mod(y, 2 * a)
    return np.where(m > a, 2 * a - m, m)


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 2, 2)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tracking_matches_unfolded_motion(n, precision):
    cfg = wl.uniform_box(n=n, size=(1.0, 1.0, 1.0), bc_type="specular", precision=precision, Kn=1e6)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    rng = np.random.default_rng(17)
    real = np.float64 if precision == "fp64" else np.float32
    tol = 1e-12 if precision == "fp64" else 2e-5
    for trial in range(300):
        c = rng.integers(len(tets))
        w = rng.dirichlet(np.ones(4))
        x = (w @ nodes[tets[c]]).astype(real).astype(np.float64)
        if len(_locate(nodes, tets, x, tol=0)) == 0:
            continue
        u = rng.normal(size=3).astype(real).astype(np.float64)
        dt = float(real(rng.uniform(0.05, 3.0)))
        # born this step (id's step field == step): t_f = dt, no collision draw
        out = s.track_one(pid=(5 << 40) | 3, cell=c, x=x, u=u, tau_cell=1.0, dt=dt, step=5)
        assert out["status"] == 0
        xe = _fold(x + u * dt, 1.0)
        assert np.allclose(out["x"], xe, atol=50 * tol * (1 + np.abs(u).max() * dt))
        hits = _locate(nodes, tets, out["x"], tol=100 * tol)
        assert out["cell"] in hits
        # number of reflections -> sign of each velocity component
        flips = np.floor_divide(x + u * dt, 1.0).astype(int) % 2
        assert np.array_equal(np.sign(out["u"]), np.sign(u) * (1 - 2 * flips))


def test_visited_tets_follow_point_location():
    cfg = wl.uniform_box(n=(3, 3, 3), bc_type="outflow", Kn=1e6, jitter_amount=0.2, seed=9)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    rng = np.random.default_rng(3)
    checked = 0
    for trial in range(150):
        c = rng.integers(len(tets))
        x = rng.dirichlet(np.ones(4)) @ nodes[tets[c]]
        u = rng.normal(size=3)
        # march the straight line; each time the containing tet changes the tracker,
        # asked for the same time, must end in that tet (away from faces)
        for t in np.linspace(0.0, 1.0, 40)[1:]:
            xe = x + u * t
            if np.any(xe < 0) or np.any(xe > 1):
                out = s.track_one(pid=(5 << 40) | 1, cell=c, x=x, u=u, tau_cell=1.0, dt=t, step=5)
                assert out["status"] == 2  # exited through the outflow boundary
                break
            hits = _locate(nodes, tets, xe, tol=-1e-9)  # strictly inside one tet
            if len(hits) != 1:
                continue
            out = s.track_one(pid=(5 << 40) | 1, cell=c, x=x, u=u, tau_cell=1.0, dt=t, step=5)
            assert out["status"] == 0 and out["cell"] == hits[0]
            np.testing.assert_allclose(out["x"], xe, atol=1e-13)
            checked += 1
    assert checked > 1000


def test_degenerate_starts_on_faces_edges_vertices():
    cfg = wl.uniform_box(n=(2, 2, 2), bc_type="specular", Kn=1e6)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    rng = np.random.default_rng(8)
    dirs = [np.array(v, float) for v in ([1, 0, 0], [1, 1, 0], [1, 1, 1], [0, -1, 0], [-1, 1, -1])]
    for c in range(0, len(tets), 3):
        P = nodes[tets[c]]
        starts = [P[0], P[3], 0.5 * (P[0] + P[1]), (P[1] + P[2] + P[3]) / 3, P.mean(0)]
        for x in starts:
            for u in dirs + [rng.normal(size=3)]:
                out = s.track_one(pid=(5 << 40) | 2, cell=c, x=x, u=u, tau_cell=1.0, dt=0.7, step=5)
                assert out["status"] == 0
                xe = _fold(x + u * 0.7, 1.0)
                np.testing.assert_allclose(out["x"], xe, atol=1e-12)
                assert out["cell"] in _locate(nodes, tets, out["x"], tol=1e-9)


def test_free_transport_time_draw():
    """t_f = min(-tau ln eta, dt) (Eq. t_f): the fraction of old particles that
    collide is 1 - exp(-dt/tau) (binomial bound)."""
    cfg = wl.uniform_box(n=(1, 1, 1), bc_type="specular", Kn=1e6)
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    n, dt, tau = 20000, 0.01, 0.02
    coll = 0
    for k in range(n):
        out = s.track_one(pid=k, cell=0, x=cfg["mesh"]["nodes"][cfg["mesh"]["tets"][0]].mean(0),
                          u=np.array([0.1, 0.2, 0.3]), tau_cell=tau, dt=dt, step=3)
        coll += out["status"] & 1
    p = 1 - np.exp(-dt / tau)
    assert abs(coll - n * p) < 5 * np.sqrt(n * p * (1 - p))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_diffuse_wall_reemission_law(precision):
    """Diffuse re-emission with full accommodation (Sec. 2.4 (e)): a particle
    that hits the x = 0 wall leaves with a flux-weighted half-Maxwellian of the
    wall temperature, u_x^2 / (2 R T_w) ~ Exp(1), and Gaussian tangential
    components N(0, R T_w); one draw per particle id."""
    from scipy import stats
    T_w = 2.0
    cfg = wl.uniform_box(n=(2, 2, 2), bc_type="wall", T_w=T_w, precision=precision, Kn=1e6)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    s = oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])
    cen = nodes[tets].mean(1)
    c = int(np.argmin(cen[:, 0] + 10 * np.abs(cen[:, 1] - 0.25) + 10 * np.abs(cen[:, 2] - 0.25)))
    x = cen[c].astype(np.float32).astype(np.float64)
    speed = 16.0
    dt = float(np.float32(x[0] / speed * (1 + 1e-4)))
    out_u = []
    for k in range(3000):
        pid = (5 << 40) | (1 << 16) | k
        out = s.track_one(pid=pid, cell=c, x=x, u=[-speed, 0.0, 0.0], tau_cell=1.0, dt=dt, step=5)
        assert out["status"] == 0
        out_u.append(out["u"])
    U = np.array(out_u)
    assert np.all(U[:, 0] > 0)
    assert stats.kstest(U[:, 0] ** 2 / (2 * T_w), "expon").pvalue > 1e-4
    for comp in (1, 2):
        assert stats.kstest(U[:, comp] / np.sqrt(T_w), "norm").pvalue > 1e-4
