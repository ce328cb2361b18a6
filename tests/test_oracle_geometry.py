"""Pins of the oracle's mesh geometry and time step (Sec. 2.4 (a)).

Volumes sum to the box; every tet closes (sum of outward face vectors = 0);
planes contain their nodes; normals point from owner to neighbour; the
projected areas dS^x = 1/2 sum |S^x| equal the area of the tet's shadow on the
y-z plane (a property of any convex body, computed here by a 2D convex hull);
the oracle's dt equals the printed formula evaluated independently.
"""
import numpy as np
import pytest
from scipy.spatial import ConvexHull

import oracle
from paper_2007_13091_gb300 import workloads as wl


@pytest.fixture(scope="module")
def jittered():
    cfg = wl.uniform_box(n=(3, 4, 2), size=(1.5, 1.0, 0.7), jitter_amount=0.25, seed=5)
    return cfg, oracle.OracleSim(cfg["mesh"], cfg["W0"], cfg["params"])


def test_volumes_and_closure(jittered):
    cfg, s = jittered
    vol = s.geometry("vol")
    assert vol.sum() == pytest.approx(1.5 * 1.0 * 0.7, rel=1e-13)
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    p = nodes[tets]
    ref = np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0])) / 6
    np.testing.assert_allclose(vol, ref, rtol=1e-13)
    n = s.geometry("face_normal")
    A = s.geometry("face_area")
    own = s.geometry("face_owner").astype(int)
    nb = s.geometry("face_nbr").astype(int)
    nc = len(tets)
    acc = np.zeros((nc, 3))
    np.add.at(acc, own, (n * A).T)
    inner = nb >= 0
    np.add.at(acc, nb[inner], -(n * A).T[inner])
    assert np.abs(acc).max() < 1e-15


def test_planes_and_orientation(jittered):
    cfg, s = jittered
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    n = s.geometry("face_normal")
    d = s.geometry("face_d")
    own = s.geometry("face_owner").astype(int)
    nb = s.geometry("face_nbr").astype(int)
    cen = s.geometry("centroid")
    # each face plane contains three nodes of its owner, and the owner's fourth
    # node lies strictly inside (n.x < d)
    for f in range(len(d)):
        vals = nodes[tets[own[f]]] @ n[:, f] - d[f]
        on = np.abs(vals) < 1e-13
        assert on.sum() == 3 and vals[~on][0] < 0
    inner = nb >= 0
    assert np.all(np.einsum("ij,ji->i", (cen[:, nb[inner]] - cen[:, own[inner]]).T, n[:, inner]) > 0)


def test_projected_areas_are_shadows(jittered):
    cfg, s = jittered
    nodes, tets = cfg["mesh"]["nodes"], cfg["mesh"]["tets"]
    dS = s.geometry("dS")
    for i in range(0, len(tets), 7):
        for axis in range(3):
            keep = [a for a in range(3) if a != axis]
            pts = nodes[tets[i]][:, keep]
            area = ConvexHull(pts).volume  # 2D hull "volume" is its area
            assert dS[axis, i] == pytest.approx(area, rel=1e-12)


def test_dt_formula():
    cfg = wl.shock_tube(nx=10, ny=2, nz=2)
    W0 = cfg["W0"].copy()
    W0[1] += 0.3 * W0[0]  # give the gas a velocity so |U| enters the formula
    W0[4] += 0.5 * 0.09 * cfg["W0"][0] + 0.0
    s = oracle.OracleSim(cfg["mesh"], W0, cfg["params"])
    s.step()
    rho = W0[0]
    U = W0[1:4] / rho
    p = (W0[4] - 0.5 * rho * (U * U).sum(0)) / 1.5
    c = 3.0 * np.sqrt(p / rho)
    dS = s.geometry("dS")
    lam = ((np.abs(U) + c) * dS).sum(0)
    dt = cfg["params"]["CFL"] * np.min(s.geometry("vol") / lam)
    assert s.last("dt") == pytest.approx(dt, rel=1e-14)


def test_mesh_errors():
    cfg = wl.uniform_box(n=(2, 2, 2))
    m = dict(cfg["mesh"])
    bad = m["tets"].copy()
    bad[0] = bad[0][[0, 1, 3, 2]]  # inverted tet
    with pytest.raises(ValueError, match="volume"):
        oracle.OracleSim({**m, "tets": bad}, cfg["W0"], cfg["params"])
    with pytest.raises(ValueError, match="boundary tag"):
        oracle.OracleSim({**m, "bfaces": m["bfaces"][1:], "btags": m["btags"][1:]}, cfg["W0"], cfg["params"])


def test_blunt_vehicle_mesh_and_start_up():
    """The generated blunt vehicle: positive volumes, the body carved out (no
    tet inside it), body faces on or near the sphere-cone surface (every
    node moved there where the volumes allow it), box sides and body tagged;
    gas-kinetic start-up steps with local time steps from the impulsive start
    keep density and pressure positive and fill the base region."""
    cfg = wl.blunt_vehicle(h0=0.1, growth=1.5)
    m, body = cfg["mesh"], cfg["body"]
    nodes, tets, bf, tags = m["nodes"], m["tets"], m["bfaces"], m["btags"]
    assert wl._volumes(nodes, tets).min() > 0.0
    # carved out: no tet lies inside the body; the staircase leaves a few
    # centroids within the surface's curvature
    assert not body.inside(nodes[tets]).all(1).any()
    assert body.inside(nodes[tets].mean(1)).mean() < 0.01
    on = np.unique(bf[tags == 2])
    d = np.linalg.norm(body.closest(nodes[on]) - nodes[on], axis=1)
    assert d.max() < 0.1 and (d < 1e-12).mean() > 0.3
    assert set(np.unique(tags).tolist()) == {0, 1, 2}
    x0 = nodes[bf[tags == 0]][:, :, 0]
    assert np.all(x0 == -1.0)
    s = oracle.OracleSim(m, cfg["W0"], cfg["params"])
    s.gks_step(150, local=True)
    W = s.state()["W"]
    U = W[1:4] / W[0]
    p = (W[4] - 0.5 * W[0] * (U * U).sum(0)) / 1.5
    assert W[0].min() > 0.0 and p.min() > 0.01
    cen = nodes[tets].mean(1)
    base = (cen[:, 0] > 1.0) & (cen[:, 0] < 1.1) & (np.hypot(cen[:, 1], cen[:, 2]) < 0.2)
    assert base.any() and W[0][base].max() < 0.5  # the wake behind the base
