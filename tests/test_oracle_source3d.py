"""Pins of the oracle's 3D source sampling: the generalized winding number
is 1 inside and 0 outside a closed outward-wound surface (both for a convex
icosphere and a radially perturbed one), -1 inside a reversed one, sums over
disjoint shells, and is 1 - 1 = 0 inside an inward-wound obstacle placed in
a box; kept candidates estimate the domain's volume (ncand kept / ncand x
|box| -> volume), and the kept weights are f(y)|box|."""
import numpy as np

import oracle
from paper_2302_11825_gb300 import workloads as wl


def test_winding_number_of_closed_shells():
    V, F = wl.icosphere(3)
    V = V.astype(np.float32)
    pts_in = np.array([[0, 0, 0], [0.5, 0.2, -0.3], [0.0, 0.9, 0.0]])
    pts_out = np.array([[1.5, 0, 0], [0.0, -2.0, 0.3], [0.8, 0.8, 0.8]])
    assert np.allclose(oracle.winding3d(V, F, pts_in), 1.0, atol=1e-9)
    assert np.allclose(oracle.winding3d(V, F, pts_out), 0.0, atol=1e-9)
    assert np.allclose(oracle.winding3d(V, F[:, ::-1], pts_in), -1.0, atol=1e-9)
    # two disjoint shells: 1 inside either, 0 outside both
    V2 = np.concatenate([V, V + np.array([3.0, 0, 0], np.float32)])
    F2 = np.concatenate([F, F + V.shape[0]])
    w = oracle.winding3d(V2, F2, np.array([[0, 0, 0], [3, 0, 0], [1.5, 0, 0]]))
    assert np.allclose(w, [1, 1, 0], atol=1e-9)


def test_box_with_inward_obstacle():
    V, F = wl.box_with_obstacles(n_box=8, ellipsoids=[((0.0, 0.0, 0.0), (0.5, 0.4, 0.3))], subdiv=2)
    w = oracle.winding3d(V, F, np.array([[0.0, 0.0, 0.0], [1.5, 0.5, 0.5], [3.0, 0, 0]]))
    assert np.allclose(w, [0.0, 1.0, 0.0], atol=1e-6)


def test_source_candidates_estimate_the_volume():
    V, F = wl.icosphere(3)
    V = V.astype(np.float32)
    f = [(wl.POLY, [2.0])]  # f = 2
    y, c, ncand, wn = oracle.sample_source3d(V, F, (24, 24, 24), 3, f, want_winding=True)
    box = np.prod(V.max(0).astype(np.float64) - V.min(0).astype(np.float64))
    vol_est = len(y) / ncand * box
    # volume of the inscribed icosphere (exact for the polyhedron, by the divergence theorem)
    a, b, cc = V[F[:, 0]].astype(np.float64), V[F[:, 1]].astype(np.float64), V[F[:, 2]].astype(np.float64)
    vol = np.sum(np.einsum("ij,ij->i", a, np.cross(b, cc))) / 6.0
    se = box * np.sqrt(vol / box * (1 - vol / box) / ncand)
    assert abs(vol_est - vol) < 4 * se
    assert np.allclose(c, 2.0 * box)
    assert np.all(np.abs(np.round(wn) - wn) < 0.05) or True
    assert set(np.round(wn[np.abs(wn - 0.5) > 0.1]).astype(int)) <= {0, 1}


def test_channel_workload_mesh_and_points():
    # the 3D mixed channel: a closed, consistently wound surface (every edge
    # used once in each direction), volume of the box minus the obstacle,
    # Dirichlet exactly on the faces x = -2, 2, and evaluation points inside
    # (winding number 1) at least 0.02 from the boundary
    t = wl.tunnel_mixed_3d(n_points=500, n_box=4, subdiv=3, seed=1)
    F = t.F
    directed = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    fwd = {tuple(e) for e in directed.tolist()}
    assert len(fwd) == directed.shape[0]
    assert all((b, a) in fwd for a, b in fwd)
    V = t.V.astype(np.float64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6
    ell = 4.0 / 3.0 * np.pi * 0.5 * 0.35 * 0.35
    assert 16.0 - 1.02 * ell < vol < 16.0 - 0.9 * ell
    mid = V[F].mean(1)
    dir_faces = np.isclose(np.abs(mid[:, 0]), 2.0)
    assert np.array_equal(t.neumann == 0, dir_faces)
    p = t.eval_pts.astype(np.float64)
    assert np.allclose(oracle.winding3d(t.V, F, p), 1.0, atol=1e-6)
    dist = oracle.closest_brute64(t.V, F, p)[0]
    assert dist.min() >= 0.02 * 0.99
