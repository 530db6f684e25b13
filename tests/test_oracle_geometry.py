"""Pins for the oracle's geometry: closest point, BVH, inside test, measures."""
import numpy as np
import pytest

import oracle
from paper_2302_11825_gb300 import workloads as wl


def _query_points(V, rng, n, dim):
    lo, hi = V.min(0) - 0.3, V.max(0) + 0.3
    far = rng.uniform(lo, hi, (n, dim))
    # points very close to the boundary: vertices and edge points nudged
    idx = rng.integers(0, V.shape[0], n // 2)
    near = V[idx] + rng.normal(0, 1e-4, (n // 2, dim))
    return np.concatenate([far, near])


@pytest.mark.parametrize("mesh", ["circle", "star", "sphere"])
def test_bvh_equals_brute_force(mesh):
    rng = np.random.default_rng(0)
    if mesh == "circle":
        V, F = wl.circle_polygon(256)
    elif mesh == "star":
        V, F = wl.star_polygon(2000, 1)
    else:
        V, F, _ = wl.perturbed_icosphere(3, 2)
    dim = V.shape[1]
    pts = _query_points(V.astype(np.float64), rng, 2000, dim)
    d0, p0, c0 = oracle.closest_brute64(V, F, pts)
    bvh = oracle.BVH(V, F)
    d1, p1, c1 = bvh.closest(pts)
    assert np.array_equal(p0, p1)
    assert np.array_equal(d0, d1)
    assert np.array_equal(c0, c1)


def test_triangle_closest_point_matches_independent_method():
    # independent method: project on the plane if the projection is inside,
    # else the best of the three edge (segment) projections.
    rng = np.random.default_rng(3)
    for _ in range(300):
        T = rng.uniform(-1, 1, (3, 3)).astype(np.float32)
        p = rng.uniform(-2, 2, 3)
        d, prim, c = oracle.closest_brute64(T, np.array([[0, 1, 2]]), p[None])
        a, b, cc = T.astype(np.float64)
        n = np.cross(b - a, cc - a)
        n /= np.linalg.norm(n)
        q = p - np.dot(p - a, n) * n
        # barycentric inside test
        M = np.stack([b - a, cc - a], 1)
        st, *_ = np.linalg.lstsq(M, q - a, rcond=None)
        best = np.inf
        if st[0] >= 0 and st[1] >= 0 and st.sum() <= 1:
            best = np.linalg.norm(p - q)
        for u, v in ((a, b), (b, cc), (cc, a)):
            t = np.clip(np.dot(p - u, v - u) / np.dot(v - u, v - u), 0, 1)
            best = min(best, np.linalg.norm(p - (u + t * (v - u))))
        assert abs(d[0] - best) < 1e-12


def test_segment_closest_point_dense_sampling():
    rng = np.random.default_rng(5)
    for _ in range(200):
        S = rng.uniform(-1, 1, (2, 2)).astype(np.float32)
        p = rng.uniform(-2, 2, 2)
        d, _, _ = oracle.closest_brute64(S, np.array([[0, 1]]), p[None])
        t = np.linspace(0, 1, 20001)
        S64 = S.astype(np.float64)
        pts = S64[0][None] + t[:, None] * (S64[1] - S64[0])[None]
        dd = np.min(np.linalg.norm(pts - p[None], axis=1))
        assert d[0] <= dd + 1e-12
        assert dd - d[0] < 1e-7


@pytest.mark.parametrize("mesh", ["star", "sphere"])
def test_fp32_canonical_argmin_agrees_with_fp64(mesh):
    rng = np.random.default_rng(9)
    if mesh == "star":
        V, F = wl.star_polygon(2000, 1)
    else:
        V, F, _ = wl.perturbed_icosphere(3, 2)
    dim = V.shape[1]
    pts = _query_points(V.astype(np.float64), rng, 1000, dim).astype(np.float32)
    d2_32, p32 = oracle.closest_brute32(V, F, pts)
    d64, p64, _ = oracle.closest_brute64(V, F, pts.astype(np.float64))
    # the FP32 distance tracks the FP64 one
    np.testing.assert_allclose(np.sqrt(d2_32.astype(np.float64)), d64, rtol=1e-5, atol=2e-6)
    # the FP32 choice is (one of) the FP64 minimisers up to rounding
    for i in range(pts.shape[0]):
        if p32[i] != p64[i]:
            dc, _, _ = oracle.closest_brute64(V, F[p32[i]:p32[i] + 1], pts[i:i + 1].astype(np.float64))
            assert dc[0] - d64[i] <= 1e-6 * max(1.0, d64[i])


def test_inside_test_matches_exact_classification():
    rng = np.random.default_rng(11)
    V, F = wl.star_polygon(20000, 0)
    pts = rng.uniform(V.min(0), V.max(0), (20000, 2)).astype(np.float32)
    exact = wl.inside_star_polygon(V, pts.astype(np.float64))
    got = oracle.inside2d_f32(V, F, pts).astype(bool)
    d, _, _ = oracle.BVH(V, F).closest(pts.astype(np.float64))
    far = d > 1e-5
    assert np.array_equal(got[far], exact[far])
    Vc, Fc = wl.circle_polygon(256)
    r = np.linalg.norm(pts, axis=1)
    gc = oracle.inside2d_f32(Vc, Fc, pts).astype(bool)
    assert np.all(gc[r < 0.99]) and not np.any(gc[r > 1.01])


def test_boundary_measures():
    V, F = wl.circle_polygon(256)
    assert abs(oracle.boundary_measure(V, F) - 256 * 2 * np.sin(np.pi / 256)) < 1e-6
    V, F = wl.icosphere(0)
    edge = 4.0 / np.sqrt(10 + 2 * np.sqrt(5))
    assert abs(oracle.boundary_measure(V, F) - 20 * np.sqrt(3) / 4 * edge ** 2) < 1e-5


def test_mesh_orientation_is_outward():
    # signed volume > 0 for outward counter-clockwise triangles; signed area > 0
    V, F, _ = wl.perturbed_icosphere(2, 0)
    a, b, c = V[F[:, 0]].astype(np.float64), V[F[:, 1]].astype(np.float64), V[F[:, 2]].astype(np.float64)
    vol = np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6
    assert 0.95 * 4 / 3 * np.pi < vol < 4 / 3 * np.pi * 1.03
    V, F = wl.star_polygon(2000, 0)
    a, b = V[F[:, 0]].astype(np.float64), V[F[:, 1]].astype(np.float64)
    assert np.sum(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]) / 2 > 0
