"""Pins for the oracle's boundary and source samplers (Sec. 4 "Sampling",
Sec. 3.2 offset boundary, Alg. 1)."""
import numpy as np

import oracle
from paper_2302_11825_gb300 import workloads as wl


def test_boundary_samples_2d_stratified_and_offset():
    V, F = wl.circle_polygon(256)
    N, l = 1024, 1e-3
    z, n, e, jac = oracle.sample_boundary(V, F, N, l, seed=3)
    # equal elements + stratification: every element gets N/256 = 4 samples (+-1)
    counts = np.bincount(e, minlength=256)
    assert np.all(np.abs(counts - 4) <= 1)
    a = V[F[e, 0]].astype(np.float64)
    b = V[F[e, 1]].astype(np.float64)
    ab = b - a
    L = np.linalg.norm(ab, axis=1)
    # unit, outward normals, perpendicular to the element (a mitered offset
    # segment is parallel to its element)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-14)
    assert np.all(np.sum(n * (a + b), 1) > 0)
    np.testing.assert_allclose(np.sum(n * ab, 1), 0.0, atol=1e-14)
    # z sits at signed distance -l from the element's line
    np.testing.assert_allclose(np.sum((z - a) * n, 1), -l, atol=1e-14)
    # ... on the element's offset copy between its two mitered vertices
    # v - l (na + nb)/(1 + na.nb), at the same fraction lam of its length
    nn = np.stack([ab[:, 1], -ab[:, 0]], 1) / L[:, None]
    # turning angle at every vertex of the (FP32) polygon; the miter
    # shortens each end of an offset segment by l tan(angle / 2)
    Vd = V.astype(np.float64)
    ed = np.roll(Vd, -1, axis=0) - Vd
    ang = np.arctan2(ed[:, 1], ed[:, 0])
    turn = np.mod(ang - np.roll(ang, 1) + np.pi, 2 * np.pi) - np.pi   # at vertex v, between edges v-1 and v
    trim0 = l * np.tan(turn[F[e, 0]] / 2)
    trim1 = l * np.tan(turn[F[e, 1]] / 2)
    t = ab / L[:, None]
    p0 = a - l * nn + trim0[:, None] * t
    p1 = b - l * nn - trim1[:, None] * t
    lam = np.sum((z - p0) * (p1 - p0), 1) / np.sum((p1 - p0) ** 2, 1)
    assert np.all((lam >= -1e-12) & (lam <= 1 + 1e-12))
    np.testing.assert_allclose(p0 + lam[:, None] * (p1 - p0), z, atol=1e-14)
    # 1/p = |dOmega| jac: jac is the offset segment's length over the element's
    np.testing.assert_allclose(jac, (L - trim0 - trim1) / L, rtol=1e-12)
    # stratified in arclength: sample i lies in the i-th 1/N slice of the boundary
    T = L[0] * 256
    s = (e * L[0] + lam * L) / T
    i = np.arange(N)
    assert np.all(s >= i / N - 1e-12) and np.all(s <= (i + 1) / N + 1e-12)


def test_boundary_samples_3d_area_weighted_uniform():
    V, F = wl.icosphere(2)
    V = V.astype(np.float32)
    N, l = 32000, 1e-2
    z, n, e, jac = oracle.sample_boundary(V, F, N, l, seed=5)
    a = V[F[e, 0]].astype(np.float64)
    e1 = V[F[e, 1]].astype(np.float64) - a
    e2 = V[F[e, 2]].astype(np.float64) - a
    cr = np.cross(e1, e2)
    n0 = cr / np.linalg.norm(cr, axis=1)[:, None]
    # the offset triangle: vertices moved inward along their (angle-weighted,
    # normalised) vertex normals, scaled so that no incident face moves by
    # less than l -- written out here independently of the oracle
    Vd = V.astype(np.float64)
    fc = np.cross(Vd[F[:, 1]] - Vd[F[:, 0]], Vd[F[:, 2]] - Vd[F[:, 0]])
    fn = fc / np.linalg.norm(fc, axis=1)[:, None]
    Nv = np.zeros_like(Vd)
    for k in range(3):
        p = Vd[F[:, (k + 1) % 3]] - Vd[F[:, k]]
        q = Vd[F[:, (k + 2) % 3]] - Vd[F[:, k]]
        cosang = np.sum(p * q, 1) / np.linalg.norm(p, axis=1) / np.linalg.norm(q, axis=1)
        np.add.at(Nv, F[:, k], np.arccos(cosang)[:, None] * fn)
    Nv /= np.linalg.norm(Nv, axis=1)[:, None]
    cmin = np.full(V.shape[0], 2.0)
    for k in range(3):
        np.minimum.at(cmin, F[:, k], np.sum(fn * Nv[F[:, k]], 1))
    Vm = Vd - l * Nv / np.maximum(cmin, 0.25)[:, None]
    P0, P1, P2 = Vm[F[e, 0]], Vm[F[e, 1]], Vm[F[e, 2]]
    cm = np.cross(P1 - P0, P2 - P0)
    np.testing.assert_allclose(n, cm / np.linalg.norm(cm, axis=1)[:, None], atol=1e-12)
    np.testing.assert_allclose(jac, np.linalg.norm(cm, axis=1) / np.linalg.norm(cr, axis=1), rtol=1e-11)
    # inside the mesh, between l and l x max|m| below the element's plane
    d = -np.sum((z - a) * n0, 1)
    assert np.all(d >= l * (1 - 1e-9)) and np.all(d <= l / cmin.min() * (1 + 1e-9))
    p = z - P0
    # barycentric coordinates inside the offset triangle
    M = np.stack([P1 - P0, P2 - P0], 2)
    bc = np.linalg.solve(np.einsum("nij,nik->njk", M, M), np.einsum("nij,ni->nj", M, p)[..., None])[..., 0]
    assert np.all(bc >= -1e-9) and np.all(bc.sum(1) <= 1 + 1e-9)
    np.testing.assert_allclose(P0 + np.einsum("nij,nj->ni", M, bc), z, atol=1e-12)
    # element counts proportional to area, within the stratification bound
    area = 0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]).astype(np.float64), axis=1)
    counts = np.bincount(e, minlength=F.shape[0])
    assert np.all(np.abs(counts - N * area / area.sum()) <= 2.0)
    # uniform in the triangle: beta0 = 1 - b1 - b2 has CDF 1 - (1-x)^2
    b0 = np.sort(1 - bc.sum(1))
    cdf = 1 - (1 - b0) ** 2
    D = np.max(np.abs(cdf - (np.arange(N) + 0.5) / N))
    assert D < 1.95 / np.sqrt(N)


def test_source_samples_area_and_newtonian_potential():
    # unit disk (fine polygon), f = 1: the source estimator must approach the
    # disk's Newtonian potential int G dy = (|x|^2 - 1)/4, gradient x/2.
    V, F = wl.circle_polygon(4096)
    one = [(wl.POLY, [1.0])]
    y, c, ncand = oracle.sample_source2d(V, F, (128, 128), seed=2, f_terms=one)
    box = float(np.prod(V.max(0).astype(np.float64) - V.min(0).astype(np.float64)))
    area = 0.5 * 4096 * np.sin(2 * np.pi / 4096)
    frac = y.shape[0] / ncand
    se = np.sqrt(frac * (1 - frac) / ncand) * box
    assert abs(frac * box - area) < 4 * se
    np.testing.assert_allclose(c, box)
    x = np.array([[0.0, 0.0], [0.4, -0.3], [-0.6, 0.5]])
    ub, us, gb, gs = oracle.gather(np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0), np.zeros(0), 1.0, x, y, c)
    est = us / ncand
    gest = gs / ncand
    exact = (np.sum(x * x, 1) - 1) / 4
    # iid Monte Carlo error bound (stratification only lowers it)
    tol = 4 * np.sqrt(box * area / ncand) * 0.2 + 1e-3
    np.testing.assert_allclose(est, exact, atol=tol)
    np.testing.assert_allclose(gest, x / 2, atol=4 * tol)


def test_source_samples_kept_set_is_the_inside_test():
    V, F = wl.star_polygon(2000, 1)
    one = [(wl.POLY, [1.0])]
    y, c, ncand = oracle.sample_source2d(V, F, (64, 64), seed=9, f_terms=one)
    assert np.all(oracle.inside2d_f32(V, F, y) == 1)
    d, _, _ = oracle.BVH(V, F).closest(y.astype(np.float64))
    assert np.all(wl.inside_star_polygon(V, y.astype(np.float64))[d > 1e-5])
