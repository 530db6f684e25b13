"""Pins for the oracle's offset Dirichlet boundary (Sec. 3.2, Fig. "Dirichlet
offset boundary"): the cache's samples lie on the boundary of a closed region
inside the domain, about l from the boundary, and the boundary integral
equation (Eq. 2) with the source samples refers to that region.

The checks below do not reuse the oracle's formulas: closedness is shown by
Green's representation formula, integrated with Gauss-Legendre / Dunavant
quadrature over the moved mesh, reproducing harmonic functions at interior
points; the miter by distances to the elements' lines; the region by areas."""
import numpy as np

import oracle
from paper_2302_11825_gb300 import workloads as wl


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1) / 2, w / 2


def _quad_2d(P, F, ngl=6):
    """Gauss-Legendre points, outward normals and weights on the segments of
    the polygon with vertex positions P (FP64)."""
    a, b = P[F[:, 0]], P[F[:, 1]]
    e = b - a
    L = np.linalg.norm(e, axis=1)
    n = np.stack([e[:, 1], -e[:, 0]], 1) / L[:, None]
    s, w = _gl(ngl)
    q = (a[:, None, :] + s[None, :, None] * e[:, None, :]).reshape(-1, 2)
    return q, np.repeat(n, ngl, 0), (L[:, None] * w[None, :]).reshape(-1)


# Dunavant's degree-4 rule on the triangle (6 points)
_DUN = [(0.445948490915965, 0.108103018168070, 0.223381589678011),
        (0.091576213509771, 0.816847572980459, 0.109951743655322)]


def _split(A, B, Cc, levels):
    """Each triangle cut into 4^levels congruent sub-triangles (midpoints)."""
    for _ in range(levels):
        ab, bc, ca = (A + B) / 2, (B + Cc) / 2, (Cc + A) / 2
        A, B, Cc = (np.concatenate(t) for t in ((A, ab, ca, ab), (ab, B, bc, bc), (ca, bc, Cc, ca)))
    return A, B, Cc


def _quad_3d(P, F, levels=0):
    bary, wts = [], []
    for a, b, w in _DUN:
        for perm in [(a, a, b), (a, b, a), (b, a, a)]:
            bary.append(perm)
            wts.append(w)
    bary, wts = np.array(bary), np.array(wts)
    A, B, Cc = _split(P[F[:, 0]], P[F[:, 1]], P[F[:, 2]], levels)
    cr = np.cross(B - A, Cc - A)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    n = cr / (2 * area)[:, None]
    q = (bary[None, :, 0, None] * A[:, None] + bary[None, :, 1, None] * B[:, None]
         + bary[None, :, 2, None] * Cc[:, None]).reshape(-1, 3)
    return q, np.repeat(n, len(wts), 0), (area[:, None] * wts[None]).reshape(-1)


def _representation(q, nq, wq, u, gu, x):
    """Eq. 2 with the oracle's gather: sum over quadrature nodes of
    (dG/dn u - G du/dn) w."""
    val, grad = u(q), gu(q)
    ub, _, _, _ = oracle.gather(q, nq, wq * val, wq * np.sum(grad * nq, 1), 1.0, x)
    return ub


def _harm2(p):
    return p[:, 0] ** 2 - p[:, 1] ** 2 + 0.3 * p[:, 0] ** 3 - 0.9 * p[:, 0] * p[:, 1] ** 2


def _harm2_grad(p):
    return np.stack([2 * p[:, 0] + 0.9 * p[:, 0] ** 2 - 0.9 * p[:, 1] ** 2, -2 * p[:, 1] - 1.8 * p[:, 0] * p[:, 1]], 1)


def _harm3(p):
    return np.exp(0.5 * p[:, 2]) * np.cos(0.3 * p[:, 0]) * np.sin(0.4 * p[:, 1])


def _harm3_grad(p):
    e, c, s = np.exp(0.5 * p[:, 2]), np.cos(0.3 * p[:, 0]), np.sin(0.4 * p[:, 1])
    return np.stack([-0.3 * e * np.sin(0.3 * p[:, 0]) * s, 0.4 * e * c * np.cos(0.4 * p[:, 1]), 0.5 * e * c * s], 1)


def test_offset_polygon_is_closed_and_reproduces_harmonic_functions():
    # star (convex lobes, concave valleys) and L-shape (one reflex corner)
    cases = [wl.star_polygon(4000, 0), wl.l_shape_polygon(8)[:2]]
    for V, F in cases:
        Vd = V.astype(np.float64)
        l = 5e-3 * wl.bbox_diagonal(V)
        m, reach = oracle.offset_disp(V, F)
        rng = np.random.default_rng(3)
        lo, hi = Vd.min(0), Vd.max(0)
        x = rng.uniform(lo, hi, (400, 2))
        x = x[oracle.inside2d_f32(V, F, x.astype(np.float32)) == 1]
        d, _, _ = oracle.BVH(V, F).closest(x)
        # points several element lengths away, where 24-point Gauss-Legendre
        # on each segment is exact to rounding
        hmax = np.max(np.linalg.norm(Vd[F[:, 1]] - Vd[F[:, 0]], axis=1))
        x = x[d > max(2 * l * reach, 2 * hmax)][:60]
        assert x.shape[0] >= 20
        moved = _representation(*_quad_2d(Vd - l * m, F, 24), _harm2, _harm2_grad, x)
        np.testing.assert_allclose(moved, _harm2(x), atol=1e-9)
        # elements translated one by one (not a closed curve) miss it
        a, b = Vd[F[:, 0]], Vd[F[:, 1]]
        nrm = np.stack([(b - a)[:, 1], -(b - a)[:, 0]], 1) / np.linalg.norm(b - a, axis=1)[:, None]
        s, w = _gl(24)
        q = ((a - l * nrm)[:, None, :] + s[None, :, None] * (b - a)[:, None, :]).reshape(-1, 2)
        wq = (np.linalg.norm(b - a, axis=1)[:, None] * w[None, :]).reshape(-1)
        trans = _representation(q, np.repeat(nrm, 24, 0), wq, _harm2, _harm2_grad, x)
        assert np.max(np.abs(trans - _harm2(x))) > 1e3 * np.max(np.abs(moved - _harm2(x)))


def test_offset_mesh_is_closed_and_reproduces_harmonic_functions():
    # smooth perturbed sphere and a box with an inward-wound ellipsoidal
    # obstacle (edges and corners, convex and concave)
    V1, F1, _ = wl.perturbed_icosphere(3, 0)
    V2, F2 = wl.box_with_obstacles(n_box=2, ellipsoids=[((0.0, 0.0, 0.0), (0.5, 0.35, 0.35))], subdiv=2)[:2]
    for V, F in ((V1, F1), (V2, F2)):
        Vd = V.astype(np.float64)
        l = 5e-3 * wl.bbox_diagonal(V)
        m, reach = oracle.offset_disp(V, F)
        rng = np.random.default_rng(5)
        x = rng.uniform(Vd.min(0), Vd.max(0), (3000, 3))
        x = x[np.abs(oracle.winding3d(V, F, x) - 1.0) < 1e-6]
        d, _, _ = oracle.BVH(V, F).closest(x)
        x = x[d > 4 * l * reach][:40]
        assert x.shape[0] >= 15
        moved = _representation(*_quad_3d(Vd - l * m, F, 3), _harm3, _harm3_grad, x)
        # every flat triangle cut into 64 and integrated by the degree-4 rule:
        # exact to ~1e-8 at these distances
        err = np.max(np.abs(moved - _harm3(x)))
        assert err < 2e-8, err
        A, B, Cc = Vd[F[:, 0]], Vd[F[:, 1]], Vd[F[:, 2]]
        fn = np.cross(B - A, Cc - A)
        fn /= np.linalg.norm(fn, axis=1)[:, None]
        trans = _representation(*_quad_3d_translated(Vd, F, fn, l, 3), _harm3, _harm3_grad, x)
        terr = np.max(np.abs(trans - _harm3(x)))
        assert terr > 1e3 * err, (terr, err)


def _quad_3d_translated(Vd, F, fn, l, levels):
    q, nq, wq = _quad_3d(Vd, F, levels)
    # _split orders sub-triangles level-major: element of sub-triangle t is t mod |F|
    per = len(wq) // F.shape[0] // 6
    fe = np.tile(np.arange(F.shape[0]), per)
    return q - l * np.repeat(fn[fe], 6, 0), nq, wq


def test_miter_keeps_every_offset_segment_at_distance_l():
    V, F = wl.star_polygon(2000, 2)
    Vd = V.astype(np.float64)
    l = 0.02
    m, reach = oracle.offset_disp(V, F)
    P = Vd - l * m
    a, b = Vd[F[:, 0]], Vd[F[:, 1]]
    e = b - a
    n = np.stack([e[:, 1], -e[:, 0]], 1) / np.linalg.norm(e, axis=1)[:, None]
    # both ends of every moved segment at signed distance -l from the line
    np.testing.assert_allclose(np.sum((P[F[:, 0]] - a) * n, 1), -l, atol=1e-13)
    np.testing.assert_allclose(np.sum((P[F[:, 1]] - a) * n, 1), -l, atol=1e-13)
    # reach = 1 / cos(half the largest turning angle)
    ang = np.arctan2(e[:, 1], e[:, 0])
    turn = np.abs(np.mod(ang - np.roll(ang, 1) + np.pi, 2 * np.pi) - np.pi)
    np.testing.assert_allclose(reach, 1.0 / np.cos(turn.max() / 2), rtol=1e-9)
    # a square's corners move along the diagonal by sqrt(2) l
    Vs, Fs, _ = wl.rect_polygon((0.0, 0.0), (1.0, 1.0), 4)
    ms, rs = oracle.offset_disp(Vs, Fs)
    np.testing.assert_allclose(rs, np.sqrt(2.0), rtol=1e-12)
    corner = np.all(np.isin(Vs, [0.0, 1.0]), axis=1)
    np.testing.assert_allclose(np.abs(ms[corner]), 1.0, rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(ms[~corner], axis=1), 1.0, rtol=1e-12)


def test_cube_corners_keep_every_face_at_distance_l():
    # box [-2,2]x[-1,1]^2: at a corner the three faces meet at right angles,
    # and the moved corner is l from all three planes (displacement sqrt(3) l)
    V, F = wl.box_surface((-2.0, -1.0, -1.0), (2.0, 1.0, 1.0), 2)
    m, reach = oracle.offset_disp(V, F)
    np.testing.assert_allclose(reach, np.sqrt(3.0), rtol=1e-12)
    Vd = V.astype(np.float64)
    corner = np.all(np.isin(np.abs(Vd), [1.0, 2.0]) & (np.abs(Vd) == np.array([2.0, 1.0, 1.0])), axis=1)
    assert corner.sum() == 8
    np.testing.assert_allclose(np.abs(m[corner]), 1.0, rtol=1e-12)
    # every moved face vertex moves inward by at least l along the face normal
    A, B, Cc = Vd[F[:, 0]], Vd[F[:, 1]], Vd[F[:, 2]]
    fn = np.cross(B - A, Cc - A)
    fn /= np.linalg.norm(fn, axis=1)[:, None]
    for k in range(3):
        assert np.all(np.sum(fn * m[F[:, k]], 1) >= 1.0 - 1e-12)


def test_samples_with_exact_data_reproduce_the_solution():
    """The sampler (z on the moved segments, 1/p = |dOmega| jac) composed with
    the gather (Eq. 3), given the exact u and du/dn at the samples, estimates
    u without the bias of translated elements."""
    V, F = wl.star_polygon(4000, 0)
    l = 5e-3 * wl.bbox_diagonal(V)
    N = 1 << 16
    z, n, e, jac = oracle.sample_boundary(V, F, N, l, seed=1)
    meas = oracle.boundary_measure(V, F)
    rng = np.random.default_rng(7)
    x = rng.uniform(-0.5, 0.5, (40, 2))
    u, q = _harm2(z), np.sum(_harm2_grad(z) * n, 1)
    ub, _, _, _ = oracle.gather(z, n, u, q, meas, x, jac=jac)
    err = np.max(np.abs(ub / N - _harm2(x)))
    # the same samples treated as translated elements (jac = 1)
    ub1, _, _, _ = oracle.gather(z, n, u, q, meas, x)
    err1 = np.max(np.abs(ub1 / N - _harm2(x)))
    assert err < 2e-4, err
    assert err1 > 10 * err, (err1, err)
    # E[jac] = |offset boundary| / |dOmega| (stratified, so very close)
    m, _ = oracle.offset_disp(V, F)
    P = V.astype(np.float64) - l * m
    L_off = np.sum(np.linalg.norm(P[F[:, 1]] - P[F[:, 0]], axis=1))
    np.testing.assert_allclose(jac.mean(), L_off / meas, rtol=1e-5)


def test_source_samples_fill_the_offset_region():
    V, F = wl.circle_polygon(1024)
    l = 0.05
    one = [(wl.POLY, [1.0])]
    y, c, ncand = oracle.sample_source2d(V, F, (160, 160), seed=3, f_terms=one, l=l)
    r = np.linalg.norm(y.astype(np.float64), axis=1)
    # inside the offset polygon (inradius cos(pi/1024) - l): nothing in the strip
    assert r.max() < 1.0 - l + 1e-6
    Vo = oracle.offset_vertices(V, F, l)
    assert np.all(oracle.inside2d_f32(Vo, F, y) == 1)
    # the kept fraction estimates the offset polygon's area
    box = float(np.prod(V.max(0).astype(np.float64) - V.min(0).astype(np.float64)))
    Vo64 = Vo.astype(np.float64)
    area = 0.5 * np.sum(Vo64[:, 0] * np.roll(Vo64[:, 1], -1) - np.roll(Vo64[:, 0], -1) * Vo64[:, 1])
    frac = y.shape[0] / ncand
    assert abs(frac * box - area) < 4 * np.sqrt(frac * (1 - frac) / ncand) * box
    # 3D: a sphere mesh's offset region is the ball of radius ~ 1 - l
    V3, F3 = wl.icosphere(3)
    V3 = V3.astype(np.float32)
    y3, _, n3 = oracle.sample_source3d(V3, F3, (20, 20, 20), 4, one, l=0.1)
    assert np.linalg.norm(y3.astype(np.float64), axis=1).max() < 0.9 + 1e-6


def test_mixed_offset_moves_only_dirichlet_elements():
    # unit square, Neumann top and bottom: the Dirichlet sides are moved by l,
    # the Neumann elements keep their vertices, junction vertices translate
    V, F, side = wl.rect_polygon((0.0, 0.0), (1.0, 1.0), 8)
    neu = (side % 2 == 0).astype(np.uint8)
    l = 0.03
    z, n, e, jac = oracle.sample_boundary_mixed(V, F, 4000, l, 2, neu)
    on_n = neu[e] == 1
    np.testing.assert_array_equal(jac[on_n], 1.0)
    Vd = V.astype(np.float64)
    a = Vd[F[e, 0]]
    d = np.sum((z - a) * n, 1)
    np.testing.assert_allclose(d[on_n], 0.0, atol=1e-15)
    np.testing.assert_allclose(d[~on_n], -l, atol=1e-14)
    np.testing.assert_allclose(jac[~on_n], 1.0, rtol=1e-13)
    m, _ = oracle.offset_disp(V, F, neu)
    assert np.all(np.linalg.norm(m, axis=1) <= 1.0 + 1e-12)
