"""Pins of the oracle's vertex-valued boundary data (the parameterisation
of g used by the differentiable solve): linear interpolation on the closest
element reproduces any affine function exactly, so walks with the vertex
values of an affine g equal walks with the closed-form g; and the estimator
is linear in the vertex values."""
import numpy as np

import oracle
from paper_2302_11825_gb300 import workloads as wl


def _affine(dim, x):
    c = np.array([0.3, -1.2, 0.7][:dim])
    return 0.5 + x @ c


def test_interpolation_of_affine_data_is_exact():
    for dim in (2, 3):
        if dim == 2:
            V, F = wl.star_polygon(500, seed=1)
        else:
            V, F, _ = wl.perturbed_icosphere(2, seed=1)
        bvh = oracle.BVH(V, F)
        gv = _affine(dim, V.astype(np.float64))
        rng = np.random.default_rng(0)
        e = rng.integers(0, F.shape[0], 200)
        if dim == 2:
            t = rng.uniform(0, 1, 200)[:, None]
            p = (1 - t) * V[F[e, 0]] + t * V[F[e, 1]]
        else:
            b = rng.dirichlet(np.ones(3), 200)
            p = b[:, :1] * V[F[e, 0]] + b[:, 1:2] * V[F[e, 1]] + b[:, 2:] * V[F[e, 2]]
        got = oracle.vertex_interp(bvh, gv, e, p.astype(np.float64))
        assert np.allclose(got, _affine(dim, p.astype(np.float64)), rtol=0, atol=1e-12)
        # a vertex indicator interpolates to the barycentric weight (hat function)
        j = F[e[0], 0]
        ind = np.zeros(V.shape[0])
        ind[j] = 1.0
        w0 = oracle.vertex_interp(bvh, ind, [e[0]], p[:1].astype(np.float64))[0]
        expect = (1 - t[0, 0]) if dim == 2 else b[0, 0]
        assert abs(w0 - expect) < 1e-12


def _disk(n, seed, r=0.6):
    # inside every star polygon of the generator (radius >= 1 - 0.3 - 0.05)
    rng = np.random.default_rng(seed)
    th = rng.uniform(0, 2 * np.pi, n)
    rr = r * np.sqrt(rng.uniform(0, 1, n))
    return np.stack([rr * np.cos(th), rr * np.sin(th)], 1).astype(np.float32)


def test_walks_with_vertex_data_match_closed_form_affine_g():
    V, F = wl.star_polygon(2000, seed=2)
    bvh = oracle.BVH(V, F)
    starts = _disk(50, 3)
    gterm = [(wl.POLY, [0.5, 0.3, -1.2])]  # 0.5 + 0.3 x - 1.2 y
    a = oracle.walks(bvh, gterm, [], starts, 8, 1e-3, 1 << 14, 5)
    b = oracle.walks(bvh, [], [], starts, 8, 1e-3, 1 << 14, 5, g_vertex=_affine(2, V.astype(np.float64)))
    assert np.array_equal(a["steps"], b["steps"])
    assert np.allclose(a["U"], b["U"], rtol=0, atol=1e-9)
    assert np.allclose(a["grad"], b["grad"], rtol=0, atol=1e-6)


def test_walk_estimates_are_linear_in_vertex_values():
    V, F = wl.star_polygon(1000, seed=4)
    bvh = oracle.BVH(V, F)
    starts = _disk(20, 5)
    rng = np.random.default_rng(6)
    g1, g2 = rng.standard_normal(V.shape[0]), rng.standard_normal(V.shape[0])
    f = [(wl.GAUSS, [0.1, 3.0, 0.2, 0.1])]
    r = [oracle.walks(bvh, [], f, starts, 4, 1e-3, 1 << 14, 7, g_vertex=gv) for gv in (g1, g2, 2 * g1 - 3 * g2)]
    r0 = oracle.walks(bvh, [], [], starts, 4, 1e-3, 1 << 14, 7, g_vertex=np.zeros(V.shape[0]))
    src = oracle.walks(bvh, [], f, starts, 4, 1e-3, 1 << 14, 7, g_vertex=np.zeros(V.shape[0]))
    # U(g, f) = U(g, 0) + U(0, f) and U(., 0) is linear in g
    lin = 2 * (r[0]["U"] - src["U"]) - 3 * (r[1]["U"] - src["U"]) + src["U"]
    assert np.allclose(r[2]["U"], lin, rtol=0, atol=1e-9 * (1 + np.abs(lin).max()))
    assert np.all(r0["U"] == 0.0)
