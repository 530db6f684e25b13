"""Pins for the oracle's walk on spheres (Sec. 3.1, Eq. 7, ball Green's function).

* the sphere sampler obeys the mean-value property and its gradient form;
* the source weights integrate the ball Green's function exactly (closed
  form of -Laplacian v = 1 in a ball: v(centre) = R^2 / (2 d));
* full walks match closed-form harmonic and Poisson solutions within the
  epsilon-shell bias plus 4 standard errors, in 2D and 3D;
* the l-ablation of the paper (start inside the shell => du/dn^ = 0).
"""
import numpy as np
import pytest

import oracle
from paper_2302_11825_gb300 import workloads as wl


def _draws(n, seed=1):
    u = np.empty((n, 3))
    for i in range(n):
        r = oracle.philox4x32_10([i, 0, 0, 0], [seed, 0])
        u[i] = [oracle.u01(int(w)) for w in r[:3]]
    return u


@pytest.mark.parametrize("dim", [2, 3])
def test_sphere_step_mean_value_and_gradient(dim):
    n = 40000
    U = _draws(n)
    c = np.array([0.2, -0.1, 0.3][:dim])
    R = 0.37
    if dim == 2:
        h = [(wl.POLY, wl.poly2d_coeffs({(3, 0): 1.0, (1, 2): -3.0, (1, 1): 2.0, (1, 0): 0.5}))]
    else:
        h = [(wl.EXP_TRIG, [1.0, 0.5, 0.3, 0.4])]
    om = np.empty((n, dim))
    wu = np.empty(n)
    wg = np.empty(n)
    rho = np.empty(n)
    for i in range(n):
        om[i], rho[i], wu[i], wg[i] = oracle.sphere_step(dim, R, *U[i])
    # directions: unit, mean 0, covariance I/d
    np.testing.assert_allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-12)
    assert np.all(np.abs(om.mean(0)) < 5 / np.sqrt(n))
    np.testing.assert_allclose(om.T @ om / n, np.eye(dim) / dim, atol=5 / np.sqrt(n))
    hv, hg = wl.eval_terms(h, dim, c[None] + R * om)
    h0, g0 = wl.eval_terms(h, dim, c[None])
    assert abs(hv.mean() - h0[0]) < 5 * hv.std() / np.sqrt(n)
    gs = (dim / R) * hv[:, None] * om
    assert np.all(np.abs(gs.mean(0) - g0[0]) < 5 * gs.std(0) / np.sqrt(n))
    # source weights: E[w_u] = -int_B G^B = -R^2/(2d)
    assert abs(wu.mean() + R * R / (2 * dim)) < 5 * wu.std() / np.sqrt(n)
    # gradient source term for f(y) = L.(y - c): E[w_g w f] = -L R^2 / (2(d+2))
    L = np.array([0.7, -0.4, 0.2][:dim])
    f = (rho[:, None] * om) @ L
    t = (wg * f)[:, None] * om
    assert np.all(np.abs(t.mean(0) + L * R * R / (2 * (dim + 2))) < 5 * t.std(0) / np.sqrt(n) + 1e-12)


def _check_walk_means(out, x, u, gu, dim, eps, W, grad_tol_scale=1.0):
    U = out["U"].reshape(len(x), W)
    G = out["grad"].reshape(len(x), W, dim)
    for k in range(len(x)):
        se = U[k].std() / np.sqrt(W)
        assert abs(U[k].mean() - u[k]) < 4 * se + 3 * eps * (1 + np.abs(gu[k]).max()), (k, U[k].mean(), u[k], se)
        gse = G[k].std(0) / np.sqrt(W)
        assert np.all(np.abs(G[k].mean(0) - gu[k]) < 4 * gse * grad_tol_scale + 0.02), (k, G[k].mean(0), gu[k])


def test_walks_2d_harmonic_and_poisson():
    V, F = wl.circle_polygon(256)
    bvh = oracle.BVH(V, F)
    x = np.array([[0.3, 0.2], [-0.5, 0.1], [0.0, -0.8], [0.6, 0.6]], np.float32)
    W, eps = 20000, 1e-4
    g = [(wl.POLY, wl.poly2d_coeffs({(3, 0): 1.0, (1, 2): -3.0}))]
    out = oracle.walks(bvh, g, [], x, W, eps, 1 << 14, seed=11)
    u, gu = wl.eval_terms(g, 2, x.astype(np.float64))
    _check_walk_means(out, x, u, gu, 2, eps, W)
    # Poisson: u = |x|^2/4, f = Laplacian u = 1
    gp = [(wl.POLY, wl.poly2d_coeffs({(2, 0): 0.25, (0, 2): 0.25}))]
    out = oracle.walks(bvh, gp, [(wl.POLY, [1.0])], x, W, eps, 1 << 14, seed=12)
    u, gu = wl.eval_terms(gp, 2, x.astype(np.float64))
    _check_walk_means(out, x, u, gu, 2, eps, W)


def test_walks_2d_gaussian_bump_source():
    V, F = wl.star_polygon(2000, 4)
    bvh = oracle.BVH(V, F)
    bump = wl.gauss_coeffs(0.2, [1.5], [(0.1, 0.05)])
    g = [(wl.POLY, wl.poly2d_coeffs({(1, 1): 1.0})), (wl.GAUSS, bump)]
    f = [(wl.GAUSS_LAPLACIAN, bump)]
    x = np.array([[0.1, 0.0], [0.3, 0.2], [-0.3, -0.2]], np.float32)
    W, eps = 20000, 1e-4
    out = oracle.walks(bvh, g, f, x, W, eps, 1 << 14, seed=13)
    u, gu = wl.eval_terms(g, 2, x.astype(np.float64))
    _check_walk_means(out, x, u, gu, 2, eps, W)


def test_walks_3d_harmonic_and_poisson():
    V, F, _ = wl.perturbed_icosphere(3, 1)
    bvh = oracle.BVH(V, F)
    x = np.array([[0.1, 0.2, -0.1], [-0.4, 0.1, 0.3], [0.0, 0.0, 0.7]], np.float32)
    W, eps = 10000, 1e-3
    g = [(wl.EXP_TRIG, [2.0, 0.5, 0.3, 0.4])]
    out = oracle.walks(bvh, g, [], x, W, eps, 1 << 14, seed=21)
    u, gu = wl.eval_terms(g, 3, x.astype(np.float64))
    _check_walk_means(out, x, u, gu, 3, eps, W)
    gp = [(wl.POLY, wl.poly3d_coeffs({(2, 0, 0): 1 / 6, (0, 2, 0): 1 / 6, (0, 0, 2): 1 / 6}))]
    out = oracle.walks(bvh, gp, [(wl.POLY, [1.0])], x, W, eps, 1 << 14, seed=22)
    u, gu = wl.eval_terms(gp, 3, x.astype(np.float64))
    _check_walk_means(out, x, u, gu, 3, eps, W)


def test_offset_inside_shell_gives_zero_normal_derivative():
    # Fig. "Ablations": l = 0.1 eps puts each ball inside the shell => du/dn^ = 0
    V, F = wl.circle_polygon(256)
    eps = 1e-3
    z, n, e, _ = oracle.sample_boundary(V, F, 64, 0.1 * eps, seed=1)
    g = [(wl.POLY, wl.poly2d_coeffs({(3, 0): 1.0, (1, 2): -3.0}))]
    out = oracle.walks(oracle.BVH(V, F), g, [], z.astype(np.float32), 4, eps, 1 << 14, seed=2)
    assert np.all(out["steps"] == 1)
    assert np.all(out["grad"] == 0.0)
    # U = g at the closest boundary point
    _, _, cp = oracle.BVH(V, F).closest(z.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(out["U"].reshape(64, 4)[:, 0], oracle.fn_eval(g, 2, cp), rtol=1e-12, atol=1e-14)


def test_walks_deterministic_and_capped():
    V, F = wl.circle_polygon(256)
    bvh = oracle.BVH(V, F)
    x = np.array([[0.1, 0.1]], np.float32)
    g = [(wl.POLY, wl.poly2d_coeffs({(1, 0): 1.0}))]
    a = oracle.walks(bvh, g, [], x, 64, 1e-4, 1 << 14, seed=5)
    b = oracle.walks(bvh, g, [], x, 64, 1e-4, 1 << 14, seed=5)
    c = oracle.walks(bvh, g, [], x, 64, 1e-4, 1 << 14, seed=5, id_base=64)
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["steps"], b["steps"])
    assert not np.array_equal(a["U"], c["U"])
    d = oracle.walks(bvh, g, [], x, 64, 1e-4, 3, seed=5)
    assert d["steps"].max() <= 3


def test_reduce_walks_is_the_per_sample_mean():
    # Alg. 1: u^ and du/dn^ of sample i are the means over its W walks of U
    # and of grad . n_i (n_i as stored, FP32)
    rng = np.random.default_rng(4)
    n, W, dim = 37, 9, 3
    U = rng.standard_normal(n * W)
    grad = rng.standard_normal((n * W, dim))
    nrm = rng.standard_normal((n, dim)).astype(np.float32)
    uh, qh = oracle.reduce_walks(U, grad, nrm, W)
    np.testing.assert_allclose(uh, U.reshape(n, W).mean(1), rtol=1e-13, atol=1e-15)
    q = np.einsum("iwd,id->iw", grad.reshape(n, W, dim), nrm.astype(np.float64)).mean(1)
    np.testing.assert_allclose(qh, q, rtol=1e-12, atol=1e-14)
    uh2, qh2 = oracle.reduce_walks(U, grad, None, W)
    assert qh2 is None and np.array_equal(uh2, uh)
