"""Pins of the oracle's screened Poisson pieces ((Delta - sigma) u = 0,
App. A): the modified Bessel functions against scipy and their Wronskian;
the screened Green's function against the PDE (finite-difference
Laplacian), the unit flux as r -> 0, and its own derivatives; the walk's
ball factors C and Qg against sphere quadrature of exact solutions
exp(a.x), |a|^2 = sigma; the screened boundary integral equation (Eq. 2)
against exact solutions on a circle and a sphere; and the screened walks'
means against the closed form."""
import numpy as np
import pytest

import oracle
from paper_2302_11825_gb300 import workloads as wl

sp = pytest.importorskip("scipy.special")

EXP_COS = 5


def test_bessel_functions_match_scipy():
    for t in np.concatenate([np.logspace(-4, 2, 61), [1.999, 2.0, 2.001, 49.9, 50.1, 80.0]]):
        for n, mine, ref in ((0, oracle.bessel_i, sp.iv), (1, oracle.bessel_i, sp.iv)):
            assert abs(mine(n, t) - ref(n, t)) <= 1e-12 * ref(n, t), (n, t)
        for n in (0, 1):
            r = sp.kv(n, t)
            assert abs(oracle.bessel_k(n, t) - r) <= 1e-12 * r, (n, t)
        # Wronskian I0 K1 + I1 K0 = 1/t
        w = oracle.bessel_i(0, t) * oracle.bessel_k(1, t) + oracle.bessel_i(1, t) * oracle.bessel_k(0, t)
        assert abs(w * t - 1.0) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_green_function(dim):
    sigma = 2.3
    k = np.sqrt(sigma)
    rng = np.random.default_rng(dim)
    h = 1e-4
    for _ in range(5):
        x = rng.uniform(-1, 1, dim)
        y = rng.uniform(-1, 1, dim)
        n = rng.standard_normal(dim)
        n /= np.linalg.norm(n)
        out = oracle.green_sigma(dim, sigma, x, y, n)
        G = lambda xx: oracle.green_sigma(dim, sigma, xx, y, n)[0]
        # fourth-order central second differences (h = 1e-3)
        hh = 1e-3
        lap = sum((-G(x + 2 * hh * e) + 16 * G(x + hh * e) - 30 * G(x) + 16 * G(x - hh * e) - G(x - 2 * hh * e))
                  / (12 * hh ** 2) for e in np.eye(dim))
        assert abs(lap - sigma * out[0]) < 1e-6 * (1 + abs(sigma * out[0]))
        for a, e in enumerate(np.eye(dim)):
            assert abs((G(x + h * e) - G(x - h * e)) / (2 * h) - out[1 + a]) < 1e-6 * (1 + abs(out[1 + a]))
        Gy = lambda yy: oracle.green_sigma(dim, sigma, x, yy, n)[0]
        assert abs((Gy(y + h * n) - Gy(y - h * n)) / (2 * h) - out[1 + dim]) < 1e-6 * (1 + abs(out[1 + dim]))
        for a, e in enumerate(np.eye(dim)):
            dn = lambda xx: oracle.green_sigma(dim, sigma, xx, y, n)[1 + dim]
            fd = (dn(x + h * e) - dn(x - h * e)) / (2 * h)
            assert abs(fd - out[2 + dim + a]) < 1e-5 * (1 + abs(out[2 + dim + a]))
    # flux of dG/dn_y through a sphere of radius rho about x is Q(k rho) -> 1
    for rho in (1e-3, 0.3):
        t = k * rho
        q = t * sp.kv(1, t) if dim == 2 else np.exp(-t) * (t + 1)
        out = oracle.green_sigma(dim, sigma, np.zeros(dim), rho * np.eye(dim)[0], np.eye(dim)[0])
        area = 2 * np.pi * rho if dim == 2 else 4 * np.pi * rho ** 2
        assert abs(out[1 + dim] * area - q) < 1e-12


def _sphere_quadrature(dim, n=64):
    if dim == 2:
        th = 2 * np.pi * np.arange(n) / n
        return np.stack([np.cos(th), np.sin(th)], 1), np.full(n, 1.0 / n)
    xg, wg = np.polynomial.legendre.leggauss(n)
    ph = 2 * np.pi * np.arange(2 * n) / (2 * n)
    ct, P = np.meshgrid(xg, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    pts = np.stack([st * np.cos(P), st * np.sin(P), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(2 * n, 1.0 / (2 * n))[None, :] / 2).ravel()
    return pts, w


@pytest.mark.parametrize("dim", [2, 3])
def test_ball_factors_by_quadrature(dim):
    sigma = 4.0
    a = np.array([1.2, -1.6]) if dim == 2 else np.array([1.2, 0.0, -1.6])
    x = np.array([0.1, -0.2, 0.3][:dim])
    nu, w = _sphere_quadrature(dim)
    for R in (0.05, 0.7, 2.5):
        t = R * np.sqrt(sigma)
        Cf, Qg = oracle.screened_factors(dim, t)
        u = np.exp((x + R * nu) @ a)
        avg = np.sum(w * u)
        assert abs(Cf * avg - np.exp(x @ a)) < 1e-12 * np.exp(x @ a)
        grad = (dim / R) * Qg * np.sum(w[:, None] * u[:, None] * nu, 0)
        assert np.allclose(grad, a * np.exp(x @ a), rtol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_bie_reproduces_exact_solutions(dim):
    sigma = 3.0
    a = np.array([1.0, np.sqrt(2.0)]) if dim == 2 else np.array([1.0, 0.0, np.sqrt(2.0)])
    nu, w = _sphere_quadrature(dim, 256 if dim == 2 else 48)
    area = 2 * np.pi if dim == 2 else 4 * np.pi
    z = nu  # unit circle / sphere, outward normal = z
    u = np.exp(z @ a)
    dudn = (z @ a) * u
    for x in (np.zeros(dim), np.array([0.3, -0.4, 0.1][:dim])):
        G = np.array([oracle.green_sigma(dim, sigma, x, zi, zi) for zi in z])
        val = np.sum(w * area * (G[:, 1 + dim] * u - G[:, 0] * dudn))
        grad = np.sum((w * area)[:, None] * (G[:, 2 + dim:] * u[:, None] - G[:, 1:1 + dim] * dudn[:, None]), 0)
        assert abs(val - np.exp(x @ a)) < 1e-9
        assert np.allclose(grad, a * np.exp(x @ a), atol=1e-8)


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_walks_match_closed_form(dim):
    alpha, beta = 2.0, 1.0  # u = exp(alpha x_last) cos(beta x_0), sigma = alpha^2 - beta^2
    sigma = alpha ** 2 - beta ** 2
    if dim == 2:
        V, F = wl.circle_polygon(512)
    else:
        V, F = wl.icosphere(4)
        V = V.astype(np.float32)
    g = [(EXP_COS, [1.0, alpha, beta])]
    bvh = oracle.BVH(V, F)
    starts = np.array([[0.0, 0.0, 0.0][:dim], [0.3, -0.2, 0.1][:dim], [-0.5, 0.1, 0.2][:dim]], np.float32)
    W = 20000
    o = oracle.walks(bvh, g, [], starts, W, 1e-4, 1 << 14, 3, sigma=sigma)
    U = o["U"].reshape(3, W)
    exact = np.exp(alpha * starts[:, -1].astype(np.float64)) * np.cos(beta * starts[:, 0].astype(np.float64))
    se = U.std(1) / np.sqrt(W)
    assert np.all(np.abs(U.mean(1) - exact) < 4 * se + 2e-3 * np.abs(exact)), (U.mean(1), exact, se)
    # gradient: grad u . e for the first start, via the walks' gradient estimates
    gr = o["grad"].reshape(3, W, dim)[0].mean(0)
    gexact = np.zeros(dim)
    gexact[-1] = alpha * exact[0]
    gse = o["grad"].reshape(3, W, dim)[0].std(0) / np.sqrt(W)
    assert np.all(np.abs(gr - gexact) < 4 * gse + 1e-2), (gr, gexact, gse)


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_step_weights(dim):
    """The screened source weights of a step against what fixes them: their
    Poisson limit (sigma -> 0), the zero of the ball's Green's function on
    its sphere, and two integrals over the ball with closed forms.  With
    (sigma - Delta) v = 1 in B(0, R), v = 0 on the sphere, v(0) = (1 - C)/sigma,
    and v(0) = int_B G = (1/R) int_0^R -w_u(rho) drho; with (sigma - Delta) v =
    e.y, grad v(0) = e (1 - Qg)/sigma = -(e/(d R)) int_0^R w_g(rho) rho drho
    (C, Qg the ball factors of the same t = R sqrt(sigma))."""
    quad = pytest.importorskip("scipy.integrate").quad
    for R in (0.1, 0.8, 2.0):
        for rho in (1e-3 * R, 0.37 * R, 0.9 * R):
            _, _, wu0, wg0 = oracle.sphere_step(dim, R, 0.1, 0.2, rho / R)
            wu, wg = oracle.screened_step_weights(dim, 1e-14, R, rho)
            assert abs(wu - wu0) <= 1e-9 * abs(wu0) and abs(wg - wg0) <= 1e-9 * abs(wg0), (R, rho, wu, wu0, wg, wg0)
        for sigma in (0.5, 4.0, 30.0):
            t = R * np.sqrt(sigma)
            Cf, Qg = oracle.screened_factors(dim, t)
            wu_R, _ = oracle.screened_step_weights(dim, sigma, R, R * (1 - 1e-12))
            assert abs(wu_R) < 1e-9 * R * R
            iv = quad(lambda r: -oracle.screened_step_weights(dim, sigma, R, r)[0], 0.0, R, limit=200,
                      epsabs=1e-14, epsrel=1e-11)[0] / R
            assert abs(iv - (1.0 - Cf) / sigma) <= 1e-9 * (1.0 - Cf) / sigma, (dim, R, sigma, iv, (1 - Cf) / sigma)
            ig = -quad(lambda r: oracle.screened_step_weights(dim, sigma, R, r)[1] * r, 0.0, R, limit=200,
                       epsabs=1e-14, epsrel=1e-11)[0] / (dim * R)
            assert abs(ig - (1.0 - Qg) / sigma) <= 1e-9 * abs(1.0 - Qg) / sigma, (dim, R, sigma, ig, (1 - Qg) / sigma)


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_walks_with_source_match_closed_form(dim):
    """(Delta - sigma) u = f with u = exp(alpha x_last) cos(beta x_0) and
    sigma != alpha^2 - beta^2, so f = (alpha^2 - beta^2 - sigma) u: the walks'
    mean value and gradient at three points against u and grad u."""
    alpha, beta, sigma = 1.5, 1.0, 3.0
    lam = alpha ** 2 - beta ** 2 - sigma
    if dim == 2:
        V, F = wl.circle_polygon(512)
    else:
        V, F = wl.icosphere(4)
        V = V.astype(np.float32)
    g = [(EXP_COS, [1.0, alpha, beta])]
    f = [(EXP_COS, [lam, alpha, beta])]
    bvh = oracle.BVH(V, F)
    starts = np.array([[0.0, 0.0, 0.0][:dim], [0.3, -0.2, 0.1][:dim], [-0.5, 0.1, 0.2][:dim]], np.float32)
    W = 20000
    o = oracle.walks(bvh, g, f, starts, W, 1e-4, 1 << 14, 5, sigma=sigma)
    U = o["U"].reshape(3, W)
    s64 = starts.astype(np.float64)
    exact = np.exp(alpha * s64[:, -1]) * np.cos(beta * s64[:, 0])
    se = U.std(1) / np.sqrt(W)
    assert np.all(np.abs(U.mean(1) - exact) < 4 * se + 2e-3 * np.abs(exact)), (U.mean(1), exact, se)
    for j in range(3):
        gr = o["grad"].reshape(3, W, dim)[j].mean(0)
        gexact = np.zeros(dim)
        gexact[0] = -beta * np.exp(alpha * s64[j, -1]) * np.sin(beta * s64[j, 0])
        gexact[-1] = alpha * exact[j]
        gse = o["grad"].reshape(3, W, dim)[j].std(0) / np.sqrt(W)
        assert np.all(np.abs(gr - gexact) < 4 * gse + 1e-2), (j, gr, gexact, gse)
    # the source matters: without it the walks miss u by many standard errors
    o0 = oracle.walks(bvh, g, [], starts, 4000, 1e-4, 1 << 14, 5, sigma=sigma)
    U0 = o0["U"].reshape(3, 4000)
    assert np.any(np.abs(U0.mean(1) - exact) > 10 * U0.std(1) / np.sqrt(4000))
