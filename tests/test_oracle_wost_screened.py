"""Pins of the oracle's screened walk on stars ((Delta - sigma) u = f with
Dirichlet and Neumann data, Eq. 1 with sigma > 0, Sec. 3.1): the ball's
screened Green's function against its radial equation, its zero on the
sphere, its unit flux at the centre and its sigma -> 0 limit; the step's
throughput factor W(r) against the flux of that Green's function, the
ball's mean-value factor and Green's identity for exp(a.x) on a sphere
inside the ball; reduction to the screened walk on spheres when there is no
Neumann element; and walk means against closed-form solutions with Neumann
data, with and without a source, inside and on the Neumann part, in 2D and
3D."""
import numpy as np
import pytest

import oracle
from paper_2302_11825_gb300 import workloads as wl

EXP_COS = 5  # A exp(alpha x_last) cos(beta x_0)


def _area(dim):
    return 2 * np.pi if dim == 2 else 4 * np.pi


@pytest.mark.parametrize("dim", [2, 3])
def test_ball_green_sigma_radial_equation_and_limits(dim):
    for sigma in (0.7, 4.0, 40.0):
        k = np.sqrt(sigma)
        for R in (0.05, 0.6, 2.0):
            G = lambda r: oracle.ball_green_sigma(dim, sigma, R, r)
            # zero on the ball's sphere
            assert abs(G(R)) <= 1e-12 * abs(G(0.5 * R))
            # (Delta - sigma) G = 0 away from the centre: G'' + (d-1)/r G' - k^2 G
            for r in (0.2 * R, 0.5 * R, 0.8 * R):
                h = 1e-3 * R
                g2 = (-G(r + 2 * h) + 16 * G(r + h) - 30 * G(r) + 16 * G(r - h) - G(r - 2 * h)) / (12 * h * h)
                g1 = (-G(r + 2 * h) + 8 * G(r + h) - 8 * G(r - h) + G(r - 2 * h)) / (12 * h)
                res = g2 + (dim - 1) / r * g1 - k * k * G(r)
                scale = abs(g2) + abs((dim - 1) / r * g1) + abs(k * k * G(r))
                assert abs(res) <= 1e-6 * scale, (sigma, R, r, res, scale)
            # the point source: the flux -|S| r^(d-1) G'(r) tends to 1 at the centre
            r = 1e-6 * R
            h = 1e-3 * r
            flux = -_area(dim) * r ** (dim - 1) * (G(r + h) - G(r - h)) / (2 * h)
            assert abs(flux - 1.0) < 1e-4, (sigma, R, flux)
    # sigma -> 0: the Laplace ball's Green's function
    for R, r in ((1.0, 0.3), (0.2, 0.15)):
        lap = np.log(R / r) / (2 * np.pi) if dim == 2 else (1 / r - 1 / R) / (4 * np.pi)
        assert abs(oracle.ball_green_sigma(dim, 1e-14, R, r) - lap) <= 1e-9 * lap
        assert oracle.ball_green_sigma(dim, 0.0, R, r) == pytest.approx(lap, rel=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_star_kernel_is_the_flux_of_the_ball_green_function(dim):
    for sigma in (0.5, 3.0, 30.0):
        for R in (0.1, 0.9, 2.5):
            G = lambda r: oracle.ball_green_sigma(dim, sigma, R, r)
            for r in (0.05 * R, 0.4 * R, 0.97 * R):
                h = 1e-4 * r
                flux = -_area(dim) * r ** (dim - 1) * (G(r + h) - G(r - h)) / (2 * h)
                W = oracle.star_kernel_sigma(dim, sigma, R, r)
                assert abs(W - flux) <= 1e-6 * abs(W) + 1e-10, (sigma, R, r, W, flux)
                assert 0.0 < W <= 1.0
            # at the sphere: the ball's screened mean-value factor (pinned by
            # sphere quadrature in test_oracle_screened.py)
            Cf, _ = oracle.screened_factors(dim, R * np.sqrt(sigma))
            assert abs(oracle.star_kernel_sigma(dim, sigma, R, R) - Cf) <= 1e-12 * Cf
            # at the centre and for sigma -> 0: 1 (the Laplace walk on stars)
            assert abs(oracle.star_kernel_sigma(dim, sigma, R, 1e-9 * R) - 1.0) < 1e-8
        assert oracle.star_kernel_sigma(dim, 0.0, 1.0, 0.4) == 1.0
        assert abs(oracle.star_kernel_sigma(dim, 1e-14, 1.0, 0.4) - 1.0) < 1e-12


def _sphere_quadrature(dim, n):
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
def test_star_step_green_identity_for_exponentials(dim):
    """Green's identity on B(x, r) inside B(x, R) with the ball's screened
    Green's function G (not zero on the inner sphere): for v = exp(a.y),
    |a|^2 = sigma, v(x) = W(r) avg_{|y-x|=r} v + G(r) (flux of grad v through
    that sphere) -- the star step's factor W and its Neumann weight G at once."""
    sigma = 2.5
    a = np.array([0.6, -np.sqrt(sigma - 0.36)]) if dim == 2 else np.array([0.6, 0.8, -np.sqrt(sigma - 1.0)])
    nu, w = _sphere_quadrature(dim, 256 if dim == 2 else 40)
    x = np.array([0.2, -0.1, 0.3][:dim])
    for R in (0.3, 1.0, 2.2):
        for r in (0.1 * R, 0.5 * R, 0.9 * R):
            y = x + r * nu
            v = np.exp(y @ a)
            avg = np.sum(w * v)
            flux = _area(dim) * r ** (dim - 1) * np.sum(w * (nu @ a) * v)
            W = oracle.star_kernel_sigma(dim, sigma, R, r)
            G = oracle.ball_green_sigma(dim, sigma, R, r)
            assert abs(W * avg + G * flux - np.exp(x @ a)) <= 1e-11 * np.exp(x @ a), (R, r)


def test_all_dirichlet_reduces_to_the_screened_walk_on_spheres():
    sigma = 3.0
    for V, F, starts, g, f in [
        (*wl.star_polygon(256, 0), 0.6 * wl.star_polygon(64, 0)[0][::3],
         [(EXP_COS, [1.0, 2.0, 1.0])], [(EXP_COS, [-1.0, 1.5, 1.0])]),
        (*wl.perturbed_icosphere(2, 0)[:2], 0.5 * wl.icosphere(1)[0][::5],
         [(EXP_COS, [1.0, 2.0, 1.0])], [(EXP_COS, [-1.0, 1.5, 1.0])]),
    ]:
        starts = np.asarray(starts, np.float32)
        w = oracle.Wost(V, F, np.zeros(F.shape[0]))
        a = w.walks(g, [], [], f, starts, None, 8, 1e-3, 4096, 5, sigma=sigma)
        b = oracle.walks(oracle.BVH(V, F), g, f, starts, 8, 1e-3, 4096, 5, sigma=sigma)
        np.testing.assert_array_equal(a["steps"], b["steps"])
        np.testing.assert_allclose(a["U"], b["U"], rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(a["grad"], b["grad"], rtol=1e-8, atol=1e-9)


def _z(U, W, exact):
    U = U.reshape(-1, W)
    se = U.std(1) / np.sqrt(W)
    return (U.mean(1) - exact) / se, U.mean(1) - exact


def _square():
    V, F, side = wl.rect_polygon((0.0, 0.0), (1.0, 1.0), 16)
    return V, F, side, (side % 2 == 0).astype(np.uint8)  # bottom and top Neumann


def _exp_cos(dim, alpha, beta, x):
    x = np.asarray(x, np.float64)
    u = np.exp(alpha * x[:, -1]) * np.cos(beta * x[:, 0])
    g = np.zeros_like(x)
    g[:, 0] = -beta * np.exp(alpha * x[:, -1]) * np.sin(beta * x[:, 0])
    g[:, -1] = alpha * u
    return u, g


@pytest.mark.parametrize("case", ["harmonic", "source"])
def test_screened_square_closed_form_inside(case):
    """u = exp(alpha y) cos(beta x) on the unit square, Neumann data
    h = n . grad u on the bottom and top sides (where u is not flat), u on
    the others; (Delta - sigma) u = (alpha^2 - beta^2 - sigma) u = f."""
    alpha, beta = 2.0, 1.0
    sigma = 3.0 if case == "harmonic" else 1.8
    lam = alpha ** 2 - beta ** 2 - sigma
    V, F, side, neu = _square()
    w = oracle.Wost(V, F, neu)
    u = [(EXP_COS, [1.0, alpha, beta])]
    f = [] if case == "harmonic" else [(EXP_COS, [lam, alpha, beta])]
    pts = np.random.default_rng(2).uniform(0.15, 0.85, (8, 2)).astype(np.float32)
    W = 4000
    o = w.walks(u, [], u, f, pts, None, W, 1e-4, 1 << 16, 41, sigma=sigma)
    ex, gex = _exp_cos(2, alpha, beta, pts)
    z, d = _z(o["U"], W, ex)
    assert np.all(np.abs(z) < 4.5), (z, d)
    G = o["grad"].reshape(-1, W, 2)
    zg = (G.mean(1) - gex) / (G.std(1) / np.sqrt(W))
    assert np.all(np.abs(zg) < 4.5), zg
    # the screening matters: the Laplace walk on stars misses u by many SE
    o0 = w.walks(u, [], u, f, pts, None, W, 1e-4, 1 << 16, 41)
    z0, _ = _z(o0["U"], W, ex)
    assert np.max(np.abs(z0)) > 10.0, z0


def test_screened_square_closed_form_on_the_neumann_boundary():
    alpha, beta, sigma = 2.0, 1.0, 1.8
    lam = alpha ** 2 - beta ** 2 - sigma
    V, F, side, neu = _square()
    w = oracle.Wost(V, F, neu)
    u = [(EXP_COS, [1.0, alpha, beta])]
    top = np.where(side == 2)[0][3:9]
    bottom = np.where(side == 0)[0][5:8]
    el = np.concatenate([top, bottom]).astype(np.int32)
    z = V[F[el]].astype(np.float64).mean(1).astype(np.float32)
    W = 4000
    o = w.walks(u, [], u, [(EXP_COS, [lam, alpha, beta])], z, el, W, 1e-4, 1 << 16, 42, sigma=sigma)
    zs, d = _z(o["U"], W, _exp_cos(2, alpha, beta, z)[0])
    assert np.all(np.abs(zs) < 4.5), (zs, d)
    assert np.all(o["grad"] == 0.0)


@pytest.mark.parametrize("case", ["harmonic", "source"])
def test_screened_cube_closed_form(case):
    b = wl.box_mixed_3d()
    w = oracle.Wost(b.V, b.F, b.neumann)
    alpha, beta = 1.5, 1.0
    sigma = alpha ** 2 - beta ** 2 if case == "harmonic" else 2.0
    lam = alpha ** 2 - beta ** 2 - sigma
    u = [(EXP_COS, [1.0, alpha, beta])]
    f = [] if case == "harmonic" else [(EXP_COS, [lam, alpha, beta])]
    pts = b.eval_pts[:6]
    W = 2000
    o = w.walks(u, [], u, f, pts, None, W, 1e-4, 1 << 16, 43, sigma=sigma)
    ex, gex = _exp_cos(3, alpha, beta, pts)
    z, d = _z(o["U"], W, ex)
    assert np.all(np.abs(z) < 4.5), (z, d)
    G = o["grad"].reshape(-1, W, 3)
    zg = (G.mean(1) - gex) / (G.std(1) / np.sqrt(W))
    assert np.all(np.abs(zg) < 4.5), zg


def test_screened_cube_closed_form_on_the_neumann_faces():
    b = wl.box_mixed_3d()
    w = oracle.Wost(b.V, b.F, b.neumann)
    alpha, beta, sigma = 1.5, 1.0, 2.0
    lam = alpha ** 2 - beta ** 2 - sigma
    u = [(EXP_COS, [1.0, alpha, beta])]
    rng = np.random.default_rng(13)
    els = rng.choice(np.where(b.neumann == 1)[0], 6, replace=False).astype(np.int32)
    bary = rng.dirichlet([2.0, 2.0, 2.0], els.size)
    z = np.einsum("ik,ikd->id", bary, b.V[b.F[els]].astype(np.float64)).astype(np.float32)
    W = 3000
    o = w.walks(u, [], u, [(EXP_COS, [lam, alpha, beta])], z, els, W, 1e-4, 1 << 16, 44, sigma=sigma)
    zs, d = _z(o["U"], W, _exp_cos(3, alpha, beta, z)[0])
    assert np.all(np.abs(zs) < 4.5), (zs, d)


def test_screened_mixed_cache_square_closed_form():
    """The whole mixed cache of Sec. 3.2 for the screened equation: Neumann
    samples carry h, offset Dirichlet samples screened walk-on-stars
    estimates of u and du/dn, and the screened gather of App. A evaluates
    Eq. 3 at interior points."""
    from tests.oracle_pipeline import mixed_pipeline
    alpha, beta = 2.0, 1.0
    sigma = alpha ** 2 - beta ** 2
    V, F, side, neu = _square()
    u = [(EXP_COS, [1.0, alpha, beta])]
    pts = wl.grid_points((0.1, 0.1), (0.9, 0.9), 12)
    uh, gh, _ = mixed_pipeline(V, F, neu, u, [], 4096, 64, 5e-3, 1e-3, 9, pts, sigma=sigma)
    ex, gex = _exp_cos(2, alpha, beta, pts)
    rmse = np.sqrt(np.mean((uh - ex) ** 2))
    assert rmse < 0.02 * (ex.max() - ex.min()), rmse
    # the Laplace cache of the same data misses by far more
    u0, _, _ = mixed_pipeline(V, F, neu, u, [], 4096, 64, 5e-3, 1e-3, 9, pts)
    assert np.sqrt(np.mean((u0 - ex) ** 2)) > 5 * rmse
