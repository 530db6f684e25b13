"""GPU parity for the screened walk on stars ((Delta - sigma) u = f with
Dirichlet and Neumann data, Eq. 1 with sigma > 0, Sec. 3.1) against the
oracle: the walks per walk when the Neumann data is zero (same paths, same
draws, the same throughput factors), the area-sampled Neumann term in
distribution, walks from the Neumann boundary, the reduction to the screened
walk on spheres, and the mixed cache (Sec. 3.2) with the screened gather and
the pointwise estimator against closed-form solutions and the oracle's
pipeline."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import mixed_pipeline

pytestmark = pytest.mark.gpu
EXP_COS = 5  # A exp(alpha x_last) cos(beta x_0)
ALPHA, BETA = 2.0, 1.0
SIGMA = ALPHA ** 2 - BETA ** 2  # u = exp(alpha x_last) cos(beta x_0) solves (Delta - sigma) u = 0
U = [(EXP_COS, [1.0, ALPHA, BETA])]


def _exact(x, alpha=ALPHA, beta=BETA):
    x = np.asarray(x, np.float64)
    return np.exp(alpha * x[:, -1]) * np.cos(beta * x[:, 0])


def _lshape():
    V, F = wl.l_shape_polygon(8)
    mid = wl.element_midpoints(V, F)
    return V, F, (mid[:, 0] > -1 + 1e-6).astype(np.uint8)


def _square():
    V, F, side = wl.rect_polygon((0.0, 0.0), (1.0, 1.0), 16)
    return V, F, (side % 2 == 0).astype(np.uint8), side


CASES = {
    "lshape": lambda: _lshape(),
    "cube": lambda: (wl.box_mixed_3d().V, wl.box_mixed_3d().F, wl.box_mixed_3d().neumann),
}


def _pts(case, n, seed):
    rng = np.random.default_rng(seed)
    if case == "cube":
        return rng.uniform(0.02, 0.98, (n, 3)).astype(np.float32)
    p = rng.uniform(-0.95, 0.95, (4 * n, 2))
    p = p[~((p[:, 0] > 0.0) & (p[:, 1] > 0.0))]
    return p[:n].astype(np.float32)


def _walk_parity(V, F, neu, g, h, f, starts, start_elem, nrm, W, eps, seed, sigma=SIGMA):
    m = bvc.Mixed(V, F, neu)
    w = oracle.Wost(V, F, neu)
    se = None if start_elem is None else torch.from_numpy(start_elem.astype(np.int32)).cuda()
    rec, steps, prim = bvc.mixed_walk(m, g, h, f, bvc.soa(starts), se, None if nrm is None else bvc.soa(nrm), W, eps,
                                      1 << 14, seed, debug=True, sigma=sigma)
    torch.cuda.synchronize()
    o = w.walks(g, h[0], h[1], f, starts, start_elem, W, eps, 1 << 14, seed, sigma=sigma)
    return rec.cpu().numpy(), steps.cpu().numpy(), prim.cpu().numpy(), o


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("src", [False, True])
def test_screened_walks_match_oracle_per_walk(case, src):
    # zero Neumann data: the same paths from the same draws, every step's
    # factor C or W(r) and the screened source weights on both sides
    V, F, neu = CASES[case]()
    dim = V.shape[1]
    f = [(EXP_COS, [-1.5, 1.5, 1.0])] if src else []
    starts = _pts(case, 96, 4)
    W = 32
    rec, steps, prim, o = _walk_parity(V, F, neu, U, ([], []), f, starts, None, None, W, 2e-3, 11)
    same = steps == o["steps"]
    assert same.mean() >= 0.97, same.mean()
    sc = np.abs(o["U"]).max() + 1e-9
    du = np.abs(rec[0] - o["U"])
    close = same & (du < 2e-4 * sc)
    assert close.mean() >= 0.97, close.mean()
    assert (prim[close] == o["prim"][close]).mean() >= 0.99
    for a in range(dim):
        dg = np.abs(rec[1 + a] - o["grad"][:, a])[close]
        assert np.quantile(dg, 0.99) < 2e-3 * (np.abs(o["grad"]).max() + 1e-9)
    # the screening is on: the Laplace walks of the same draws differ
    r0, _, _, _ = _walk_parity(V, F, neu, U, ([], []), f, starts, None, None, W, 2e-3, 11, sigma=0.0)
    assert np.mean(np.abs(r0[0] - rec[0]) > 1e-3 * sc) > 0.5


@pytest.mark.parametrize("case", list(CASES))
def test_screened_neumann_term_matches_oracle_in_distribution(case):
    V, F, neu = CASES[case]()
    starts = _pts(case, 8, 5)
    W = 4096
    rec, steps, _, o = _walk_parity(V, F, neu, U, ([], U), [], starts, None, None, W, 1e-3, 12)
    Ug, Uo = rec[0].reshape(-1, W), o["U"].reshape(-1, W)
    z = (Ug.mean(1) - Uo.mean(1)) / np.sqrt(Ug.var(1) / W + Uo.var(1) / W)
    assert np.all(np.abs(z) < 4.5), z
    zg = (Ug.mean(1) - _exact(starts)) / np.sqrt(Ug.var(1) / W)
    assert np.all(np.abs(zg) < 4.5), zg


def test_screened_walks_from_the_neumann_boundary():
    V, F, neu, side = _square()
    el = np.concatenate([np.where(side == 2)[0][3:9], np.where(side == 0)[0][5:8]]).astype(np.int32)
    z = V[F[el]].astype(np.float64).mean(1).astype(np.float32)
    n = np.zeros_like(z)
    n[:, 1] = np.where(side[el] == 2, 1.0, -1.0)
    W = 4096
    rec, steps, _, o = _walk_parity(V, F, neu, U, ([], U), [], z, el, n, W, 1e-4, 13)
    h = oracle.neumann_eval([], U, 2, z.astype(np.float64), n.astype(np.float64))
    np.testing.assert_allclose(rec[1].reshape(-1, W), np.repeat(h[:, None], W, 1), rtol=1e-6, atol=1e-6)
    Ug = rec[0].reshape(-1, W)
    zs = (Ug.mean(1) - _exact(z)) / np.sqrt(Ug.var(1) / W)
    assert np.all(np.abs(zs) < 4.5), zs


def test_screened_all_dirichlet_mixed_walks_equal_screened_walk_on_spheres():
    V, F = wl.star_polygon(512, 0)
    m = bvc.Mixed(V, F, np.zeros(F.shape[0]))
    g = bvc.Geometry(V, F)
    pts = np.random.default_rng(6).uniform(-0.7, 0.7, (256, 2)).astype(np.float32)
    pts = pts[wl.inside_star_polygon(V, pts.astype(np.float64))][:64]
    W = 256
    a = bvc.EvalState(bvc.soa(pts))
    b = bvc.EvalState(bvc.soa(pts))
    bvc.wost_estimate(m, U, None, [], a, W, 1e-3, 4096, 7, sigma=SIGMA)
    bvc.wos_estimate(g, U, [], b, W, 1e-3, 4096, 7, sigma=SIGMA)
    ua, _ = bvc.get_solution(a)
    ub, _ = bvc.get_solution(b)
    torch.cuda.synchronize()
    ua, ub = ua.cpu().numpy(), ub.cpu().numpy()
    # the same walks (all stars are balls): equal up to the rounding of
    # the two kernels' factor expressions and of paths that split
    assert np.median(np.abs(ua - ub) / np.abs(ub).max()) < 1e-5
    assert np.mean(np.abs(ua - ub) < 1e-3 * np.abs(ub).max()) > 0.9


def _solve(V, F, neu, N, W, l, eps, seed, pts, src_grid=(0, 0), f=()):
    m = bvc.Mixed(V, F, neu)
    opts = bvc.cache_opts(N, W, l, eps, seed, src_grid=src_grid, sigma=SIGMA)
    cache = bvc.Cache(V.shape[1], N, n_src_cand=bvc.n_candidates(V.shape[1], src_grid))
    bvc.mixed_cache_build(m, U, ([], U), list(f), opts, cache)
    assert cache.struct.sigma == SIGMA
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(cache, st)
    u, g = bvc.get_solution(st)
    torch.cuda.synchronize()
    return m, cache, u.cpu().numpy(), g.cpu().numpy()


def test_screened_mixed_cache_square_closed_form_and_oracle():
    V, F, neu, side = _square()
    pts = wl.grid_points((0.1, 0.1), (0.9, 0.9), 12).astype(np.float32)
    m, cache, u, _ = _solve(V, F, neu, 4096, 64, 5e-3, 1e-3, 9, pts)
    ex = _exact(pts)
    rng_u = ex.max() - ex.min()
    e_gpu = np.sqrt(np.mean((u - ex) ** 2))
    assert e_gpu < 0.02 * rng_u, e_gpu
    # the oracle's pipeline on the same samples and draws
    uo, _, (z, n, e, u_hat, q_hat) = mixed_pipeline(V, F, neu, U, [], 4096, 64, 5e-3, 1e-3, 9,
                                                    pts.astype(np.float64), sigma=SIGMA)
    np.testing.assert_array_equal(cache.z.cpu().numpy().T, z.astype(np.float32))
    onn = neu[e] == 1
    np.testing.assert_allclose(cache.dudn_hat.cpu().numpy()[onn], q_hat[onn], rtol=1e-6, atol=1e-6)
    # the per-sample estimates agree in distribution (the area-sampled
    # Neumann term picks its points differently on the two sides, so single
    # walks differ, and one cache's error is shared by all its points: the
    # oracle's own RMSE over seeds 9-16 spans 0.015-0.069 here)
    for dv in (cache.u_hat.cpu().numpy() - u_hat, (cache.dudn_hat.cpu().numpy() - q_hat)[~onn]):
        zd = dv.mean() / (dv.std() / np.sqrt(dv.size))
        assert abs(zd) < 4.5, zd
    e_orc = np.sqrt(np.mean((uo - ex) ** 2))
    assert e_orc < 0.02 * rng_u
    assert np.sqrt(np.mean((u - uo) ** 2)) < 3.0 * max(e_gpu, e_orc) + 1e-3
    # the screened gather of the same cache against the oracle's, element by element
    ub, _, _, _ = oracle.gather(cache.z.cpu().numpy().T, cache.nrm.cpu().numpy().T, cache.u_hat.cpu().numpy(),
                                cache.dudn_hat.cpu().numpy(), cache.struct.bnd_measure, pts.astype(np.float64),
                                jac=cache.jac.cpu().numpy(), sigma=SIGMA)
    _, _, _, _, ab = oracle.gather(cache.z.cpu().numpy().T, cache.nrm.cpu().numpy().T, cache.u_hat.cpu().numpy(),
                                   cache.dudn_hat.cpu().numpy(), cache.struct.bnd_measure, pts.astype(np.float64),
                                   jac=cache.jac.cpu().numpy(), sigma=SIGMA, want_abs=True)
    err = np.abs(u - ub / 4096) / np.maximum(np.abs(ub / 4096), ab[:, 0] / 4096)
    assert err.max() < 1e-5, err.max()


def test_screened_mixed_cache_cube_closed_form_and_pointwise():
    b = wl.box_mixed_3d()
    pts = np.random.default_rng(2).uniform(0.15, 0.85, (1500, 3)).astype(np.float32)
    m, cache, u, _ = _solve(b.V, b.F, b.neumann, 4096, 64, b.offset_l, b.eps, 3, pts)
    ex = _exact(pts)
    assert np.sqrt(np.mean((u - ex) ** 2)) < 0.03 * (ex.max() - ex.min())
    # pointwise walks on stars at a few points: within 4.5 SE of u
    W = 2048
    st = bvc.EvalState(bvc.soa(pts[:16]))
    bvc.wost_estimate(m, U, ([], U), [], st, W, b.eps, 1 << 14, 5, sigma=SIGMA)
    up, _ = bvc.get_solution(st)
    rec, _, _ = bvc.mixed_walk(m, U, ([], U), [], bvc.soa(pts[:16]), None, None, W, b.eps, 1 << 14, 5, tag=3,
                               sigma=SIGMA)
    torch.cuda.synchronize()
    Ug = rec[0].cpu().numpy().reshape(16, W)
    np.testing.assert_allclose(up.cpu().numpy(), Ug.astype(np.float64).mean(1), rtol=1e-5, atol=1e-6)
    zs = (Ug.mean(1) - ex[:16]) / np.sqrt(Ug.var(1) / W)
    assert np.all(np.abs(zs) < 4.5), zs


def test_screened_arguments_checked():
    V, F, neu, _ = _square()
    m = bvc.Mixed(V, F, neu)
    pts = bvc.soa(np.full((4, 2), 0.5, np.float32))
    st = bvc.EvalState(pts)
    for s in (-1.0, float("nan"), float("inf")):
        with pytest.raises(bvc.BvcError):
            bvc.wost_estimate(m, U, None, [], st, 8, 1e-3, 64, 1, sigma=s)
        with pytest.raises(bvc.BvcError):
            bvc.mixed_walk(m, U, None, [], pts, None, None, 8, 1e-3, 64, 1, sigma=s)
    opts = bvc.cache_opts(64, 8, 5e-3, 1e-3, 1, sigma=1.0, clamp_c=2.0)
    with pytest.raises(bvc.BvcError):
        bvc.mixed_cache_build(m, U, None, [], opts, bvc.Cache(2, 64))
