"""Many right-hand sides from one set of walks: Laplace (f = 0), and with a
source term f_k = sum_b A[k][b] psi_b over shared bumps.

The walks' paths do not depend on g, and U and n.grad of each walk are
linear in g (Sec. 3.1, Eq. 7).  So the batched path -- end-point walks,
per-sample monomial moments, projection -- must give, for every right-hand
side g_k, the u^ and du/dn^ of the single-RHS cache build with the same
seed up to rounding, and the batched gather must give the single-RHS Eq. 3
value.  Each g_k is a random harmonic polynomial, so it is also the exact
solution, and one right-hand side is compared with the oracle's pipeline.
"""
import numpy as np
import pytest
import torch

from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import difference_bound, oracle_cache, oracle_evaluate

pytestmark = pytest.mark.gpu


def _single(geom, coeffs_k, opts, dim, n, pts_soa):
    cache = bvc.cache_build(geom, [(wl.POLY, coeffs_k)], [], opts, bvc.Cache(dim, n))
    st = bvc.EvalState(pts_soa)
    bvc.evaluate(cache, st)
    u, _ = bvc.get_solution(st)
    return cache, u


def _check_against_single(geom, dim, n, W, l, eps, C, pts, ks, seed=3):
    opts = bvc.cache_opts(n, W, l, eps, seed)
    Cd = torch.tensor(C, dtype=torch.float64, device="cuda")
    mc = bvc.multi_cache_build(geom, Cd, opts, bvc.MultiCache(dim, n, C.shape[0]))
    pts_soa = bvc.soa(pts)
    um = bvc.evaluate_multi(mc, pts_soa)
    torch.cuda.synchronize()
    for k in ks:
        sc, us = _single(geom, C[k], opts, dim, n, pts_soa)
        torch.cuda.synchronize()
        assert torch.equal(sc.z, mc.z) and torch.equal(sc.nrm, mc.nrm)
        scale_u = sc.u_hat.abs().max().item()
        scale_q = sc.dudn_hat.abs().max().item()
        du = (mc.u_hat[k] - sc.u_hat).abs().max().item()
        dq = (mc.dudn_hat[k] - sc.dudn_hat).abs().max().item()
        dg = (um[k] - us).abs().max().item()
        print(f"[multi vs single] dim={dim} k={k} max|du^|={du:.2e} (scale {scale_u:.2e}) "
              f"max|dq^|={dq:.2e} (scale {scale_q:.2e}) max|du(x)|={dg:.2e}")
        # FP32 monomials and sums in both paths: a few FP32 ulps of the scale
        assert du <= 2e-5 * scale_u
        assert dq <= 2e-5 * scale_q
        assert dg <= 2e-5 * us.abs().max().item()
    return mc, um


def test_multi_2d_circle_matches_single_rhs():
    w = wl.circle_laplace(n_samples=2048, walks=16)
    geom = bvc.Geometry(w.V, w.F)
    C = wl.random_harmonic_polys(2, 40, seed=11)
    pts = w.eval_pts[:3000]
    _check_against_single(geom, 2, w.n_samples, w.walks, w.offset_l, w.eps, C, pts, ks=(0, 31, 32, 39))


def test_multi_2d_star_matches_single_rhs_and_closed_form():
    w = wl.star_poisson(n_samples=4096, walks=32, grid=40, n_seg=4000, manufactured=True)
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = w.eval_pts[~near]
    C = wl.random_harmonic_polys(2, 33, seed=12) * 0.5
    mc, um = _check_against_single(geom, 2, w.n_samples, w.walks, w.offset_l, w.eps, C, pts, ks=(5, 32))
    um = um.cpu().numpy()
    for k in (5, 32):
        exact, _ = wl.eval_terms([(wl.POLY, C[k])], 2, pts.astype(np.float64))
        rel = np.sqrt(np.mean((um[k] - exact) ** 2)) / np.sqrt(np.mean(exact ** 2))
        print(f"[multi star] k={k} relRMSE_vs_exact={rel:.3e}")
        assert rel < 0.1


def test_multi_3d_sphere_matches_single_rhs():
    V, F, r = wl.perturbed_icosphere(3, seed=2)
    eps = 1e-3 * wl.bbox_diagonal(V)
    geom = bvc.Geometry(V, F)
    C = wl.random_harmonic_polys(3, 35, seed=13)
    pts = wl.random_points_in(("sphere", (0.0, 0.0, 0.0), (0.9, 0.9, 0.9)), 2000, seed=4)
    _check_against_single(geom, 3, 2048, 8, 5 * eps, eps, C, pts, ks=(0, 34))


def test_multi_rhs_vs_oracle_pipeline():
    w = wl.circle_laplace(n_samples=1024, walks=16)
    geom = bvc.Geometry(w.V, w.F)
    C = wl.random_harmonic_polys(2, 3, seed=14)
    pts = w.eval_pts
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, 0)
    mc = bvc.multi_cache_build(geom, torch.tensor(C, device="cuda"), opts, bvc.MultiCache(2, w.n_samples, 3))
    um = bvc.evaluate_multi(mc, bvc.soa(pts)).cpu().numpy()
    for k in range(3):
        g = [(wl.POLY, C[k])]
        c = oracle_cache(w.V, w.F, g, [], w.n_samples, w.walks, w.offset_l, w.eps, 0)
        uo, _ = oracle_evaluate(c, pts.astype(np.float64))
        exact, _ = wl.eval_terms(g, 2, pts.astype(np.float64))
        du = np.abs(mc.u_hat[k].cpu().numpy() - c["u_hat"])
        dq = np.abs(mc.dudn_hat[k].cpu().numpy() - c["q_hat"])
        bound = difference_bound(c, du, dq, pts.astype(np.float64))
        print(f"[multi vs oracle] k={k} RMSE_vs_oracle={np.sqrt(np.mean((um[k] - uo) ** 2)):.3e} "
              f"RMSE_vs_exact={np.sqrt(np.mean((um[k] - exact) ** 2)):.3e} max|diff|/bound="
              f"{np.max(np.abs(um[k] - uo) / bound):.3f}")
        # element-wise: every point's difference is explained by the samples'
        # differences (walks that diverge between FP32 and FP64) and the
        # gather's FP32 tolerance
        assert np.all(np.abs(um[k] - uo) <= bound)


def test_reprojection_equals_rebuild_and_is_linear():
    w = wl.circle_laplace(n_samples=1024, walks=8)
    geom = bvc.Geometry(w.V, w.F)
    C1 = torch.tensor(wl.random_harmonic_polys(2, 20, seed=15), device="cuda")
    C2 = torch.tensor(wl.random_harmonic_polys(2, 20, seed=16), device="cuda")
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, 7)
    a = bvc.multi_cache_build(geom, C1, opts, bvc.MultiCache(2, w.n_samples, 20))
    b = bvc.multi_cache_build(geom, C2, opts, bvc.MultiCache(2, w.n_samples, 20))
    u1 = a.u_hat.clone()
    bvc.multi_cache_project(C2, a)
    torch.cuda.synchronize()
    assert torch.equal(a.mom_u, b.mom_u) and torch.equal(a.u_hat, b.u_hat)
    assert torch.equal(a.dudn_hat, b.dudn_hat) and torch.equal(a.packed, b.packed)
    bvc.multi_cache_project(C1 + C2, a)
    torch.cuda.synchronize()
    assert torch.allclose(a.u_hat, u1 + b.u_hat, rtol=1e-12, atol=1e-12)


def test_multi_rejects_source_grid_and_bad_shapes():
    w = wl.circle_laplace(n_samples=256, walks=4)
    geom = bvc.Geometry(w.V, w.F)
    C = torch.zeros((2, bvc.poly_terms(2)), dtype=torch.float64, device="cuda")
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, 0, src_grid=(8, 8))
    with pytest.raises(RuntimeError):
        bvc.multi_cache_build(geom, C, opts, bvc.MultiCache(2, w.n_samples, 2))
    with pytest.raises(ValueError):
        bvc.multi_cache_build(geom, C[:, :5].contiguous(), bvc.cache_opts(256, 4, w.offset_l, w.eps, 0),
                              bvc.MultiCache(2, w.n_samples, 2))


def _source_case(dim):
    if dim == 2:
        w = wl.star_poisson(n_samples=2048, walks=32, grid=48, n_seg=4000, src_grid=(64, 64))
        V, F, pts, l, eps = w.V, w.F, w.eval_pts, w.offset_l, w.eps
        sigma, centres, grid = w.meta["sigma"], w.meta["centres"], w.src_grid
    else:
        V, F, r = wl.perturbed_icosphere(3, seed=2)
        eps = 1e-3 * wl.bbox_diagonal(V)
        l = 5 * eps
        rng = np.random.default_rng(5)
        centres = rng.uniform(-0.4, 0.4, (5, 3))
        sigma, grid = 0.15, (24, 24, 24)
        pts = wl.random_points_in(("sphere", (0.0, 0.0, 0.0), (0.9, 0.9, 0.9)), 1500, seed=4)
    return V, F, pts, l, eps, sigma, centres, grid


@pytest.mark.parametrize("dim", [2, 3])
def test_multi_source_matches_single_rhs(dim):
    """Many right-hand sides with a source term: g_k polynomial, f_k = sum_b
    A[k][b] psi_b over shared bumps.  Each right-hand side's u^, du/dn^, source
    candidates and Eq. 3 + Eq. 4 value equal the single-RHS cache build with
    (g_k, f_k) on the same seed, up to rounding (per-bump FP32 sums against
    the single path's FP32 sum of f)."""
    V, F, pts, l, eps, sigma, centres, grid = _source_case(dim)
    geom = bvc.Geometry(V, F)
    near = bvc.classify_near(geom, bvc.soa(pts), l).cpu().numpy().astype(bool)
    pts = pts[~near]
    B = len(centres)
    shape = [(wl.GAUSS, wl.gauss_coeffs(sigma, np.ones(B), centres))]
    K = 37
    rng = np.random.default_rng(21 + dim)
    Cg = wl.random_harmonic_polys(dim, K, seed=17 + dim) * 0.5
    A = rng.uniform(-10.0, 10.0, (K, B))
    coeffs = np.concatenate([Cg, A], 1)
    n, W = 2048, 16 if dim == 3 else 32
    opts = bvc.cache_opts(n, W, l, eps, 9, src_grid=grid)
    M = bvc.n_candidates(dim, grid)
    mc = bvc.multi_cache_build_source(geom, shape, torch.tensor(coeffs, device="cuda"), opts,
                                      bvc.MultiCache(dim, n, K, n_src_cand=M))
    assert mc.n_bumps == B
    pts_soa = bvc.soa(pts)
    um = bvc.evaluate_multi(mc, pts_soa)
    torch.cuda.synchronize()
    for k in (0, 20, 36):
        f_k = [(wl.GAUSS, wl.gauss_coeffs(sigma, A[k], centres))]
        sc = bvc.cache_build(geom, [(wl.POLY, Cg[k])], f_k, opts, bvc.Cache(dim, n, n_src_cand=M))
        st = bvc.EvalState(pts_soa, grad=False)
        bvc.evaluate(sc, st)
        us, _ = bvc.get_solution(st)
        torch.cuda.synchronize()
        kept = int(sc.n_src_dev.item())
        assert kept == int(mc.n_src_dev.item()) and kept > 0
        assert torch.equal(sc.src_y[:, :kept], mc.src_y[:, :kept])
        assert torch.equal(sc.z, mc.z)
        scale_u = sc.u_hat.abs().max().item()
        scale_q = sc.dudn_hat.abs().max().item()
        du = (mc.u_hat[k] - sc.u_hat).abs().max().item()
        dq = (mc.dudn_hat[k] - sc.dudn_hat).abs().max().item()
        dg = (um[k] - us).abs().max().item()
        print(f"[multi source vs single] dim={dim} k={k} bumps={B} kept={kept}/{M} max|du^|={du:.2e} "
              f"(scale {scale_u:.2e}) max|dq^|={dq:.2e} (scale {scale_q:.2e}) max|du(x)|={dg:.2e} "
              f"(scale {us.abs().max().item():.2e})")
        # FP32 per-walk sums in both paths, in different orders
        assert du <= 5e-5 * scale_u
        assert dq <= 5e-5 * scale_q
        assert dg <= 5e-5 * us.abs().max().item()
        if dim == 2 and k == 20:
            # and against the oracle's pipeline for (g_k, f_k), element-wise
            c = oracle_cache(V, F, [(wl.POLY, Cg[k])], f_k, n, W, l, eps, 9, src_grid=grid)
            uo, _ = oracle_evaluate(c, pts.astype(np.float64))
            assert c["y"].shape[0] == kept
            c_multi = mc.src_psi[:kept, :B].cpu().numpy().astype(np.float64) @ A[k]
            dc = np.abs(c_multi - c["c"])
            bound = difference_bound(c, np.abs(mc.u_hat[k].cpu().numpy() - c["u_hat"]),
                                     np.abs(mc.dudn_hat[k].cpu().numpy() - c["q_hat"]), pts.astype(np.float64), dc)
            umk = um[k].cpu().numpy()
            print(f"[multi source vs oracle] k={k} max|diff|/bound={np.max(np.abs(umk - uo) / bound):.3f}")
            assert np.all(np.abs(umk - uo) <= bound)


def test_multi_source_reprojection_is_linear():
    V, F, pts, l, eps, sigma, centres, grid = _source_case(2)
    geom = bvc.Geometry(V, F)
    B = len(centres)
    shape = [(wl.GAUSS, wl.gauss_coeffs(sigma, np.ones(B), centres))]
    rng = np.random.default_rng(3)
    c1 = torch.tensor(rng.normal(size=(8, bvc.poly_terms(2) + B)), device="cuda")
    c2 = torch.tensor(rng.normal(size=(8, bvc.poly_terms(2) + B)), device="cuda")
    opts = bvc.cache_opts(512, 8, l, eps, 4, src_grid=grid)
    M = bvc.n_candidates(2, grid)
    a = bvc.multi_cache_build_source(geom, shape, c1, opts, bvc.MultiCache(2, 512, 8, n_src_cand=M))
    p = bvc.soa(pts[:500])
    u1 = bvc.evaluate_multi(a, p).clone()
    bvc.multi_cache_project(c2, a)
    u2 = bvc.evaluate_multi(a, p).clone()
    bvc.multi_cache_project(c1 + c2, a)
    u12 = bvc.evaluate_multi(a, p)
    torch.cuda.synchronize()
    scale = (u1.abs().max() + u2.abs().max()).item()
    assert (u12 - u1 - u2).abs().max().item() <= 1e-5 * scale
    with pytest.raises(ValueError):
        bvc.multi_cache_project(c1[:, :bvc.poly_terms(2)].contiguous(), a)
