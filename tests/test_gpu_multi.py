"""Many right-hand sides (Laplace, f = 0) from one set of walks.

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
from tests.oracle_pipeline import oracle_bvc

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
        uo, _ = oracle_bvc(w.V, w.F, g, [], w.n_samples, w.walks, w.offset_l, w.eps, pts, 0)
        exact, _ = wl.eval_terms(g, 2, pts.astype(np.float64))
        rmse_oracle = np.sqrt(np.mean((um[k] - uo) ** 2))
        rmse_exact = np.sqrt(np.mean((um[k] - exact) ** 2))
        print(f"[multi vs oracle] k={k} RMSE_vs_oracle={rmse_oracle:.3e} RMSE_vs_exact={rmse_exact:.3e}")
        # same Philox streams: only diverging walks separate the two
        assert rmse_oracle < 0.05 * rmse_exact


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
