"""Differentiation: boundary data from vertex values and Gaussian-bump
source amplitudes as parameters; gradients of L = sum_x lam(x) u(x) from the
adjoint gather and the adjoint walk replay.

With fixed seeds the estimator is linear in (g_vertex, A), so
  - the adjoint must match central differences of the GPU forward along any
    direction (up to FP32 rounding of the forward), and
  - the oracle's directional derivative along d is exactly the oracle's u
    for the parameters d (linearity), which the adjoint must match up to the
    walks whose FP32 and FP64 paths diverge.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import oracle_bvc

pytestmark = pytest.mark.gpu

GAUSS = wl.GAUSS


def _star_problem(n_seg=2000, N=2048, W=16, grid=(48, 48), seed=3):
    w = wl.star_poisson(n_samples=N, walks=W, grid=40, n_seg=n_seg, src_grid=grid)
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = w.eval_pts[~near][:600]
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-0.5, 0.5, (8, 2))
    bumps = (GAUSS, 0.08, centres)
    solver = bvc.DiffSolver(geom, bvc.soa(pts), N, W, w.offset_l, w.eps, seed, bumps=bumps, src_grid=grid)
    gv = torch.tensor(np.sin(3 * w.V[:, 0]) + w.V[:, 1] ** 2, dtype=torch.float64, device="cuda")
    amps = torch.tensor(rng.uniform(-5, 5, 8), dtype=torch.float64, device="cuda")
    lam = torch.tensor(rng.standard_normal(pts.shape[0]), dtype=torch.float64, device="cuda")
    return w, geom, pts, solver, gv, amps, lam, bumps


def _grads(solver, gv, amps, lam):
    g = gv.clone().requires_grad_(True)
    a = amps.clone().requires_grad_(True)
    u = solver(g, a)
    (u * lam).sum().backward()
    return g.grad.clone(), a.grad.clone(), u.detach()


def test_vertex_data_forward_matches_closed_form_affine_g():
    w = wl.circle_laplace(n_samples=1024, walks=16)
    geom = bvc.Geometry(w.V, w.F)
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, 2)
    gterm = [(wl.POLY, [0.5, 0.3, -1.2])]
    a = bvc.cache_build(geom, gterm, [], opts, bvc.Cache(2, w.n_samples))
    gv = torch.tensor(0.5 + 0.3 * w.V[:, 0] - 1.2 * w.V[:, 1], dtype=torch.float32, device="cuda")
    b = bvc.cache_build_vg(geom, gv, [], opts, bvc.Cache(2, w.n_samples))
    torch.cuda.synchronize()
    du = (a.u_hat - b.u_hat).abs().max().item()
    dq = (a.dudn_hat - b.dudn_hat).abs().max().item()
    print(f"[vertex g] max|du^|={du:.2e} max|dq^|={dq:.2e}")
    assert du < 1e-5 and dq < 1e-5 * a.dudn_hat.abs().max().item() * 50


def test_adjoint_matches_central_differences():
    w, geom, pts, solver, gv, amps, lam, bumps = _star_problem()
    ggv, gam, u0 = _grads(solver, gv, amps, lam)
    rng = np.random.default_rng(11)
    checks = []
    for kind in ("gv", "gv", "amp", "amp", "vertex"):
        d_gv = torch.zeros_like(gv)
        d_a = torch.zeros_like(amps)
        if kind == "gv":
            d_gv = torch.tensor(rng.standard_normal(gv.numel()), dtype=torch.float64, device="cuda")
        elif kind == "amp":
            d_a = torch.tensor(rng.standard_normal(8), dtype=torch.float64, device="cuda")
        else:
            d_gv[int(torch.argmax(ggv.abs()))] = 1.0
        h = 0.5
        up = solver(gv + h * d_gv, amps + h * d_a)
        um = solver(gv - h * d_gv, amps - h * d_a)
        fd = ((up - um) * lam).sum().item() / (2 * h)
        ad = (ggv * d_gv).sum().item() + (gam * d_a).sum().item()
        checks.append((kind, fd, ad))
        print(f"[adjoint vs FD] {kind}: fd={fd:.6e} adjoint={ad:.6e} rel={abs(fd - ad) / max(abs(fd), 1e-30):.2e}")
    for kind, fd, ad in checks:
        assert abs(fd - ad) <= 2e-4 * max(abs(fd), 1e-3), (kind, fd, ad)


def test_adjoint_matches_oracle_gradient():
    w, geom, pts, solver, gv, amps, lam, bumps = _star_problem(n_seg=1500, N=1024, W=8, grid=(32, 32))
    ggv, gam, _ = _grads(solver, gv, amps, lam)
    lam_h = lam.cpu().numpy()
    rng = np.random.default_rng(12)
    kind_, sigma, centres = bumps
    for trial in range(3):
        d_gv = rng.standard_normal(gv.numel()) if trial != 1 else np.zeros(gv.numel())
        d_a = rng.standard_normal(8) if trial != 0 else np.zeros(8)
        f = bvc.bump_terms(kind_, sigma, centres, d_a)
        # the oracle solve with parameters d is its directional derivative
        uo, _ = oracle_bvc(w.V, w.F, [], f, w.n_samples, w.walks, w.offset_l, w.eps, pts, 3,
                           src_grid=(32, 32), g_vertex=d_gv)
        ref = float(np.dot(lam_h, uo))
        ad = float(np.dot(ggv.cpu().numpy(), d_gv) + np.dot(gam.cpu().numpy(), d_a))
        scale = float(np.dot(np.abs(lam_h), np.abs(uo)))
        print(f"[adjoint vs oracle] trial={trial}: oracle={ref:.6e} adjoint={ad:.6e} "
              f"rel={abs(ref - ad) / max(abs(ref), 1e-30):.2e} (vs sum|terms| {abs(ref - ad) / scale:.2e})")
        assert abs(ref - ad) <= 2e-3 * scale


def test_adjoint_3d_laplace_central_differences():
    V, F, _ = wl.perturbed_icosphere(3, seed=4)
    geom = bvc.Geometry(V, F)
    eps = 1e-3 * wl.bbox_diagonal(V)
    pts = wl.random_points_in(("sphere", (0, 0, 0), (0.85, 0.85, 0.85)), 500, seed=5)
    solver = bvc.DiffSolver(geom, bvc.soa(pts), 2048, 8, 5 * eps, eps, 7)
    gv = torch.tensor(np.exp(0.5 * V[:, 2]) * np.cos(0.3 * V[:, 0]), dtype=torch.float64, device="cuda")
    lam = torch.tensor(np.random.default_rng(1).standard_normal(500), dtype=torch.float64, device="cuda")
    g = gv.clone().requires_grad_(True)
    u = solver(g)
    (u * lam).sum().backward()
    d = torch.tensor(np.random.default_rng(2).standard_normal(gv.numel()), dtype=torch.float64, device="cuda")
    fd = ((solver(gv + 0.5 * d) - solver(gv - 0.5 * d)) * lam).sum().item()
    ad = (g.grad * d).sum().item()
    print(f"[adjoint 3D] fd={fd:.6e} adjoint={ad:.6e} rel={abs(fd - ad) / abs(fd):.2e}")
    assert abs(fd - ad) <= 2e-4 * abs(fd)


def test_adjoint_rejects_non_bump_sources():
    w = wl.circle_laplace(n_samples=64, walks=2)
    geom = bvc.Geometry(w.V, w.F)
    opts = bvc.cache_opts(64, 2, w.offset_l, w.eps, 0)
    cache = bvc.Cache(2, 64)
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    gg = torch.zeros(w.V.shape[0], dtype=torch.float64, device="cuda")
    ga = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        bvc.cache_adjoint(geom, [(wl.POLY, [1.0])], opts, cache, z, z, None, gg, ga)


def test_source_reuse_equals_fresh_build():
    w = wl.star_poisson(n_samples=512, walks=4, grid=16, n_seg=2000, src_grid=(40, 40))
    geom = bvc.Geometry(w.V, w.F)
    opts = bvc.cache_opts(512, 4, w.offset_l, w.eps, 3, src_grid=(40, 40))
    a = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(2, 512, n_src_cand=1600))
    f2 = [(wl.GAUSS, [0.08, 2.0, 0.1, 0.2, -1.0, -0.3, 0.1])]
    fresh = bvc.cache_build(geom, w.g, f2, opts, bvc.Cache(2, 512, n_src_cand=1600))
    reuse = bvc.Cache(2, 512, n_src_cand=1600)
    reuse.src_y.copy_(a.src_y)
    reuse.n_src_dev.copy_(a.n_src_dev)
    opts.reuse_sources = 1
    bvc.cache_build(geom, w.g, f2, opts, reuse)
    torch.cuda.synchronize()
    k = int(fresh.n_src_dev.item())
    assert torch.equal(reuse.src_c[:k], fresh.src_c[:k]) and torch.equal(reuse.src_packed, fresh.src_packed)
    assert torch.equal(reuse.u_hat, fresh.u_hat)
