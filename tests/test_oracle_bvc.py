"""End-to-end pins for the oracle's BVC estimator (Alg. 1, Eq. 3-6).

* unbiasedness via linearity (the paper's "Bias" paragraph): at tiny cache
  sizes the mean over many independent caches converges to the closed form;
* the circle configuration (256-gon, g = Re z^3, 1024 samples x 64 walks,
  l = 1e-3, eps = l/5): replicate caches put the closed form within 3 SE;
* Poisson with a source cache on a disk: u = |x|^2/4, f = 1;
* global error falls with more boundary samples (Fig. "GlobalError").
"""
import numpy as np

import oracle
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import oracle_bvc

RE_Z3 = [(wl.POLY, wl.poly2d_coeffs({(3, 0): 1.0, (1, 2): -3.0}))]


def _replicas(V, F, g, f, N, W, l, eps, pts, seeds, src_grid=None):
    bvh = oracle.BVH(V, F)
    us, gs = [], []
    for s in seeds:
        u, gr = oracle_bvc(V, F, g, f, N, W, l, eps, pts, s, src_grid, bvh=bvh)
        us.append(u)
        gs.append(gr)
    return np.array(us), np.array(gs)


def test_unbiased_with_tiny_caches():
    V, F = wl.circle_polygon(256)
    pts = np.array([[0.0, 0.0], [0.3, -0.2], [-0.5, 0.4]])
    R = 600
    us, gs = _replicas(V, F, RE_Z3, [], 4, 4, 2e-2, 4e-3, pts, range(1000, 1000 + R))
    exact, gexact = wl.eval_terms(RE_Z3, 2, pts)
    se = us.std(0) / np.sqrt(R)
    # bias allowance: eps-shell and the offset polygon's gaps at vertices
    assert np.all(np.abs(us.mean(0) - exact) < 3.5 * se + 0.02), (us.mean(0), exact, se)
    gse = gs.std(0) / np.sqrt(R)
    assert np.all(np.abs(gs.mean(0) - gexact) < 3.5 * gse + 0.05)


def test_circle_configuration_within_3_se():
    w = wl.circle_laplace()
    rng = np.random.default_rng(0)
    pts = w.eval_pts[rng.choice(w.eval_pts.shape[0], 120, replace=False)].astype(np.float64)
    us, gs = _replicas(w.V, w.F, w.g, w.f, w.n_samples, w.walks, w.offset_l, w.eps, pts, range(8))
    exact, gexact = wl.eval_terms(w.exact, 2, pts)
    se = us.std(0, ddof=1) / np.sqrt(us.shape[0])
    z = (us.mean(0) - exact) / se
    assert np.mean(np.abs(z) < 3.0) >= 0.95
    assert np.sqrt(np.mean(z * z)) < 1.5
    gse = gs.std(0, ddof=1) / np.sqrt(gs.shape[0])
    gz = (gs.mean(0) - gexact) / gse
    assert np.mean(np.abs(gz) < 3.0) >= 0.95


def test_poisson_disk_with_source_cache():
    V, F = wl.circle_polygon(256)
    g = [(wl.POLY, wl.poly2d_coeffs({(2, 0): 0.25, (0, 2): 0.25}))]
    f = [(wl.POLY, [1.0])]
    pts = np.array([[0.0, 0.0], [0.3, -0.2], [-0.5, 0.4], [0.1, 0.7]])
    us, gs = _replicas(V, F, g, f, 512, 32, 1e-2, 2e-3, pts, range(6), src_grid=(64, 64))
    exact, gexact = wl.eval_terms(g, 2, pts)
    se = us.std(0, ddof=1) / np.sqrt(us.shape[0])
    assert np.all(np.abs(us.mean(0) - exact) < 4 * se + 5e-3), (us.mean(0), exact, se)


def test_error_falls_with_cache_size():
    V, F = wl.circle_polygon(256)
    pts = wl.grid_points((-0.8, -0.8), (0.8, 0.8), 8)
    pts = pts[np.sum(pts * pts, 1) < 0.8]
    exact, _ = wl.eval_terms(RE_Z3, 2, pts)
    bvh = oracle.BVH(V, F)
    rmse = []
    for N in (64, 1024):
        errs = []
        for s in range(4):
            u, _ = oracle_bvc(V, F, RE_Z3, [], N, 16, 1e-2, 2e-3, pts, 50 + s, bvh=bvh)
            errs.append(np.mean((u - exact) ** 2))
        rmse.append(np.sqrt(np.mean(errs)))
    ratio = rmse[0] / rmse[1]
    assert 2.0 < ratio < 8.0, rmse
