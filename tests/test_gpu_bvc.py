"""End-to-end on the GPU: the whole cache build (K1-K4 + pack) and the
gather reproduce the oracle's pipeline on the same Philox streams and the
closed-form solution within 3 standard errors; pointwise WoS (K6) replays
the oracle per point.  The RMSE against the FP64 oracle is printed for every
result."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import oracle_bvc

pytestmark = pytest.mark.gpu


def _gpu_bvc(geom, w, seed, pts, src_grid=(0, 0)):
    n_src = src_grid[0] * src_grid[1]
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, seed, src_grid=src_grid)
    cache = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(w.dim, w.n_samples, n_src_cand=n_src))
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(cache, st)
    u, grad = bvc.get_solution(st)
    torch.cuda.synchronize()
    return u.cpu().numpy(), grad.cpu().numpy().T


def test_circle_end_to_end_vs_closed_form_and_oracle():
    w = wl.circle_laplace()
    geom = bvc.Geometry(w.V, w.F)
    pts = w.eval_pts
    us, gs = [], []
    for s in range(8):
        u, g = _gpu_bvc(geom, w, s, pts)
        us.append(u)
        gs.append(g)
    us, gs = np.array(us), np.array(gs)
    exact, gexact = wl.eval_terms(w.exact, 2, pts.astype(np.float64))
    se = us.std(0, ddof=1) / np.sqrt(8)
    z = (us.mean(0) - exact) / se
    frac3 = np.mean(np.abs(z) < 3)
    rmse_exact = np.sqrt(np.mean((us[0] - exact) ** 2))
    uo, go = oracle_bvc(w.V, w.F, w.g, w.f, w.n_samples, w.walks, w.offset_l, w.eps, pts, 0)
    rmse_oracle = np.sqrt(np.mean((us[0] - uo) ** 2))
    grmse_oracle = np.sqrt(np.mean((gs[0] - go) ** 2))
    print(f"[e2e circle] M={pts.shape[0]} within3SE={frac3:.3f} rmsZ={np.sqrt(np.mean(z * z)):.3f} "
          f"RMSE_vs_exact={rmse_exact:.3e} RMSE_vs_oracle={rmse_oracle:.3e} gradRMSE_vs_oracle={grmse_oracle:.3e}")
    assert frac3 >= 0.95
    assert np.sqrt(np.mean(z * z)) < 1.5
    # same streams: the GPU and the oracle differ only through diverging walks
    assert rmse_oracle < 0.05 * rmse_exact


def test_star_poisson_manufactured_small_vs_closed_form():
    w = wl.star_poisson(n_samples=8192, walks=32, grid=48, n_seg=4000, src_grid=(96, 96), manufactured=True)
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = w.eval_pts[~near]
    us = np.array([_gpu_bvc(geom, w, s, pts, w.src_grid)[0] for s in range(6)])
    exact, _ = wl.eval_terms(w.exact, 2, pts.astype(np.float64))
    se = us.std(0, ddof=1) / np.sqrt(us.shape[0])
    z = (us.mean(0) - exact) / se
    uo, _ = oracle_bvc(w.V, w.F, w.g, w.f, w.n_samples, w.walks, w.offset_l, w.eps, pts, 0, src_grid=w.src_grid)
    rmse_oracle = np.sqrt(np.mean((us[0] - uo) ** 2))
    rmse_exact = np.sqrt(np.mean((us[0] - exact) ** 2))
    print(f"[e2e star manufactured] M={pts.shape[0]} within3SE={np.mean(np.abs(z) < 3):.3f} "
          f"RMSE_vs_exact={rmse_exact:.3e} RMSE_vs_oracle={rmse_oracle:.3e}")
    assert np.mean(np.abs(z) < 3) >= 0.93
    assert rmse_oracle < 0.1 * rmse_exact


def test_wos_estimate_replays_oracle():
    w = wl.star_poisson(n_samples=16, walks=4, grid=24, n_seg=4000, manufactured=True)
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = w.eval_pts[~near][:257]
    W = 64
    st = bvc.EvalState(bvc.soa(pts))
    bvc.wos_estimate(geom, w.g, w.f, st, W, w.eps, 1 << 14, seed=4)
    ug, gg = bvc.get_solution(st)
    torch.cuda.synchronize()
    assert st.counts.cpu().tolist() == [W, 0]
    o = oracle.walks(oracle.BVH(w.V, w.F), w.g, w.f, pts, W, w.eps, 1 << 14, 4, 0, oracle.TAG_POINTWISE)
    uo = o["U"].reshape(-1, W).mean(1)
    go = o["grad"].reshape(-1, W, 2).mean(1)
    ug = ug.cpu().numpy()
    rng_u = np.abs(o["U"]).max()
    agree = np.abs(ug - uo) <= 1e-4 * rng_u
    exact, _ = wl.eval_terms(w.exact, 2, pts.astype(np.float64))
    print(f"[wos pointwise] points={pts.shape[0]} agree={agree.mean():.3f} "
          f"RMSE_vs_oracle={np.sqrt(np.mean((ug - uo) ** 2)):.3e} RMSE_vs_exact={np.sqrt(np.mean((ug - exact) ** 2)):.3e} "
          f"gradRMSE_vs_oracle={np.sqrt(np.mean((gg.cpu().numpy().T - go) ** 2)):.3e}")
    assert agree.mean() >= 0.97
    # progressive: a second call with the next id range refines the same sums
    bvc.wos_estimate(geom, w.g, w.f, st, W, w.eps, 1 << 14, seed=4, id_base=pts.shape[0] * W)
    u2, _ = bvc.get_solution(st)
    torch.cuda.synchronize()
    assert st.counts.cpu().tolist() == [2 * W, 0]
    o2 = oracle.walks(oracle.BVH(w.V, w.F), w.g, w.f, pts, W, w.eps, 1 << 14, 4, pts.shape[0] * W,
                      oracle.TAG_POINTWISE)
    u2o = (o["U"].reshape(-1, W).sum(1) + o2["U"].reshape(-1, W).sum(1)) / (2 * W)
    assert np.mean(np.abs(u2.cpu().numpy() - u2o) <= 1e-4 * rng_u) >= 0.97


def test_profiler_counts_library_launches():
    w = wl.circle_laplace(n_samples=256, walks=8)
    geom = bvc.Geometry(w.V, w.F)
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, seed=1)
    cache = bvc.Cache(2, w.n_samples)
    st = bvc.EvalState(bvc.soa(w.eval_pts))
    bvc.profile_begin()
    bvc.cache_build(geom, w.g, w.f, opts, cache)
    bvc.evaluate(cache, st)
    bvc.get_solution(st)
    prof = bvc.profile_end()
    for k in ("sample_boundary", "walk", "reduce_walks", "pack_boundary", "gather_boundary", "get_solution"):
        assert prof[k][0] >= 1 and prof[k][1] > 0.0, (k, prof)


def test_counting_mode_gives_same_walks():
    w = wl.circle_laplace(n_samples=256, walks=8)
    geom = bvc.Geometry(w.V, w.F)
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, seed=1)
    a = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(2, w.n_samples))
    geom.stats(reset=True)
    geom.set_counting(True)
    b = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(2, w.n_samples))
    s = geom.stats(reset=True)
    geom.set_counting(False)
    assert torch.equal(a.u_hat, b.u_hat) and torch.equal(a.dudn_hat, b.dudn_hat)
    assert s["nodes"] >= s["steps"] > 0 and s["prims"] >= s["steps"]
