"""End-to-end on the GPU: the whole cache build (K1-K4 + pack) and the
gather reproduce the oracle's pipeline on the same Philox streams (point by
point, within what the samples' diverging walks and the gather's FP32
tolerance allow); pointwise WoS (K6) replays the oracle per point.  The RMSE
against the FP64 oracle is printed for every result; the closed-form checks
are in test_gpu_closed_form.py."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import oracle_cache, oracle_evaluate

pytestmark = pytest.mark.gpu


def _solve_vs_oracle(w, geom, pts, seed, src_grid=(0, 0)):
    """One GPU solve and the oracle's pipeline on the same Philox streams.

    The two caches differ only where walks diverge (FP32 against FP64 paths),
    so at every point the difference of the solutions is bounded by the
    triangle inequality over the samples' differences,
        |u_gpu - u_oracle| <= sum_i (|dG/dn| |du^_i| + |G| |ddu/dn^_i|) / (p N)
                              + sum_j |G| |dc_j| / M + 1e-5 sum |terms|,
    the last part being the gather's own FP32 tolerance."""
    n_src = src_grid[0] * src_grid[1]
    opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, seed, src_grid=src_grid)
    cache = bvc.cache_build(geom, w.g, w.f, opts, bvc.Cache(w.dim, w.n_samples, n_src_cand=n_src))
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(cache, st)
    u, grad = bvc.get_solution(st)
    torch.cuda.synchronize()
    u = u.cpu().numpy()
    c = oracle_cache(w.V, w.F, w.g, w.f, w.n_samples, w.walks, w.offset_l, w.eps, seed,
                     src_grid=src_grid if n_src else None)
    uo, go = oracle_evaluate(c, pts.astype(np.float64))
    du = np.abs(cache.u_hat.cpu().numpy() - c["u_hat"])
    dq = np.abs(cache.dudn_hat.cpu().numpy() - c["q_hat"])
    z, n = c["z"], c["n"]
    _, _, _, _, ab_u = oracle.gather(z, n, du, np.zeros_like(du), c["measure"], pts, want_abs=True, jac=c["jac"])
    _, _, _, _, ab_q = oracle.gather(z, n, np.zeros_like(dq), dq, c["measure"], pts, want_abs=True, jac=c["jac"])
    _, _, _, _, ab = oracle.gather(z, n, c["u_hat"], c["q_hat"], c["measure"], pts, c["y"], c["c"], want_abs=True,
                                   jac=c["jac"])
    bound = (ab_u[:, 0] + ab_q[:, 0]) / w.n_samples + 1e-5 * ab[:, 0] / w.n_samples
    if c["n_src"]:
        k = c["y"].shape[0]
        assert int(cache.n_src_dev.item()) == k
        dc = np.abs(cache.src_c[:k].cpu().numpy() - c["c"])
        _, _, _, _, ab_c = oracle.gather(np.zeros((0, w.dim)), np.zeros((0, w.dim)), np.zeros(0), np.zeros(0), 1.0,
                                         pts, c["y"], dc, want_abs=True)
        bound += ab_c[:, 1 + w.dim] / c["n_src"] + 1e-5 * ab[:, 1 + w.dim] / c["n_src"]
    return u, uo, bound, du, dq


def test_circle_whole_solve_vs_oracle():
    w = wl.circle_laplace()
    geom = bvc.Geometry(w.V, w.F)
    pts = w.eval_pts
    u, uo, bound, du, dq = _solve_vs_oracle(w, geom, pts, 0)
    exact, _ = wl.eval_terms(w.exact, 2, pts.astype(np.float64))
    print(f"[e2e circle] M={pts.shape[0]} RMSE_vs_exact={np.sqrt(np.mean((u - exact) ** 2)):.3e} "
          f"RMSE_vs_oracle={np.sqrt(np.mean((u - uo) ** 2)):.3e} samples differing: u^ {np.mean(du > 1e-6):.4f} "
          f"du/dn^ {np.mean(dq > 1e-6):.4f}")
    # element-wise: every point's difference is explained by the samples'
    # differences (diverging walks) and the gather's FP32 tolerance
    assert np.all(np.abs(u - uo) <= bound), np.max(np.abs(u - uo) / bound)


def test_star_manufactured_small_vs_oracle():
    w = wl.star_poisson(n_samples=8192, walks=32, grid=48, n_seg=4000, src_grid=(96, 96), manufactured=True)
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = w.eval_pts[~near]
    u, uo, bound, du, dq = _solve_vs_oracle(w, geom, pts, 0, w.src_grid)
    exact, _ = wl.eval_terms(w.exact, 2, pts.astype(np.float64))
    print(f"[e2e star manufactured] M={pts.shape[0]} RMSE_vs_exact={np.sqrt(np.mean((u - exact) ** 2)):.3e} "
          f"RMSE_vs_oracle={np.sqrt(np.mean((u - uo) ** 2)):.3e} samples differing: u^ {np.mean(du > 1e-6):.4f} "
          f"du/dn^ {np.mean(dq > 1e-6):.4f}")
    assert np.all(np.abs(u - uo) <= bound), np.max(np.abs(u - uo) / bound)


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


def test_star_reference_spot_checked_by_the_oracle():
    """The literal 2D Poisson configuration has no closed form; its RMSE
    reference (bench.py) is high-count pointwise walk on spheres on the GPU.
    On 256 of the reference's points the oracle's FP64 walks (other Philox
    streams) agree with the GPU's within 4 combined standard errors."""
    w = wl.star_poisson(grid=64)
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = w.eval_pts[~near][::max(1, int((~near).sum()) // 256)][:256]
    Wg, Wo = 1 << 16, 1 << 11
    st = bvc.EvalState(bvc.soa(pts), grad=False)
    ws = bvc.workspace(bvc.wos_workspace_size(2, st.m, 4096)[1])
    s1, s2 = np.zeros(st.m), np.zeros(st.m)
    for c in range(Wg // 4096):
        bvc.eval_state_reset(st)
        bvc.wos_estimate(geom, w.g, w.f, st, 4096, w.eps, 1 << 14, 777, c * st.m * 4096, ws)
        u, _ = bvc.get_solution(st)
        torch.cuda.synchronize()
        u = u.cpu().numpy()
        s1 += u
        s2 += u * u
    k = Wg // 4096
    ref = s1 / k
    se_g = np.sqrt(np.maximum(s2 / k - ref ** 2, 0.0) / k)
    o = oracle.walks(oracle.BVH(w.V, w.F), w.g, w.f, pts, Wo, w.eps, 1 << 14, 31, 0, oracle.TAG_POINTWISE)
    U = o["U"].reshape(-1, Wo)
    uo, se_o = U.mean(1), U.std(1, ddof=1) / np.sqrt(Wo)
    z = (ref - uo) / np.sqrt(se_g ** 2 + se_o ** 2)
    print(f"[star reference] points={st.m} GPU {Wg} walks (SE rms {np.sqrt(np.mean(se_g ** 2)):.2e}) vs oracle "
          f"{Wo} walks (SE rms {np.sqrt(np.mean(se_o ** 2)):.2e}): rms z {np.sqrt(np.mean(z * z)):.2f}, "
          f"max |z| {np.abs(z).max():.2f}")
    assert np.mean(np.abs(z) < 4) >= 0.99 and np.sqrt(np.mean(z * z)) < 1.3
