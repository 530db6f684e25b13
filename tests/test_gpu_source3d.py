"""3D source samples (K4 in 3D): candidates on the jittered grid kept by the
generalized winding number.  Positions are bit-exact against the oracle's
(same Philox draws, same FP64 rounding); the keep decisions agree except
where the oracle's FP64 winding number lies within 1e-3 of the threshold
(the GPU sums solid angles in FP32).  End to end, a 3D Poisson problem with
a closed-form solution lies within 3 standard errors, and the source
amplitudes' adjoint matches central differences."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import oracle_bvc

pytestmark = pytest.mark.gpu

QUAD6 = [0, 0, 0, 0, 1 / 6, 0, 0, 1 / 6, 0, 1 / 6]  # |x|^2 / 6 in the POLY order


def _gpu_sources(V, F, grid, seed, f):
    geom = bvc.Geometry(V, F)
    ncand = grid[0] * grid[1] * grid[2]
    cache = bvc.Cache(3, 1, n_src_cand=ncand)
    bvc.sample_source(geom, f, grid, seed, cache)
    torch.cuda.synchronize()
    k = int(cache.n_src_dev.item())
    return cache.src_y[:, :k].cpu().numpy().T, cache.src_c[:k].cpu().numpy(), ncand


@pytest.mark.parametrize("mesh", ["sphere", "box_obstacles"])
def test_candidates_and_weights_match_oracle(mesh):
    if mesh == "sphere":
        V, F = wl.icosphere(3)
        V = V.astype(np.float32)
    else:
        V, F = wl.box_with_obstacles(n_box=4, ellipsoids=[((-0.5, 0, 0), (0.6, 0.5, 0.5)),
                                                          ((0.2, 0.1, 0), (0.5, 0.5, 0.4))], subdiv=3)
    grid = (20, 18, 16)
    f = [(wl.GAUSS, [0.3, 2.0, 0.1, 0.0, 0.2])]
    yg, cg, ncand = _gpu_sources(V, F, grid, 5, f)
    yo, co, _, wn = oracle.sample_source3d(V, F, grid, 5, f, want_winding=True)
    amb = np.abs(wn - 0.5) < 1e-3
    print(f"[source3d {mesh}] candidates={ncand} kept gpu={len(yg)} oracle={len(yo)} ambiguous={amb.sum()}")
    if amb.sum() == 0:
        assert np.array_equal(yg, yo)
        assert np.allclose(cg, co, rtol=2e-6, atol=1e-7 * np.abs(co).max())
    else:
        assert abs(len(yg) - len(yo)) <= amb.sum()
    # overlapping obstacles: the overlap has winding number -1 and is excluded
    if mesh == "box_obstacles":
        assert set(np.round(wn[np.abs(wn - np.round(wn)) < 1e-3]).astype(int)) <= {-1, 0, 1}


def test_poisson_3d_closed_form_and_oracle():
    V, F, _ = wl.perturbed_icosphere(3, seed=1, amp=0.0)
    geom = bvc.Geometry(V, F)
    g = [(wl.POLY, QUAD6)]
    f = [(wl.POLY, [1.0])]
    eps = 1e-3 * wl.bbox_diagonal(V)
    N, W, grid = 4096, 16, (24, 24, 24)
    pts = wl.random_points_in(("sphere", (0, 0, 0), (0.8, 0.8, 0.8)), 400, seed=2)
    ncand = grid[0] * grid[1] * grid[2]
    us = []
    for s in range(6):
        opts = bvc.cache_opts(N, W, 5 * eps, eps, s, src_grid=grid)
        cache = bvc.cache_build(geom, g, f, opts, bvc.Cache(3, N, n_src_cand=ncand))
        st = bvc.EvalState(bvc.soa(pts))
        bvc.evaluate(cache, st)
        us.append(bvc.get_solution(st)[0].cpu().numpy())
    us = np.array(us)
    exact = np.sum(pts.astype(np.float64) ** 2, 1) / 6
    z = (us.mean(0) - exact) / (us.std(0, ddof=1) / np.sqrt(len(us)))
    uo, _ = oracle_bvc(V, F, g, f, N, W, 5 * eps, eps, pts, 0, src_grid=grid)
    rmse_o = np.sqrt(np.mean((us[0] - uo) ** 2))
    rmse_e = np.sqrt(np.mean((us[0] - exact) ** 2))
    print(f"[poisson 3D] within3SE={np.mean(np.abs(z) < 3):.3f} rmsZ={np.sqrt(np.mean(z * z)):.2f} "
          f"RMSE_vs_exact={rmse_e:.3e} RMSE_vs_oracle={rmse_o:.3e}")
    assert np.mean(np.abs(z) < 3) >= 0.93
    assert rmse_o < 0.1 * rmse_e


def test_adjoint_3d_source_amplitudes_central_differences():
    V, F, _ = wl.perturbed_icosphere(3, seed=3)
    geom = bvc.Geometry(V, F)
    eps = 1e-3 * wl.bbox_diagonal(V)
    pts = wl.random_points_in(("sphere", (0, 0, 0), (0.8, 0.8, 0.8)), 300, seed=4)
    rng = np.random.default_rng(5)
    bumps = (wl.GAUSS, 0.25, rng.uniform(-0.5, 0.5, (8, 3)))
    solver = bvc.DiffSolver(geom, bvc.soa(pts), 2048, 8, 5 * eps, eps, 9, bumps=bumps, src_grid=(16, 16, 16))
    gv = torch.tensor(V[:, 0] ** 2 - V[:, 1] * V[:, 2], dtype=torch.float64, device="cuda")
    amps = torch.tensor(rng.uniform(-3, 3, 8), dtype=torch.float64, device="cuda")
    lam = torch.tensor(rng.standard_normal(300), dtype=torch.float64, device="cuda")
    a = amps.clone().requires_grad_(True)
    g = gv.clone().requires_grad_(True)
    (solver(g, a) * lam).sum().backward()
    for trial in range(2):
        d = torch.tensor(rng.standard_normal(8), dtype=torch.float64, device="cuda")
        fd = ((solver(gv, amps + 0.5 * d) - solver(gv, amps - 0.5 * d)) * lam).sum().item()
        ad = (a.grad * d).sum().item()
        print(f"[adjoint 3D source] fd={fd:.6e} adjoint={ad:.6e} rel={abs(fd - ad) / abs(fd):.2e}")
        assert abs(fd - ad) <= 2e-4 * abs(fd)
