"""Screened Poisson (sigma > 0, f = 0): the GPU walks replay the oracle's
(same Philox streams; FP32 Bessel approximations against FP64 series), the
screened gather matches the oracle's on an identical cache, and whole
solves lie within 3 standard errors of the exact solution
u = exp(alpha x_last) cos(beta x_0), sigma = alpha^2 - beta^2."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import oracle_bvc

pytestmark = pytest.mark.gpu

EXP_COS = 5
ALPHA, BETA = 2.0, 1.0
SIGMA = ALPHA ** 2 - BETA ** 2
G = [(EXP_COS, [1.0, ALPHA, BETA])]


def _exact(pts):
    p = np.asarray(pts, dtype=np.float64)
    return np.exp(ALPHA * p[:, -1]) * np.cos(BETA * p[:, 0])


def _mesh(dim):
    if dim == 2:
        V, F = wl.circle_polygon(256)
        return V, F
    V, F = wl.icosphere(3)
    return V.astype(np.float32), F


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_walks_replay_oracle(dim):
    V, F = _mesh(dim)
    geom = bvc.Geometry(V, F)
    rng = np.random.default_rng(dim)
    d = rng.standard_normal((200, dim))
    pts = (d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0, 0.85, (200, 1))).astype(np.float32)
    W, eps = 32, 1e-3
    st = bvc.EvalState(bvc.soa(pts))
    bvc.wos_estimate(geom, G, [], st, W, eps, 1 << 14, seed=5, sigma=SIGMA)
    ug, gg = bvc.get_solution(st)
    torch.cuda.synchronize()
    o = oracle.walks(oracle.BVH(V, F), G, [], pts, W, eps, 1 << 14, 5, 0, oracle.TAG_POINTWISE, sigma=SIGMA)
    uo = o["U"].reshape(-1, W).mean(1)
    rng_u = np.abs(o["U"]).max()
    agree = np.abs(ug.cpu().numpy() - uo) <= 1e-4 * rng_u
    print(f"[screened walks {dim}D] agree={agree.mean():.3f} RMSE_vs_oracle={np.sqrt(np.mean((ug.cpu().numpy() - uo) ** 2)):.3e}")
    assert agree.mean() >= 0.97


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_gather_matches_oracle(dim):
    rng = np.random.default_rng(10 + dim)
    N, M = 3000, 700
    z = rng.standard_normal((N, dim))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    n = z.copy()
    z = (z * 0.99).astype(np.float32)
    n = n.astype(np.float32)
    uh, qh = rng.standard_normal(N), rng.standard_normal(N)
    pts = (rng.uniform(-0.6, 0.6, (M, dim))).astype(np.float32)
    cache = bvc.Cache(dim, N)
    cache.z.copy_(torch.tensor(z.T.copy()))
    cache.nrm.copy_(torch.tensor(n.T.copy()))
    cache.u_hat.copy_(torch.tensor(uh))
    cache.dudn_hat.copy_(torch.tensor(qh))
    meas = 2 * np.pi if dim == 2 else 4 * np.pi
    cache.struct.bnd_measure = meas
    cache.struct.sigma = SIGMA
    bvc.cache_pack(cache)
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(cache, st)
    u, g = bvc.get_solution(st)
    torch.cuda.synchronize()
    ub, _, gb, _, ab = oracle.gather(z.astype(np.float64), n.astype(np.float64), uh, qh, meas,
                                     pts.astype(np.float64), want_abs=True, sigma=SIGMA)
    err_u = np.abs(u.cpu().numpy() - ub / N) / np.maximum(np.abs(ub / N), ab[:, 0] / N)
    err_g = np.abs(g.cpu().numpy().T - gb / N) / np.maximum(np.abs(gb / N), ab[:, 1:1 + dim] / N)
    print(f"[screened gather {dim}D] max rel u {err_u.max():.2e} grad {err_g.max():.2e}")
    assert err_u.max() < 1e-5 and err_g.max() < 1e-5


@pytest.mark.parametrize("dim", [2, 3])
def test_screened_solve_closed_form_and_oracle(dim):
    V, F = _mesh(dim)
    geom = bvc.Geometry(V, F)
    rng = np.random.default_rng(20 + dim)
    d = rng.standard_normal((300, dim))
    pts = (d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0, 0.8, (300, 1))).astype(np.float32)
    # offsets small enough that the l = 5 eps offset bias (Sec. 3.2) stays below the standard error
    N, W, l, eps = 2048, 32, 1e-3 if dim == 2 else 2e-3, 2e-4 if dim == 2 else 4e-4
    us = []
    for s in range(8):
        opts = bvc.cache_opts(N, W, l, eps, s, sigma=SIGMA)
        cache = bvc.cache_build(geom, G, [], opts, bvc.Cache(dim, N))
        st = bvc.EvalState(bvc.soa(pts))
        bvc.evaluate(cache, st)
        us.append(bvc.get_solution(st)[0].cpu().numpy())
    us = np.array(us)
    exact = _exact(pts)
    z = (us.mean(0) - exact) / (us.std(0, ddof=1) / np.sqrt(len(us)))
    uo, _ = oracle_bvc(V, F, G, [], N, W, l, eps, pts, 0, sigma=SIGMA)
    rmse_o = np.sqrt(np.mean((us[0] - uo) ** 2))
    rmse_e = np.sqrt(np.mean((us[0] - exact) ** 2))
    print(f"[screened solve {dim}D] within3SE={np.mean(np.abs(z) < 3):.3f} rmsZ={np.sqrt(np.mean(z * z)):.2f} "
          f"RMSE_vs_exact={rmse_e:.3e} RMSE_vs_oracle={rmse_o:.3e}")
    assert np.mean(np.abs(z) < 3) >= 0.93 and np.sqrt(np.mean(z * z)) < 1.5
    assert rmse_o < 0.1 * rmse_e


def test_screened_rejects_sources():
    V, F = _mesh(2)
    geom = bvc.Geometry(V, F)
    opts = bvc.cache_opts(64, 2, 1e-3, 2e-4, 0, sigma=SIGMA)
    with pytest.raises(RuntimeError):
        bvc.cache_build(geom, G, [(wl.POLY, [1.0])], opts, bvc.Cache(2, 64))
