"""Regions of interest and the clamped double-layer kernel (Sec. 3.2-3.3).

* A region cache (samples on a circle inside a star domain, walks in the
  domain) matches the oracle's composition of the same steps and the exact
  harmonic solution inside the region.
* The clamped gather matches the oracle's clamped gather on an identical
  cache.
* The direction-sampled remainder matches the oracle's (same Philox
  directions and walk ids).
* Near the boundary the clamped estimate alone is biased; clamped plus the
  remainder lies within 3 standard errors of the exact solution.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

G3 = [(wl.POLY, [0, 0, 0, 0, 0, 0, 1, 0, -3, 0])]  # x^3 - 3 x y^2


def _exact(p):
    p = np.asarray(p, dtype=np.float64)
    return p[:, 0] ** 3 - 3 * p[:, 0] * p[:, 1] ** 2


def _disk(n, centre, r, seed):
    rng = np.random.default_rng(seed)
    th = rng.uniform(0, 2 * np.pi, n)
    rr = r * np.sqrt(rng.uniform(0, 1, n))
    return (np.asarray(centre)[None] + np.stack([rr * np.cos(th), rr * np.sin(th)], 1)).astype(np.float32)


def test_region_cache_matches_oracle_and_closed_form():
    Vd, Fd = wl.star_polygon(2000, seed=1)
    Vr, Fr = wl.circle_polygon(256, radius=0.4)
    Vr = (Vr + np.array([0.1, 0.05], np.float32)).astype(np.float32)
    dom, reg = bvc.Geometry(Vd, Fd), bvc.Geometry(Vr, Fr)
    pts = _disk(400, (0.1, 0.05), 0.3, 3)
    N, W, eps = 2048, 32, 1e-3
    us = []
    for s in range(8):
        opts = bvc.cache_opts(N, W, 0.0, eps, s)
        cache = bvc.cache_build_region(dom, reg, G3, [], opts, bvc.Cache(2, N))
        st = bvc.EvalState(bvc.soa(pts))
        bvc.evaluate(cache, st)
        us.append(bvc.get_solution(st)[0].cpu().numpy())
    us = np.array(us)
    exact = _exact(pts)
    z = (us.mean(0) - exact) / (us.std(0, ddof=1) / np.sqrt(len(us)))
    # oracle: samples on the region, walks in the domain
    zo, no, _, _ = oracle.sample_boundary(Vr, Fr, N, 0.0, 0)
    z32, n32 = zo.astype(np.float32), no.astype(np.float32)
    o = oracle.walks(oracle.BVH(Vd, Fd), G3, [], z32, W, eps, 1 << 14, 0, 0, oracle.TAG_WALK)
    uh, qh = oracle.reduce_walks(o["U"], o["grad"], n32, W)
    ub, _, _, _ = oracle.gather(z32, n32, uh, qh, oracle.boundary_measure(Vr, Fr), pts.astype(np.float64))
    uo = ub / N
    rmse_o = np.sqrt(np.mean((us[0] - uo) ** 2))
    rmse_e = np.sqrt(np.mean((us[0] - exact) ** 2))
    print(f"[region] within3SE={np.mean(np.abs(z) < 3):.3f} rmsZ={np.sqrt(np.mean(z * z)):.2f} "
          f"RMSE_vs_exact={rmse_e:.3e} RMSE_vs_oracle={rmse_o:.3e}")
    assert np.mean(np.abs(z) < 3) >= 0.93 and np.sqrt(np.mean(z * z)) < 1.5
    assert rmse_o < 0.1 * rmse_e


@pytest.mark.parametrize("dim", [2, 3])
def test_clamped_gather_matches_oracle(dim):
    rng = np.random.default_rng(30 + dim)
    N, M, c = 3000, 600, 0.8
    z = rng.standard_normal((N, dim))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    n = z.astype(np.float32)
    z = (0.99 * z).astype(np.float32)
    uh, qh = rng.standard_normal(N), rng.standard_normal(N)
    d = rng.standard_normal((M, dim))
    pts = (d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0.5, 0.985, (M, 1))).astype(np.float32)
    cache = bvc.Cache(dim, N)
    cache.z.copy_(torch.tensor(z.T.copy()))
    cache.nrm.copy_(torch.tensor(n.T.copy()))
    cache.u_hat.copy_(torch.tensor(uh))
    cache.dudn_hat.copy_(torch.tensor(qh))
    meas = 2 * np.pi if dim == 2 else 4 * np.pi
    cache.struct.bnd_measure = meas
    cache.struct.clamp_c = c
    bvc.cache_pack(cache)
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(cache, st)
    u, g = bvc.get_solution(st)
    torch.cuda.synchronize()
    ub, _, gb, _, ab = oracle.gather(z.astype(np.float64), n.astype(np.float64), uh, qh, meas,
                                     pts.astype(np.float64), want_abs=True, clamp_c=c)
    err = np.abs(u.cpu().numpy() - ub / N) / np.maximum(np.abs(ub / N), ab[:, 0] / N)
    errg = np.abs(g.cpu().numpy().T - gb / N) / np.maximum(np.abs(gb / N), ab[:, 1:1 + dim] / N)
    print(f"[clamped gather {dim}D] max rel u {err.max():.2e} grad {errg.max():.2e}")
    assert err.max() < 1e-5 and errg.max() < 1e-5


def test_clamp_correction_matches_oracle():
    V, F = wl.circle_polygon(512)
    geom = bvc.Geometry(V, F)
    l, c, eps = 0.01, 1.0, 2e-3
    rng = np.random.default_rng(7)
    th = rng.uniform(0, 2 * np.pi, 300)
    rr = 1.0 - l - rng.uniform(0.002, 0.04, 300)
    pts = np.stack([rr * np.cos(th), rr * np.sin(th)], 1).astype(np.float32)
    uc, nh = bvc.clamp_correction(geom, geom, l, G3, [], c, bvc.soa(pts), 64, 16, eps, seed=9)
    uc = uc.cpu().numpy()
    uo, nho = oracle.clamp_correction(oracle.BVH(V, F), G3, V, F, l, pts.astype(np.float64), c, 64, 16, eps, seed=9)
    scale = np.abs(uo).max()
    d = np.abs(uc - uo) / scale
    print(f"[clamp correction] hits gpu={nh} oracle={nho} median rel={np.median(d):.2e} "
          f"p95={np.quantile(d, 0.95):.2e} max={d.max():.2e}")
    assert abs(nh - nho) <= max(3, 0.002 * nho)
    assert np.median(d) < 1e-4 and np.quantile(d, 0.95) < 1e-2


def test_clamped_estimate_with_remainder_is_unbiased():
    # Eq. 8: clamped gather + remainder has the expectation of the unclamped
    # gather.  Per seed the same cache (same samples and walks) is gathered
    # with and without the clamp; the remainder uses fresh directions and
    # walks.  Points 0.002-0.02 beyond the offset boundary, where the
    # unclamped double layer is sampled poorly.
    w = wl.circle_laplace(n_samples=1024, walks=32)
    geom = bvc.Geometry(w.V, w.F)
    rng = np.random.default_rng(11)
    th = rng.uniform(0, 2 * np.pi, 200)
    rr = 1.0 - w.offset_l - rng.uniform(0.002, 0.02, 200)
    pts = np.stack([rr * np.cos(th), rr * np.sin(th)], 1).astype(np.float32)
    P = bvc.soa(pts)
    c = 5.0
    un, cl, co = [], [], []
    for s in range(12):
        for clamp in (0.0, c):
            opts = bvc.cache_opts(w.n_samples, w.walks, w.offset_l, w.eps, s, clamp_c=clamp)
            cache = bvc.cache_build(geom, w.g, [], opts, bvc.Cache(2, w.n_samples))
            st = bvc.EvalState(P)
            bvc.evaluate(cache, st)
            (cl if clamp else un).append(bvc.get_solution(st)[0].cpu().numpy())
        uc, _ = bvc.clamp_correction(geom, geom, w.offset_l, w.g, [], c, P, 32, 8, w.eps, seed=100 + s)
        co.append(cl[-1] + uc.cpu().numpy())
    un, cl, co = np.array(un), np.array(cl), np.array(co)

    def z_of(d):
        return d.mean(0) / (d.std(0, ddof=1) / np.sqrt(len(d)) + 1e-300)

    zc, zk = z_of(cl - un), z_of(co - un)
    print(f"[clamp bias] clamped - unclamped: mean |diff|={np.abs((cl - un).mean(0)).mean():.3e} "
          f"rms z={np.sqrt(np.mean(zc ** 2)):.2f}; clamped + remainder - unclamped: "
          f"mean |diff|={np.abs((co - un).mean(0)).mean():.3e} rms z={np.sqrt(np.mean(zk ** 2)):.2f}; "
          f"sd unclamped={un.std(0).mean():.3e} sd clamped+remainder={co.std(0).mean():.3e}")
    assert np.sqrt(np.mean(zc ** 2)) > 3.0          # clamping alone is biased here
    assert np.mean(np.abs(zk) < 3) >= 0.93 and np.sqrt(np.mean(zk ** 2)) < 1.5
