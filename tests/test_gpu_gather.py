"""GPU parity for the gather (K5, Eq. 3-6) given an identical cache: relative
error |delta| / max(|ref|, sum |terms|) <= 1e-5, with FP32 pair terms and
FP64 accumulation; plus progressive accumulation (Alg. 1 running sums) and
GetSolution."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl
from tests.oracle_pipeline import oracle_cache

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _gpu_cache_from(c, dim, measure):
    """Device cache holding exactly the oracle's z, n, jac, u^, du/dn^ (and sources)."""
    N = c["z"].shape[0]
    ncand = c["n_src"]
    cache = bvc.Cache(dim, N, n_src_cand=ncand)
    cache.z.copy_(torch.from_numpy(np.ascontiguousarray(c["z"].T)))
    cache.nrm.copy_(torch.from_numpy(np.ascontiguousarray(c["n"].T)))
    cache.jac.copy_(torch.from_numpy(c["jac"].astype(np.float32)))
    cache.u_hat.copy_(torch.from_numpy(c["u_hat"]))
    cache.dudn_hat.copy_(torch.from_numpy(c["q_hat"]))
    if ncand:
        k = c["y"].shape[0]
        cache.src_y[:, :k].copy_(torch.from_numpy(np.ascontiguousarray(c["y"].T)))
        cache.src_c[:k].copy_(torch.from_numpy(c["c"]))
        cache.n_src_dev.fill_(k)
    cache.set_measure(measure)
    bvc.cache_pack(cache)
    return cache


def _compare(cache, c, pts, dim, label):
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(cache, st)
    torch.cuda.synchronize()
    ub, us, gb, gs, ab = oracle.gather(c["z"], c["n"], c["u_hat"], c["q_hat"], c["measure"], pts, c["y"], c["c"],
                                       want_abs=True, jac=c["jac"])
    errs = {}
    errs["u_bnd"] = np.abs(st.u_bnd.cpu().numpy() - ub) / np.maximum(np.abs(ub), ab[:, 0])
    errs["g_bnd"] = np.abs(st.grad_bnd.cpu().numpy().T - gb) / np.maximum(np.abs(gb), ab[:, 1:1 + dim])
    if c["n_src"]:
        errs["u_src"] = np.abs(st.u_src.cpu().numpy() - us) / np.maximum(np.abs(us), ab[:, 1 + dim])
        errs["g_src"] = np.abs(st.grad_src.cpu().numpy().T - gs) / np.maximum(np.abs(gs), ab[:, 2 + dim:])
    print(f"[gather {label}] " + " ".join(f"{k}={v.max():.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v.max() < TOL, (k, v.max())
    counts = st.counts.cpu().numpy()
    assert counts[0] == cache.n and counts[1] == cache.n_src_cand
    return st


def test_gather_circle_configuration():
    w = wl.circle_laplace()
    c = oracle_cache(w.V, w.F, w.g, w.f, w.n_samples, w.walks, w.offset_l, w.eps, seed=0)
    cache = _gpu_cache_from(c, 2, c["measure"])
    _compare(cache, c, w.eval_pts, 2, "circle N=1024 M=%d" % w.eval_pts.shape[0])


def test_gather_star_with_source_ragged():
    w = wl.star_poisson(n_samples=3000, walks=8, grid=64, n_seg=2000, src_grid=(70, 50))
    c = oracle_cache(w.V, w.F, w.g, w.f, w.n_samples, w.walks, w.offset_l, w.eps, seed=1, src_grid=w.src_grid)
    cache = _gpu_cache_from(c, 2, c["measure"])
    pts = w.eval_pts[:2501]
    _compare(cache, c, pts, 2, "star N=3000 Ms=%d M=2501" % c["y"].shape[0])


def test_gather_sphere_3d():
    V, F, _ = wl.perturbed_icosphere(4, 0)
    g = [(wl.EXP_TRIG, [1.0, 0.5, 0.3, 0.4])]
    c = oracle_cache(V, F, g, [], 3001, 4, 0.02, 0.004, seed=2)
    rng = np.random.default_rng(0)
    pts = rng.uniform(-0.6, 0.6, (2049, 3)).astype(np.float32)
    cache = _gpu_cache_from(c, 3, c["measure"])
    _compare(cache, c, pts, 3, "sphere N=3001 M=2049")


def test_gather_full_size_3d_sampled():
    # the 3D workload's sizes: 262144 cache samples, 512^2-plane + 1M points;
    # the oracle checks 48 sampled points, the GPU computes all of them.
    w = wl.icosphere_laplace()
    rng = np.random.default_rng(5)
    N = w.n_samples
    d = rng.standard_normal((N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    c = {"z": (d * 0.97).astype(np.float32), "n": d.astype(np.float32),
         "jac": rng.uniform(0.9, 1.1, N).astype(np.float32).astype(np.float64),
         "u_hat": rng.standard_normal(N), "q_hat": rng.standard_normal(N), "measure": 4 * np.pi,
         "y": None, "c": None, "n_src": 0, "N": N}
    cache = _gpu_cache_from(c, 3, c["measure"])
    st = bvc.EvalState(bvc.soa(w.eval_pts))
    bvc.evaluate(cache, st)
    torch.cuda.synchronize()
    sel = rng.choice(w.eval_pts.shape[0], 48, replace=False)
    ub, _, gb, _, ab = oracle.gather(c["z"], c["n"], c["u_hat"], c["q_hat"], c["measure"], w.eval_pts[sel],
                                     want_abs=True, jac=c["jac"])
    eu = np.abs(st.u_bnd.cpu().numpy()[sel] - ub) / np.maximum(np.abs(ub), ab[:, 0])
    eg = np.abs(st.grad_bnd.cpu().numpy().T[sel] - gb) / np.maximum(np.abs(gb), ab[:, 1:4])
    print(f"[gather full 3D] M={w.eval_pts.shape[0]} N={N} u={eu.max():.2e} g={eg.max():.2e}")
    assert eu.max() < TOL and eg.max() < TOL
    assert np.all(np.isfinite(st.u_bnd.cpu().numpy()))


def test_gather_full_size_2d_sampled():
    # the 2D configuration's sizes: 65,536 boundary samples and 33,983 kept
    # source samples against the 511,540 gathered points of the 1024^2 grid;
    # the oracle checks 48 sampled points, the GPU computes all of them
    w = wl.star_poisson()
    geom = bvc.Geometry(w.V, w.F)
    near = bvc.classify_near(geom, bvc.soa(w.eval_pts), w.offset_l).cpu().numpy().astype(bool)
    pts = w.eval_pts[~near]
    rng = np.random.default_rng(8)
    N = w.n_samples
    z, n, _, jac = oracle.sample_boundary(w.V, w.F, N, w.offset_l, 2)
    y, cw, ncand = oracle.sample_source2d(w.V, w.F, w.src_grid, 2, w.f, l=w.offset_l)
    c = {"z": z.astype(np.float32).astype(np.float64), "n": n.astype(np.float32).astype(np.float64),
         "jac": jac.astype(np.float32).astype(np.float64), "u_hat": rng.standard_normal(N),
         "q_hat": rng.standard_normal(N), "measure": oracle.boundary_measure(w.V, w.F), "y": y, "c": cw,
         "n_src": ncand, "N": N}
    cache = _gpu_cache_from(c, 2, c["measure"])
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(cache, st)
    torch.cuda.synchronize()
    sel = rng.choice(pts.shape[0], 48, replace=False)
    ub, us, gb, gs, ab = oracle.gather(c["z"], c["n"], c["u_hat"], c["q_hat"], c["measure"], pts[sel], y, cw,
                                       want_abs=True, jac=c["jac"])
    eu = np.abs(st.u_bnd.cpu().numpy()[sel] - ub) / np.maximum(np.abs(ub), ab[:, 0])
    eg = np.abs(st.grad_bnd.cpu().numpy().T[sel] - gb) / np.maximum(np.abs(gb), ab[:, 1:3])
    es = np.abs(st.u_src.cpu().numpy()[sel] - us) / np.maximum(np.abs(us), ab[:, 3])
    egs = np.abs(st.grad_src.cpu().numpy().T[sel] - gs) / np.maximum(np.abs(gs), ab[:, 4:6])
    print(f"[gather full 2D] M={pts.shape[0]} N={N} Ms={y.shape[0]} u={eu.max():.2e} g={eg.max():.2e} "
          f"u_src={es.max():.2e} g_src={egs.max():.2e}")
    assert eu.max() < TOL and eg.max() < TOL and es.max() < TOL and egs.max() < TOL


def test_progressive_accumulation_and_solution():
    w = wl.circle_laplace(n_samples=512, walks=8)
    c1 = oracle_cache(w.V, w.F, w.g, w.f, 512, 8, w.offset_l, w.eps, seed=11)
    c2 = oracle_cache(w.V, w.F, w.g, w.f, 512, 8, w.offset_l, w.eps, seed=12)
    k1 = _gpu_cache_from(c1, 2, c1["measure"])
    k2 = _gpu_cache_from(c2, 2, c2["measure"])
    pts = w.eval_pts[:700]
    st = bvc.EvalState(bvc.soa(pts))
    bvc.evaluate(k1, st)
    bvc.evaluate(k2, st)
    u, grad = bvc.get_solution(st)
    torch.cuda.synchronize()
    assert st.counts.cpu().tolist() == [1024, 0]
    ub1, _, gb1, _ = oracle.gather(c1["z"], c1["n"], c1["u_hat"], c1["q_hat"], c1["measure"], pts, jac=c1["jac"])
    ub2, _, gb2, _ = oracle.gather(c2["z"], c2["n"], c2["u_hat"], c2["q_hat"], c2["measure"], pts, jac=c2["jac"])
    ref = (ub1 + ub2) / 1024
    np.testing.assert_allclose(u.cpu().numpy(), ref, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(grad.cpu().numpy().T, (gb1 + gb2) / 1024, rtol=1e-4, atol=1e-4)


def test_empty_evaluation_set_and_empty_cache():
    w = wl.circle_laplace(n_samples=256, walks=4)
    c = oracle_cache(w.V, w.F, w.g, w.f, 256, 4, w.offset_l, w.eps, seed=1)
    cache = _gpu_cache_from(c, 2, c["measure"])
    st = bvc.EvalState(torch.zeros((2, 0), dtype=torch.float32, device="cuda"))
    bvc.evaluate(cache, st)
    assert st.counts.cpu().tolist() == [256, 0]
    empty = bvc.Cache(2, 0)
    st2 = bvc.EvalState(bvc.soa(w.eval_pts[:10]))
    bvc.evaluate(empty, st2)
    u, _ = bvc.get_solution(st2)
    assert torch.all(u == 0)
