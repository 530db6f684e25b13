"""Alg. 1 (UpdateSolution + GetSolution) composed from the oracle's steps.

Test helper: builds one boundary cache (and source cache) with the oracle and
evaluates u, grad u at points.  The cache positions, normals and measure
ratios are rounded to FP32 before the walks and the gather, as the library
stores them.  The samples lie on the offset boundary at l (Sec. 3.2) and the
source samples fill the region inside it.
"""
import numpy as np

import oracle


def oracle_cache(V, F, g, f, N, W, l, eps, seed, src_grid=None, max_steps=1 << 14, bvh=None, g_vertex=None,
                 sigma=0.0):
    bvh = bvh or oracle.BVH(V, F)
    z, n, e, jac = oracle.sample_boundary(V, F, N, l, seed)
    z32, n32 = z.astype(np.float32), n.astype(np.float32)
    out = oracle.walks(bvh, g, f, z32, W, eps, max_steps, seed, id_base=0, tag=oracle.TAG_WALK, g_vertex=g_vertex,
                       sigma=sigma)
    u_hat, q_hat = oracle.reduce_walks(out["U"], out["grad"], n32, W)
    cache = {"z": z32, "n": n32, "u_hat": u_hat, "q_hat": q_hat, "elem": e,
             "jac": jac.astype(np.float32).astype(np.float64),
             "measure": oracle.boundary_measure(V, F), "walks": out, "N": N,
             "y": None, "c": None, "n_src": 0, "sigma": sigma}
    if f and src_grid is not None:
        if V.shape[1] == 2:
            y, c, ncand = oracle.sample_source2d(V, F, src_grid, seed, f, l=l)
        else:
            y, c, ncand = oracle.sample_source3d(V, F, src_grid, seed, f, l=l)
        cache.update(y=y, c=c, n_src=ncand)
    return cache


def oracle_evaluate(cache, pts):
    ub, us, gb, gs = oracle.gather(cache["z"], cache["n"], cache["u_hat"], cache["q_hat"], cache["measure"],
                                   pts, cache["y"], cache["c"], sigma=cache.get("sigma", 0.0), jac=cache["jac"])
    u = ub / cache["N"]
    grad = gb / cache["N"]
    if cache["n_src"]:
        u = u + us / cache["n_src"]
        grad = grad + gs / cache["n_src"]
    return u, grad


def difference_bound(cache, du, dq, pts, dc=None, rel=1e-5):
    """Element-wise bound on |u_gpu(x) - u_oracle(x)| for two caches on the
    same samples whose estimates differ by du, dq (per boundary sample) and dc
    (per kept source candidate): the triangle inequality over Eq. 3 and Eq. 4,
        sum_i (|dG/dn| |du_i| + |G| |dq_i|) / (p N) + sum_j |G| |dc_j| / M,
    plus rel x the sum of |terms| (the gather's own FP32 tolerance)."""
    z, n, jac = cache["z"], cache["n"], cache["jac"]
    N = cache["N"]
    _, _, _, _, ab_u = oracle.gather(z, n, du, np.zeros_like(du), cache["measure"], pts, want_abs=True, jac=jac,
                                     sigma=cache.get("sigma", 0.0))
    _, _, _, _, ab_q = oracle.gather(z, n, np.zeros_like(dq), dq, cache["measure"], pts, want_abs=True, jac=jac,
                                     sigma=cache.get("sigma", 0.0))
    _, _, _, _, ab = oracle.gather(z, n, cache["u_hat"], cache["q_hat"], cache["measure"], pts, cache["y"],
                                   cache["c"], want_abs=True, jac=jac, sigma=cache.get("sigma", 0.0))
    dim = pts.shape[1]
    bound = (ab_u[:, 0] + ab_q[:, 0]) / N + rel * ab[:, 0] / N
    if cache["n_src"]:
        if dc is not None:
            _, _, _, _, ab_c = oracle.gather(np.zeros((0, dim)), np.zeros((0, dim)), np.zeros(0), np.zeros(0), 1.0,
                                             pts, cache["y"], dc, want_abs=True, sigma=cache.get("sigma", 0.0))
            bound = bound + ab_c[:, 1 + dim] / cache["n_src"]
        bound = bound + rel * ab[:, 1 + dim] / cache["n_src"]
    return bound


def oracle_bvc(V, F, g, f, N, W, l, eps, pts, seed, src_grid=None, max_steps=1 << 14, bvh=None, g_vertex=None,
               sigma=0.0):
    cache = oracle_cache(V, F, g, f, N, W, l, eps, seed, src_grid, max_steps, bvh, g_vertex, sigma)
    return oracle_evaluate(cache, pts)


def mixed_pipeline(V, F, neu, u, f, N, W, l, eps, seed, pts, sigma=0.0):
    """The mixed cache (Sec. 3.2) with the oracle: samples on the Neumann
    part keep offset 0 and carry du/dn = h; Dirichlet samples lie on the
    offset boundary built from the Dirichlet elements and carry walk
    estimates of u and du/dn; Eq. 3 at the points.  sigma > 0: the screened
    walks on stars and the screened gather of App. A."""
    dim = V.shape[1]
    w = oracle.Wost(V, F, neu)
    z, n, e, jac = oracle.sample_boundary_mixed(V, F, N, l, seed, neu)
    on_n = neu[e] == 1
    se = np.where(on_n, e, -1).astype(np.int32)
    o = w.walks(u, [], u, f, z.astype(np.float32), se, W, eps, 1 << 16, seed, sigma=sigma)
    u_hat = o["U"].reshape(N, W).mean(1)
    q_walk = np.einsum("iwd,id->i", o["grad"].reshape(N, W, dim), n) / W
    h = oracle.neumann_eval([], u, dim, z.astype(np.float32).astype(np.float64), n.astype(np.float32)
                            .astype(np.float64))
    q_hat = np.where(on_n, h, q_walk)
    ub, _, gb, _ = oracle.gather(z.astype(np.float32), n.astype(np.float32), u_hat, q_hat,
                                 oracle.boundary_measure(V, F), pts, jac=jac.astype(np.float32), sigma=sigma)
    return ub / N, gb / N, (z, n, e, u_hat, q_hat)
