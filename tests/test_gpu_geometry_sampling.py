"""GPU parity: closest-point queries (bit-exact primitive index and canonical
FP32 distance), boundary samples (K1) and source samples (K4) against the
oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_11825_gb300 import bvc
from paper_2302_11825_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _mesh(name):
    if name == "circle":
        return wl.circle_polygon(256)
    if name == "star20k":
        return wl.star_polygon(20000, 0)
    if name == "sphere4":
        V, F, _ = wl.perturbed_icosphere(4, 0)
        return V, F
    if name == "sphere8":
        V, F, _ = wl.perturbed_icosphere(8, 0)
        return V, F
    raise KeyError(name)


def _points(V, n, seed):
    rng = np.random.default_rng(seed)
    dim = V.shape[1]
    lo, hi = V.min(0) - 0.2, V.max(0) + 0.2
    far = rng.uniform(lo, hi, (n, dim))
    idx = rng.integers(0, V.shape[0], n // 2 + 3)
    near = V[idx].astype(np.float64) + rng.normal(0, 1e-3, (idx.size, dim))
    vert = V[rng.integers(0, V.shape[0], 7)].astype(np.float64)  # exact ties at shared vertices
    return np.concatenate([far, near, vert]).astype(np.float32)


@pytest.mark.parametrize("mesh,n", [("circle", 3000), ("star20k", 3000), ("sphere4", 2000), ("sphere8", 384)])
def test_closest_point_bit_exact(mesh, n):
    V, F = _mesh(mesh)
    geom = bvc.Geometry(V, F)
    pts = _points(V, n, 1)
    d2, prim, cp = bvc.query_closest(geom, bvc.soa(pts), want_cp=True)
    torch.cuda.synchronize()
    d2o, primo = oracle.closest_brute32(V, F, pts)
    np.testing.assert_array_equal(prim.cpu().numpy(), primo)
    np.testing.assert_array_equal(d2.cpu().numpy(), d2o)
    # the closest point is on the chosen element and at the FP64 distance
    d64, _, _ = oracle.closest_brute64(V, F, pts.astype(np.float64))
    cpn = cp.cpu().numpy().T.astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(cpn - pts, axis=1), d64, rtol=1e-5, atol=3e-6)


def test_closest_point_empty_query():
    V, F = _mesh("circle")
    geom = bvc.Geometry(V, F)
    d2, prim, _ = bvc.query_closest(geom, torch.zeros((2, 0), dtype=torch.float32, device="cuda"))
    assert d2.numel() == 0


def test_classify_near_matches_distance():
    V, F = _mesh("star20k")
    geom = bvc.Geometry(V, F)
    pts = _points(V, 4000, 2)
    near = bvc.classify_near(geom, bvc.soa(pts), 0.02).cpu().numpy()
    d2o, _ = oracle.closest_brute32(V, F, pts)
    # near = closer than l x reach, the largest vertex displacement of the
    # offset boundary (FP32, rounded up), so the whole strip between the
    # boundary and the offset boundary is flagged
    _, reach = oracle.offset_disp(V, F)
    assert geom.info().offset_reach == reach
    lr = np.float32(0.02) * np.nextafter(np.float32(reach), np.float32(np.inf))
    np.testing.assert_array_equal(near, (d2o < lr * lr).astype(np.uint8))


@pytest.mark.parametrize("mesh,n,l", [("circle", 1024, 1e-3), ("star20k", 1000, 0.019), ("sphere4", 3001, 0.01)])
def test_boundary_samples_match_oracle(mesh, n, l):
    V, F = _mesh(mesh)
    geom = bvc.Geometry(V, F)
    assert geom.boundary_measure == oracle.boundary_measure(V, F)
    z, nrm, elem, jac = bvc.sample_boundary(geom, n, l, seed=17)
    zo, no, eo, jo = oracle.sample_boundary(V, F, n, l, seed=17)
    np.testing.assert_array_equal(elem.cpu().numpy(), eo)
    np.testing.assert_array_equal(z.cpu().numpy().T, zo.astype(np.float32))
    np.testing.assert_array_equal(nrm.cpu().numpy().T, no.astype(np.float32))
    np.testing.assert_array_equal(jac.cpu().numpy(), jo.astype(np.float32))


@pytest.mark.parametrize("l", [0.0, 0.019])
def test_source_samples_match_oracle(l):
    # kept inside the offset boundary at l (the moved polygon, Sec. 3.2)
    V, F = _mesh("star20k")
    geom = bvc.Geometry(V, F)
    rng = np.random.default_rng(3)
    bumps = wl.gauss_coeffs(0.05, rng.uniform(-10, 10, 8), rng.uniform(-0.5, 0.5, (8, 2)))
    f = [(wl.GAUSS, bumps)]
    grid = (96, 80)
    cache = bvc.Cache(2, 1, n_src_cand=grid[0] * grid[1])
    bvc.sample_source(geom, f, grid, seed=5, cache=cache, l=l)
    torch.cuda.synchronize()
    yo, co, ncand = oracle.sample_source2d(V, F, grid, 5, f, l=l)
    kept = int(cache.n_src_dev.item())
    assert kept == yo.shape[0]
    np.testing.assert_array_equal(cache.src_y[:, :kept].cpu().numpy().T, yo)
    np.testing.assert_allclose(cache.src_c[:kept].cpu().numpy(), co, rtol=2e-6, atol=1e-6 * np.abs(co).max())


def test_source_grid_in_3d_needs_three_entries():
    # 3D source samples take a G0 x G1 x G2 grid; a 2-entry grid is rejected
    V, F = _mesh("sphere4")
    geom = bvc.Geometry(V, F)
    cache = bvc.Cache(3, 1, n_src_cand=16)
    with pytest.raises(bvc.BvcError) as e:
        bvc.sample_source(geom, [(wl.POLY, [1.0])], (4, 4), 0, cache)
    assert e.value.status == bvc.ERR_INVALID_ARG
    cache = bvc.Cache(3, 1, n_src_cand=64)
    bvc.sample_source(geom, [(wl.POLY, [1.0])], (4, 4, 4), 0, cache)
