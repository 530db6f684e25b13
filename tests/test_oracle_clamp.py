"""Pins of the oracle's clamped double-layer correction (Sec. 3.3, Eq. 8-9):
the ray crossings of a closed boundary seen from inside have signs summing
to +1 in every direction (the signed solid angle of a closed surface), and
with the samples on the Dirichlet boundary itself (u = g there, walks stop
at once) the direction-sampled correction matches a deterministic
quadrature of int [dG/dn - clamp_c(dG/dn)] g dz."""
import numpy as np
import pytest

import oracle
from paper_2302_11825_gb300 import workloads as wl


def _dirs(dim, n, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, dim))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("dim", [2, 3])
def test_crossing_signs_sum_to_one_inside(dim):
    if dim == 2:
        V, F = wl.star_polygon(600, seed=1)
        x = np.array([0.1, -0.05])
    else:
        V, F, _ = wl.perturbed_icosphere(2, seed=1, amp=0.2)
        x = np.array([0.05, 0.1, -0.1])
    for om in _dirs(dim, 50, 2):
        t, e, nw = oracle.ray_hits(V, F, 0.0, x, om, 100.0)
        assert len(t) % 2 == 1
        assert int(np.sum(np.sign(nw))) == 1
    # the offset boundary (the mesh with its vertices moved inward, a closed
    # surface) is crossed with signs summing to 1 in every direction too
    for om in _dirs(dim, 400, 3):
        t, e, nw = oracle.ray_hits(V, F, 0.02, x, om, 100.0)
        assert int(np.sum(np.sign(nw))) == 1


def test_correction_matches_quadrature_on_the_boundary():
    # unit circle polygon, samples on the boundary (l = 0): u(z) = g(z)
    V, F = wl.circle_polygon(128)
    g = [(wl.POLY, [0.3, 1.0, -0.5])]  # 0.3 + x - 0.5 y
    c = 2.0
    pts = np.array([[0.97, 0.0], [0.0, -0.985], [0.5, 0.6]])
    corr, nhit = oracle.clamp_correction(oracle.BVH(V, F), g, V, F, 0.0, pts, c, 40000, 1, 1e-6, seed=4)
    # quadrature: per segment, Gauss-Legendre with 400 nodes
    xg, wg = np.polynomial.legendre.leggauss(400)
    ref = np.zeros(len(pts))
    for k, x in enumerate(pts):
        for e in range(F.shape[0]):
            a, b = V[F[e, 0]].astype(np.float64), V[F[e, 1]].astype(np.float64)
            L = np.linalg.norm(b - a)
            n = np.array([b[1] - a[1], -(b[0] - a[0])]) / L
            s = 0.5 * (xg + 1)
            z = a[None] + s[:, None] * (b - a)[None]
            d = z - x
            gn = (d @ n) / (2 * np.pi * np.sum(d * d, 1))
            excess = np.sign(gn) * np.maximum(np.abs(gn) - c, 0.0)
            gz = 0.3 + z[:, 0] - 0.5 * z[:, 1]
            ref[k] += np.sum(0.5 * wg * excess * gz) * L
    print("correction", corr, "quadrature", ref, "hits", nhit)
    se = np.abs(ref) * 0.05 + 2e-3
    assert np.all(np.abs(corr - ref) < se)
    assert abs(ref[2]) < 1e-12 and corr[2] == 0.0  # far from the boundary: nothing to correct
