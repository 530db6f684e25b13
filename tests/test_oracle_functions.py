"""Pins of the oracle's closed-form function terms (the g, f and Neumann
potentials of Eq. 1): values against the encoding's definitions written out
monomial by monomial, GAUSS_LAPLACIAN against a finite-difference Laplacian of
GAUSS, EXP_COS against its equation Delta u = (alpha^2 - beta^2) u, and the
gradients against central differences of the values."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2302_11825_gb300 import workloads as wl


def _monomials(dim):
    # degree t = 0..4, then power of x descending, then (3D) power of y descending
    out = []
    for t in range(5):
        for i in range(t, -1, -1):
            if dim == 2:
                out.append((i, t - i))
            else:
                for j in range(t - i, -1, -1):
                    out.append((i, j, t - i - j))
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_polynomial_terms_follow_the_encoding(dim):
    mons = _monomials(dim)
    assert len(mons) == (15 if dim == 2 else 35)
    rng = np.random.default_rng(dim)
    c = rng.standard_normal(len(mons))
    x = rng.uniform(-1.2, 1.2, (50, dim))
    want = sum(ck * np.prod([x[:, a] ** p for a, p in enumerate(m)], axis=0) for ck, m in zip(c, mons))
    np.testing.assert_allclose(oracle.fn_eval([(wl.POLY, c)], dim, x), want, rtol=1e-12, atol=1e-12)
    # missing trailing coefficients are zero
    np.testing.assert_allclose(oracle.fn_eval([(wl.POLY, c[:4])], dim, x),
                               sum(ck * np.prod([x[:, a] ** p for a, p in enumerate(m)], axis=0)
                                   for ck, m in zip(c[:4], mons[:4])), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_gaussian_terms_and_their_laplacian(dim):
    rng = np.random.default_rng(10 + dim)
    s = 0.3
    amps = [1.5, -0.7]
    cen = rng.uniform(-0.5, 0.5, (2, dim))
    coeffs = [s] + list(itertools.chain.from_iterable([a, *c] for a, c in zip(amps, cen)))
    x = rng.uniform(-1.0, 1.0, (40, dim))
    want = sum(a * np.exp(-np.sum((x - c) ** 2, 1) / (2 * s * s)) for a, c in zip(amps, cen))
    np.testing.assert_allclose(oracle.fn_eval([(wl.GAUSS, coeffs)], dim, x), want, rtol=1e-12, atol=1e-14)
    # GAUSS_LAPLACIAN is the Laplacian of GAUSS (4th-order central differences)
    h = 1e-3
    lap = np.zeros(x.shape[0])
    for a in range(dim):
        e = np.zeros(dim)
        e[a] = h
        f = [oracle.fn_eval([(wl.GAUSS, coeffs)], dim, x + k * e) for k in (-2, -1, 0, 1, 2)]
        lap += (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h)
    np.testing.assert_allclose(oracle.fn_eval([(wl.GAUSS_LAPLACIAN, coeffs)], dim, x), lap, rtol=1e-6, atol=1e-6)


def test_exp_trig_and_exp_cos_terms():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.0, 1.0, (40, 3))
    A, al, be, ga = 1.3, 0.7, 1.1, 0.9
    np.testing.assert_allclose(oracle.fn_eval([(wl.EXP_TRIG, [A, al, be, ga])], 3, x),
                               A * np.exp(al * x[:, 2]) * np.cos(be * x[:, 0]) * np.sin(ga * x[:, 1]),
                               rtol=1e-12, atol=1e-14)
    for dim in (2, 3):
        p = x[:, :dim]
        A, al, be = 0.8, 1.4, 0.6
        u = oracle.fn_eval([(5, [A, al, be])], dim, p)
        np.testing.assert_allclose(u, A * np.exp(al * p[:, -1]) * np.cos(be * p[:, 0]), rtol=1e-12, atol=1e-14)
        # a solution of Delta u = (alpha^2 - beta^2) u
        h = 1e-3
        lap = np.zeros(p.shape[0])
        for a in range(dim):
            e = np.zeros(dim)
            e[a] = h
            f = [oracle.fn_eval([(5, [A, al, be])], dim, p + k * e) for k in (-2, -1, 0, 1, 2)]
            lap += (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h)
        np.testing.assert_allclose(lap, (al * al - be * be) * u, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradients_are_central_differences(dim):
    rng = np.random.default_rng(20 + dim)
    terms = [(wl.POLY, rng.standard_normal(15 if dim == 2 else 35)),
             (wl.GAUSS, [0.4, 1.2] + list(rng.uniform(-0.3, 0.3, dim))),
             (wl.GAUSS_LAPLACIAN, [0.5, -0.8] + list(rng.uniform(-0.3, 0.3, dim))),
             (5, [0.9, 0.5, 1.3])]
    if dim == 3:
        terms[3] = (wl.EXP_TRIG, [1.1, 0.4, 0.8, 1.2])
    x = rng.uniform(-0.8, 0.8, (30, dim))
    g = oracle.fn_grad(terms, dim, x)
    h = 1e-5
    for a in range(dim):
        e = np.zeros(dim)
        e[a] = h
        fd = (oracle.fn_eval(terms, dim, x + e) - oracle.fn_eval(terms, dim, x - e)) / (2 * h)
        np.testing.assert_allclose(g[:, a], fd, rtol=1e-7, atol=1e-7)
