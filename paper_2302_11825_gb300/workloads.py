"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no step of the method.  It builds the inputs that both the
CUDA path and the CPU oracle consume:

* boundary meshes: a regular polygon (unit circle), a noisy 7-lobed star
  polygon, and a radially perturbed icosphere -- counter-clockwise polygons
  and outward-wound triangles, as the library requires;
* evaluation point sets (grids clipped to the domain, uniform random
  interior points);
* the coefficients of the boundary data g and source f of Eq. 1, as term
  lists ``[(kind, coeffs), ...]`` in the library's function encoding;
* closed-form exact solutions (value and gradient) used to measure error.

Function encoding (the library's ``bvc_term``): kind 1 POLY (monomials of
total degree <= 4, ordered by degree t, then power of x descending, then (3D)
power of y descending), kind 2 GAUSS ``[s, A_1, c_1, A_2, c_2, ...]`` =
sum A_k exp(-|x-c_k|^2/(2 s^2)), kind 3 GAUSS_LAPLACIAN (its Laplacian, same
coefficients), kind 4 EXP_TRIG ``[A, alpha, beta, gamma]`` =
A exp(alpha z) cos(beta x) sin(gamma y).

The paper's own scenes (wind tunnel, cage, spacesuit, gallery) are not
available; these generators stand in for them with the sizes of the
benchmark configurations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

POLY, GAUSS, GAUSS_LAPLACIAN, EXP_TRIG = 1, 2, 3, 4


# ---------------------------------------------------------------- meshes
def circle_polygon(n_seg: int, radius: float = 1.0):
    """Regular n-gon inscribed in a circle, counter-clockwise."""
    th = 2.0 * np.pi * np.arange(n_seg) / n_seg
    V = np.stack([radius * np.cos(th), radius * np.sin(th)], 1).astype(np.float32)
    F = np.stack([np.arange(n_seg), (np.arange(n_seg) + 1) % n_seg], 1).astype(np.int32)
    return V, F


def _fourier_noise(seed: int, n_modes: int = 16):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n_modes)
    b = rng.standard_normal(n_modes)
    k = np.arange(1, n_modes + 1)

    def noise(th):
        th = np.asarray(th, dtype=np.float64)
        return (a[None, :] * np.cos(np.outer(th, k)) + b[None, :] * np.sin(np.outer(th, k))) @ (1.0 / k)

    fine = np.linspace(0.0, 2.0 * np.pi, 1 << 16, endpoint=False)
    scale = 1.0 / np.max(np.abs(noise(fine)))
    return lambda th: scale * noise(th)


def star_radius_fn(seed: int, lobes: int = 7, amp: float = 0.3, noise_amp: float = 0.05):
    """r(theta) = 1 + amp sin(lobes theta) + noise_amp * n(theta), where n is a
    smooth seeded Fourier series (16 modes, N(0,1)/k coefficients) scaled to
    max |n| = 1."""
    noise = _fourier_noise(seed)
    return lambda th: 1.0 + amp * np.sin(lobes * np.asarray(th)) + noise_amp * noise(th)


def star_polygon(n_seg: int, seed: int):
    """Nonconvex star polygon, vertices at uniform angles, counter-clockwise."""
    r = star_radius_fn(seed)
    th = 2.0 * np.pi * np.arange(n_seg) / n_seg
    rr = r(th)
    V = np.stack([rr * np.cos(th), rr * np.sin(th)], 1).astype(np.float32)
    F = np.stack([np.arange(n_seg), (np.arange(n_seg) + 1) % n_seg], 1).astype(np.int32)
    return V, F


def inside_star_polygon(V: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Exact inside test for a polygon star-shaped about the origin whose
    vertices sit at uniform angles (as built by ``star_polygon``)."""
    n = V.shape[0]
    pts = np.asarray(pts, dtype=np.float64)
    th = np.mod(np.arctan2(pts[:, 1], pts[:, 0]), 2.0 * np.pi)
    i = np.minimum((th / (2.0 * np.pi) * n).astype(np.int64), n - 1)
    a = V[i].astype(np.float64)
    b = V[(i + 1) % n].astype(np.float64)
    cross = (b[:, 0] - a[:, 0]) * (pts[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (pts[:, 0] - a[:, 0])
    return cross > 0.0


def distance_to_polygon(V: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Brute-force distance from points to a closed polygon (generator use)."""
    a = V.astype(np.float64)
    b = np.roll(a, -1, axis=0)
    ab = b - a
    den = np.sum(ab * ab, 1)
    out = np.empty(pts.shape[0])
    for s in range(0, pts.shape[0], 256):
        p = pts[s:s + 256, None, :].astype(np.float64)
        t = np.clip(np.sum((p - a[None]) * ab[None], 2) / den[None], 0.0, 1.0)
        c = a[None] + t[..., None] * ab[None]
        out[s:s + 256] = np.sqrt(np.min(np.sum((p - c) ** 2, 2), 1))
    return out


_ICO_T = (1.0 + 5.0 ** 0.5) / 2.0


def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4^subdiv triangles, outward counter-clockwise."""
    t = _ICO_T
    V = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(subdiv):
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        e = np.concatenate([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)])
        key = np.sort(e, 1)
        uniq, inv = np.unique(key[:, 0] * (V.shape[0] + 1) + key[:, 1], return_inverse=True)
        i0 = uniq // (V.shape[0] + 1)
        i1 = uniq % (V.shape[0] + 1)
        mid = V[i0] + V[i1]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        nf = F.shape[0]
        m = V.shape[0] + inv
        ab, bc, ca = m[:nf], m[nf:2 * nf], m[2 * nf:]
        V = np.concatenate([V, mid])
        F = np.concatenate([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
                            np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)])
    return V, F.astype(np.int32)


def radial_noise_fn(seed: int, n_waves: int = 16):
    """n(p) = sum_j cos(k_j . p + phi_j), |k_j| ~ U[2,8], directions uniform,
    phases uniform; normalised below so that max |n| = 1 on the mesh."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n_waves, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    k = d * rng.uniform(2.0, 8.0, (n_waves, 1))
    phi = rng.uniform(0.0, 2.0 * np.pi, n_waves)
    return lambda p: np.cos(np.asarray(p, dtype=np.float64) @ k.T + phi[None, :]).sum(1)


def perturbed_icosphere(subdiv: int, seed: int, amp: float = 0.02):
    """Icosphere with vertices moved radially by a factor 1 + amp * n(p),
    n a seeded sum of plane waves scaled to max |n| = 1 over the vertices.
    Returns (V float32, F int32, radius function r(unit direction))."""
    V, F = icosphere(subdiv)
    noise = radial_noise_fn(seed)
    nv = noise(V)
    scale = 1.0 / np.max(np.abs(nv))

    def r(u):
        return 1.0 + amp * scale * noise(u)

    V = V * r(V)[:, None]
    return V.astype(np.float32), F, r


# ---------------------------------------------------------------- evaluation sets
def grid_points(lo, hi, n: int) -> np.ndarray:
    """Cell centres of an n x n grid over the box [lo, hi] (2D)."""
    xs = lo[0] + (np.arange(n) + 0.5) * (hi[0] - lo[0]) / n
    ys = lo[1] + (np.arange(n) + 0.5) * (hi[1] - lo[1]) / n
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], 1)


def random_in_star_body(n: int, r_fn, seed: int, shrink: float = 0.99) -> np.ndarray:
    """Uniform points in the body {|p| <= shrink r(p/|p|)} (star-shaped about 0):
    uniform direction, accepted with probability (r/r_max)^3, radius
    shrink r xi^(1/3)."""
    rng = np.random.default_rng(seed)
    out = []
    have = 0
    rmax = 1.0 + 0.021
    while have < n:
        m = 2 * (n - have) + 1024
        d = rng.standard_normal((m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        r = r_fn(d)
        keep = rng.uniform(size=m) < (r / rmax) ** 3
        d, r = d[keep], r[keep]
        rad = shrink * r * rng.uniform(size=d.shape[0]) ** (1.0 / 3.0)
        out.append(d * rad[:, None])
        have += d.shape[0]
    return np.concatenate(out)[:n]


# ---------------------------------------------------------------- problem data
def poly2d_coeffs(monomials: dict) -> list:
    """{(i, j): c} for c x^i y^j -> POLY coefficient list (2D order)."""
    out = []
    for t in range(5):
        for i in range(t, -1, -1):
            out.append(float(monomials.get((i, t - i), 0.0)))
    while out and out[-1] == 0.0 and len(out) > 1:
        out.pop()
    return out


def poly3d_coeffs(monomials: dict) -> list:
    """{(i, j, k): c} for c x^i y^j z^k -> POLY coefficient list (3D order)."""
    out = []
    for t in range(5):
        for i in range(t, -1, -1):
            for j in range(t - i, -1, -1):
                out.append(float(monomials.get((i, j, t - i - j), 0.0)))
    while out and out[-1] == 0.0 and len(out) > 1:
        out.pop()
    return out


def gauss_coeffs(sigma: float, amps, centres) -> list:
    out = [float(sigma)]
    for a, c in zip(amps, centres):
        out += [float(a)] + [float(x) for x in c]
    return out


def eval_terms(terms, dim: int, x: np.ndarray):
    """Closed-form value and gradient of a term list at points x[n, dim]."""
    x = np.asarray(x, dtype=np.float64)
    val = np.zeros(x.shape[0])
    grad = np.zeros((x.shape[0], dim))
    for kind, coeffs in terms:
        c = np.asarray(coeffs, dtype=np.float64)
        if kind == POLY:
            idx = 0
            for t in range(5):
                if dim == 2:
                    exps = [(i, t - i) for i in range(t, -1, -1)]
                else:
                    exps = [(i, j, t - i - j) for i in range(t, -1, -1) for j in range(t - i, -1, -1)]
                for e in exps:
                    if idx >= c.size:
                        break
                    if c[idx] != 0.0:
                        mono = np.prod([x[:, a] ** e[a] for a in range(dim)], 0)
                        val += c[idx] * mono
                        for a in range(dim):
                            if e[a] > 0:
                                ee = list(e)
                                ee[a] -= 1
                                grad[:, a] += c[idx] * e[a] * np.prod([x[:, b] ** ee[b] for b in range(dim)], 0)
                    idx += 1
        elif kind in (GAUSS, GAUSS_LAPLACIAN):
            s = c[0]
            per = 1 + dim
            nb = (c.size - 1) // per
            for k in range(nb):
                A = c[1 + k * per]
                ctr = c[2 + k * per: 2 + k * per + dim]
                dx = x - ctr[None, :]
                r2 = np.sum(dx * dx, 1)
                e = np.exp(-r2 / (2 * s * s))
                if kind == GAUSS:
                    val += A * e
                    grad += (A * e * (-1.0 / (s * s)))[:, None] * dx
                else:
                    q = r2 / s ** 4 - dim / s ** 2
                    val += A * q * e
                    dq = 2.0 / s ** 4
                    grad += (A * e * (dq - q / (s * s)))[:, None] * dx
        elif kind == EXP_TRIG:
            A, al, be, ga = c[:4]
            ez = np.exp(al * x[:, 2])
            cx, sx = np.cos(be * x[:, 0]), np.sin(be * x[:, 0])
            cy, sy = np.cos(ga * x[:, 1]), np.sin(ga * x[:, 1])
            val += A * ez * cx * sy
            grad[:, 0] += A * ez * (-be * sx) * sy
            grad[:, 1] += A * ez * cx * (ga * cy)
            grad[:, 2] += A * al * ez * cx * sy
        else:
            raise ValueError(f"unknown term kind {kind}")
    return val, grad


# ---------------------------------------------------------------- configurations
@dataclass
class Workload:
    """One synthetic problem: mesh, data, cache sizes and evaluation set."""
    name: str
    dim: int
    V: np.ndarray
    F: np.ndarray
    g: list
    f: list
    n_samples: int
    walks: int
    offset_l: float
    eps: float
    eval_pts: np.ndarray
    src_grid: tuple = (0, 0)
    exact: list | None = None          # closed-form solution terms, if any
    seed: int = 0
    meta: dict = field(default_factory=dict)


def bbox_diagonal(V: np.ndarray) -> float:
    return float(np.linalg.norm(V.max(0).astype(np.float64) - V.min(0).astype(np.float64)))


def circle_laplace(n_samples: int = 1024, walks: int = 64, grid: int = 64, n_seg: int = 256,
                   seed: int = 0) -> Workload:
    """2D Laplace on the unit circle as a 256-gon; g = Re(z^3) = x^3 - 3xy^2
    (harmonic, so u = g); 1024 samples offset l = 1e-3 inward x 64 walks;
    u and grad u on a 64x64 grid clipped to r < 0.95.  The shell is l/5."""
    V, F = circle_polygon(n_seg)
    g = [(POLY, poly2d_coeffs({(3, 0): 1.0, (1, 2): -3.0}))]
    pts = grid_points((-1.0, -1.0), (1.0, 1.0), grid)
    pts = pts[np.sum(pts * pts, 1) < 0.95 ** 2]
    l = 1e-3
    return Workload("circle_laplace_256seg", 2, V, F, g, [], n_samples, walks, l, l / 5.0,
                    pts.astype(np.float32), exact=g, seed=seed)


def star_poisson(n_samples: int = 65536, walks: int = 256, grid: int = 1024, n_seg: int = 20000,
                 src_grid=(256, 256), seed: int = 0, manufactured: bool = False,
                 n_bumps: int = 8, sigma: float = 0.05) -> Workload:
    """2D Poisson on a nonconvex 20k-segment star, r = 1 + 0.3 sin 7t + 0.05 n(t);
    f = 8 Gaussian bumps (sigma 0.05, amplitudes U[-10,10], centres uniform in
    the domain at distance >= 3 sigma from the boundary); g = x^2 - y^2;
    65536 samples x 256 walks; 65536 source candidates; 1024^2 grid clipped to
    the domain.  eps = 1e-3 x bbox diagonal, l = 5 eps.

    ``manufactured=True`` keeps the geometry, sizes and bump centres but sets
    u* = x^2 - y^2 + sum A_k exp(-|x-c_k|^2/(2 sigma^2)), f = Laplacian(u*),
    g = u* on the boundary, so that the exact solution is known."""
    V, F = star_polygon(n_seg, seed)
    rng = np.random.default_rng(seed + 1)
    amps = rng.uniform(-10.0, 10.0, n_bumps)
    lo, hi = V.min(0).astype(np.float64), V.max(0).astype(np.float64)
    centres = []
    while len(centres) < n_bumps:
        c = rng.uniform(lo, hi, (64, 2))
        ok = inside_star_polygon(V, c)
        c = c[ok]
        if c.shape[0]:
            d = distance_to_polygon(V, c)
            c = c[d >= 3.0 * sigma]
        centres += [tuple(p) for p in c[: n_bumps - len(centres)]]
    centres = np.asarray(centres)
    quad = [(POLY, poly2d_coeffs({(2, 0): 1.0, (0, 2): -1.0}))]
    bumps = gauss_coeffs(sigma, amps, centres)
    if manufactured:
        g = quad + [(GAUSS, bumps)]
        f = [(GAUSS_LAPLACIAN, bumps)]
        exact = g
    else:
        g = quad
        f = [(GAUSS, bumps)]
        exact = None
    pts = grid_points(lo, hi, grid)
    pts = pts[inside_star_polygon(V, pts)]
    eps = 1e-3 * bbox_diagonal(V)
    name = "star_poisson_20kseg" + ("_manufactured" if manufactured else "")
    return Workload(name, 2, V, F, g, f, n_samples, walks, 5.0 * eps, eps, pts.astype(np.float32),
                    src_grid=tuple(src_grid), exact=exact, seed=seed,
                    meta={"amps": amps, "centres": centres, "sigma": sigma})


def icosphere_laplace(subdiv: int = 8, n_samples: int = 262144, walks: int = 128, plane: int = 512,
                      n_random: int = 1_000_000, seed: int = 0) -> Workload:
    """3D Laplace on a perturbed icosphere (subdivision 8: 1,310,720 triangles,
    radial noise 2%); g = exp(0.5 z) cos(0.3 x) sin(0.4 y) (harmonic);
    262144 samples x 128 walks; evaluate a 512 x 512 slice plane z = 0 plus
    1M uniform random interior points.  eps = 1e-3 x bbox diagonal, l = 5 eps."""
    V, F, r = perturbed_icosphere(subdiv, seed)
    g = [(EXP_TRIG, [1.0, 0.5, 0.3, 0.4])]
    lo, hi = V.min(0).astype(np.float64), V.max(0).astype(np.float64)
    pl = grid_points(lo[:2], hi[:2], plane)
    pl3 = np.concatenate([pl, np.zeros((pl.shape[0], 1))], 1)
    rad = np.linalg.norm(pl3, axis=1)
    u = pl3 / np.maximum(rad, 1e-30)[:, None]
    pl3 = pl3[rad < r(u) * (1.0 - 1e-5)]
    rnd = random_in_star_body(n_random, r, seed + 7)
    pts = np.concatenate([pl3, rnd]).astype(np.float32)
    eps = 1e-3 * bbox_diagonal(V)
    return Workload(f"icosphere{subdiv}_laplace", 3, V, F, g, [], n_samples, walks, 5.0 * eps, eps, pts,
                    exact=g, seed=seed, meta={"n_plane": pl3.shape[0], "n_random": rnd.shape[0]})


# ---------------------------------------------------------------- many right-hand sides
def poly_exponents(dim: int):
    """Exponent tuples of the POLY monomials (degree <= 4) in library order."""
    out = []
    for t in range(5):
        for i in range(t, -1, -1):
            if dim == 2:
                out.append((i, t - i))
            else:
                for j in range(t - i, -1, -1):
                    out.append((i, j, t - i - j))
    return out


def harmonic_basis(dim: int) -> np.ndarray:
    """Orthonormal basis (rows, in monomial coefficients) of the harmonic
    polynomials of degree <= 4: the null space of the Laplacian on the
    monomial coefficients (9 functions in 2D, 25 in 3D)."""
    ex = poly_exponents(dim)
    index = {e: n for n, e in enumerate(ex)}
    L = np.zeros((len(ex), len(ex)))
    for col, e in enumerate(ex):
        for a in range(dim):
            if e[a] >= 2:
                f = list(e)
                f[a] -= 2
                L[index[tuple(f)], col] += e[a] * (e[a] - 1)
    _, sv, vt = np.linalg.svd(L)
    rank = int(np.sum(sv > 1e-9))
    return vt[rank:]


def random_harmonic_polys(dim: int, k: int, seed: int) -> np.ndarray:
    """k random harmonic polynomials up to degree 4 with N(0,1) coordinates
    in an orthonormal harmonic basis: [k][n_monomials] coefficients."""
    B = harmonic_basis(dim)
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, B.shape[0])) @ B


def perturbed_ellipsoid(subdiv: int, axes, seed: int, amp: float = 0.02, centre=(0.0, 0.0, 0.0)):
    """An icosphere stretched to the given semi-axes, radially perturbed,
    moved to `centre`; outward counter-clockwise triangles."""
    V, F, _ = perturbed_icosphere(subdiv, seed, amp)
    V = V.astype(np.float64) * np.asarray(axes)[None, :] + np.asarray(centre)[None, :]
    return V.astype(np.float32), F


def batched_meshes(n_meshes: int = 16, seed: int = 0):
    """Meshes of uneven size (about 10k to 500k triangles): perturbed
    icospheres and ellipsoids, and unions of two disjoint ellipsoids.
    Returns a list of (name, V, F, inside(p) predicate)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_meshes):
        kind = i % 4
        sub = [5, 6, 7, 6][kind] if i % 8 < 4 else [6, 5, 6, 7][kind]
        if kind == 0 or (kind == 2 and sub == 7):
            V, F, r = perturbed_icosphere(sub, seed + i)
            out.append((f"icosphere{sub}_{i}", V, F, ("sphere", (0.0, 0.0, 0.0), (0.97, 0.97, 0.97))))
        elif kind in (1, 2):
            ax = tuple(rng.uniform(0.6, 1.4, 3))
            V, F = perturbed_ellipsoid(sub, ax, seed + i)
            out.append((f"ellipsoid{sub}_{i}", V, F, ("ellipsoid", (0.0, 0.0, 0.0), tuple(0.97 * a for a in ax))))
        else:
            ax1 = tuple(rng.uniform(0.5, 0.9, 3))
            ax2 = tuple(rng.uniform(0.5, 0.9, 3))
            c1, c2 = (-1.2, 0.0, 0.0), (1.2, 0.0, 0.0)
            V1, F1 = perturbed_ellipsoid(sub - 1, ax1, seed + i, centre=c1)
            V2, F2 = perturbed_ellipsoid(sub - 1, ax2, seed + 100 + i, centre=c2)
            V = np.concatenate([V1, V2])
            F = np.concatenate([F1, F2 + V1.shape[0]]).astype(np.int32)
            out.append((f"union{sub - 1}x2_{i}", V, F,
                        ("union", (c1, c2), (tuple(0.97 * a for a in ax1), tuple(0.97 * a for a in ax2)))))
    return out


def random_points_in(shape, n: int, seed: int) -> np.ndarray:
    """Uniform points inside the shrunk body described by `shape` (the 0.97
    shrink keeps them inside the radially perturbed surfaces)."""
    rng = np.random.default_rng(seed)
    kind = shape[0]
    if kind == "union":
        (c1, c2), (a1, a2) = shape[1], shape[2]
        v1, v2 = np.prod(a1), np.prod(a2)
        n1 = int(round(n * v1 / (v1 + v2)))
        return np.concatenate([random_points_in(("ellipsoid", c1, a1), n1, seed + 1),
                               random_points_in(("ellipsoid", c2, a2), n - n1, seed + 2)])
    c, a = np.asarray(shape[1]), np.asarray(shape[2])
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(size=n) ** (1.0 / 3.0) * 0.98
    return (c[None, :] + d * r[:, None] * a[None, :]).astype(np.float32)


@dataclass
class BatchedWorkload:
    """Independent 3D Laplace problems on meshes of uneven size, each with k
    random harmonic polynomial Dirichlet data (their own exact solutions)."""
    name: str
    meshes: list            # (name, V, F, shape) per mesh
    n_samples: int          # boundary samples per mesh
    walks: int
    n_points: int           # evaluation points per mesh
    k: int                  # right-hand sides per mesh
    coeffs: np.ndarray      # [meshes][k][35] monomial coefficients
    pts: list               # [n_points][3] float32 per mesh
    eps: list               # shell per mesh: 1e-3 x bbox diagonal
    offset_l: list          # 5 eps


def batched_laplace(n_meshes: int = 16, n_samples: int = 32768, walks: int = 128, n_points: int = 65536,
                    k: int = 64, seed: int = 0) -> BatchedWorkload:
    """16 perturbed icospheres, ellipsoids and unions of two disjoint
    ellipsoids (20k to 330k triangles) x 64 harmonic polynomials of degree
    <= 4; 32k boundary samples x 128 walks and 64k uniform interior points
    per mesh.  The walk count is not fixed by the batched configuration: it
    takes the 128 of the single 3D configuration."""
    meshes = batched_meshes(n_meshes, seed)
    coeffs = np.stack([random_harmonic_polys(3, k, seed=1000 + seed + j) for j in range(n_meshes)])
    pts = [random_points_in(m[3], n_points, seed=2000 + seed + j) for j, m in enumerate(meshes)]
    eps = [1e-3 * bbox_diagonal(m[1]) for m in meshes]
    return BatchedWorkload(f"batched{n_meshes}_laplace_k{k}", meshes, n_samples, walks, n_points, k, coeffs, pts,
                           eps, [5.0 * e for e in eps])


# ---------------------------------------------------------------- box with obstacles
def box_surface(lo, hi, cells_per_unit: int):
    """Surface of an axis-aligned box as a triangle grid, wound outward."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    n = [max(1, int(round((hi[a] - lo[a]) * cells_per_unit))) for a in range(3)]
    V, F = [], []
    for axis in range(3):
        u, v = [(1, 2), (2, 0), (0, 1)][axis]
        for side, val in ((0, lo[axis]), (1, hi[axis])):
            nu, nv = n[u], n[v]
            base = sum(len(x) for x in V)
            grid = np.zeros(((nu + 1) * (nv + 1), 3))
            iu, iv = np.meshgrid(np.arange(nu + 1), np.arange(nv + 1), indexing="ij")
            grid[:, axis] = val
            grid[:, u] = lo[u] + iu.ravel() * (hi[u] - lo[u]) / nu
            grid[:, v] = lo[v] + iv.ravel() * (hi[v] - lo[v]) / nv
            V.append(grid)
            for i in range(nu):
                for j in range(nv):
                    a = base + i * (nv + 1) + j
                    b, c, d = a + (nv + 1), a + (nv + 1) + 1, a + 1
                    # (u, v, axis) is right-handed: u x v = +axis
                    tri = [(a, b, c), (a, c, d)] if side == 1 else [(a, c, b), (a, d, c)]
                    F.extend(tri)
    V = np.concatenate(V)
    # merge duplicated edge vertices
    key = np.round(V * 1e6).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    return V[first].astype(np.float32), inv.ravel()[np.asarray(F)].astype(np.int32)


def box_with_obstacles(lo=(-2.0, -1.0, -1.0), hi=(2.0, 1.0, 1.0), n_box: int = 8, ellipsoids=(), subdiv: int = 4,
                       seed: int = 0, amp: float = 0.0):
    """The boundary of a box minus a union of ellipsoids: the box wound
    outward, each ellipsoid (an icosphere scaled by its semi-axes, optionally
    radially perturbed) wound inward.  Overlapping ellipsoids are left as
    they are (a self-intersecting boundary, no repair)."""
    Vb, Fb = box_surface(lo, hi, n_box)
    Vs, Fs = [Vb], [Fb]
    off = Vb.shape[0]
    for k, (c, ax) in enumerate(ellipsoids):
        Ve, Fe = perturbed_ellipsoid(subdiv, ax, seed + k, amp=amp, centre=c) if amp > 0 else (None, None)
        if Ve is None:
            Vi, Fi = icosphere(subdiv)
            Ve = (Vi * np.asarray(ax)[None, :] + np.asarray(c)[None, :]).astype(np.float32)
            Fe = Fi
        Vs.append(Ve)
        Fs.append(Fe[:, ::-1] + off)
        off += Ve.shape[0]
    return np.concatenate(Vs).astype(np.float32), np.concatenate(Fs).astype(np.int32)


@dataclass
class InverseWorkload:
    """Differentiable inverse problem: Delta u = f in a box minus a union of
    overlapping ellipsoids, u = g on its (self-intersecting, unrepaired)
    boundary; g at the mesh vertices = Phi c with Gaussian radial basis
    functions (rbf_centres, rbf_sigma), f = sum_k A_k Gaussian bumps."""
    name: str
    V: np.ndarray
    F: np.ndarray
    ellipsoids: list
    rbf_centres: np.ndarray
    rbf_sigma: float
    bump_centres: np.ndarray
    bump_sigma: float
    c_true: np.ndarray
    a_true: np.ndarray
    obs_pts: np.ndarray
    n_samples: int
    walks: int
    eps: float
    offset_l: float
    src_grid: tuple


def in_domain_box_obstacles(p, lo, hi, ellipsoids, margin: float) -> np.ndarray:
    """Points inside the box and outside every ellipsoid, at least `margin`
    (box walls) or a relative margin (ellipsoids) away from the boundary."""
    p = np.asarray(p, dtype=np.float64)
    ok = np.all((p > np.asarray(lo) + margin) & (p < np.asarray(hi) - margin), axis=1)
    for c, ax in ellipsoids:
        r = np.sqrt(np.sum(((p - np.asarray(c)) / np.asarray(ax)) ** 2, axis=1))
        ok &= r > 1.0 + margin / min(ax)
    return ok


def inverse_problem(n_obs: int = 100000, n_samples: int = 65536, walks: int = 64, subdiv: int = 6,
                    n_rbf: int = 256, seed: int = 0) -> InverseWorkload:
    """Box [-2,2] x [-1,1]^2 with an obstacle of 5 overlapping ellipsoids
    (icospheres of subdivision 6, 81920 triangles each: about 410k
    triangles); g = Phi c with 256 Gaussian RBFs centred at seeded boundary
    vertices; 8 Gaussian source bumps; 100k seeded interior observation
    points; 65536 samples x 64 walks and a 64 x 32 x 32 source grid (the
    configuration fixes neither).  eps = 1e-3 x bbox diagonal, l = 5 eps."""
    rng = np.random.default_rng(seed)
    lo, hi = (-2.0, -1.0, -1.0), (2.0, 1.0, 1.0)
    ell = []
    for k in range(5):
        c = (-0.8 + 0.4 * k + rng.uniform(-0.05, 0.05), rng.uniform(-0.15, 0.15), rng.uniform(-0.15, 0.15))
        ax = tuple(rng.uniform(0.3, 0.45, 3))
        ell.append((c, ax))
    V, F = box_with_obstacles(lo, hi, n_box=8, ellipsoids=ell, subdiv=subdiv)
    rbf_c = V[rng.choice(V.shape[0], n_rbf, replace=False)].astype(np.float64)
    bc = []
    while len(bc) < 8:
        q = rng.uniform(lo, hi, (64, 3))
        q = q[in_domain_box_obstacles(q, lo, hi, ell, 0.3)]
        bc.extend(q[: 8 - len(bc)])
    obs = []
    while sum(len(o) for o in obs) < n_obs:
        q = rng.uniform(lo, hi, (2 * n_obs, 3))
        obs.append(q[in_domain_box_obstacles(q, lo, hi, ell, 0.05)])
    obs = np.concatenate(obs)[:n_obs].astype(np.float32)
    eps = 1e-3 * bbox_diagonal(V)
    return InverseWorkload(f"inverse_box5ellipsoids_{F.shape[0] // 1000}k", V, F, ell, rbf_c, 0.4,
                           np.asarray(bc), 0.15, rng.standard_normal(n_rbf), rng.uniform(-10, 10, 8), obs,
                           n_samples, walks, eps, 5 * eps, (64, 32, 32))


# ---------------------------------------------------------------- mixed boundaries
def rect_polygon(lo, hi, n_per_unit: int):
    """Counter-clockwise polygon of an axis-aligned rectangle with sides cut
    into segments of length ~1/n_per_unit.  Returns V, F and each element's
    side: 0 bottom (y = lo), 1 right (x = hi), 2 top, 3 left."""
    (x0, y0), (x1, y1) = lo, hi
    corners = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
    V, side = [], []
    for s in range(4):
        a, b = np.asarray(corners[s], float), np.asarray(corners[(s + 1) % 4], float)
        n = max(1, int(round(np.linalg.norm(b - a) * n_per_unit)))
        for k in range(n):
            V.append(a + (b - a) * k / n)
            side.append(s)
    V = np.asarray(V, dtype=np.float32)
    n = V.shape[0]
    F = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32)
    return V, F, np.asarray(side, np.int32)


def l_shape_polygon(n_per_unit: int):
    """[-1,1]^2 without the quadrant (0,1] x (0,1], counter-clockwise; the
    corner (0,0) is reflex.  Returns V, F."""
    corners = [(-1.0, -1.0), (1.0, -1.0), (1.0, 0.0), (0.0, 0.0), (0.0, 1.0), (-1.0, 1.0)]
    V = []
    for s in range(len(corners)):
        a, b = np.asarray(corners[s], float), np.asarray(corners[(s + 1) % len(corners)], float)
        n = max(1, int(round(np.linalg.norm(b - a) * n_per_unit)))
        for k in range(n):
            V.append(a + (b - a) * k / n)
    V = np.asarray(V, dtype=np.float32)
    n = V.shape[0]
    F = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32)
    return V, F


def element_midpoints(V, F) -> np.ndarray:
    return V[F].astype(np.float64).mean(1)


@dataclass
class MixedWorkload:
    """A mixed Dirichlet / Neumann problem (Eq. 1, sigma = 0): g on the
    Dirichlet part, h = value + n . grad(potential) on the Neumann part."""
    name: str
    dim: int
    V: np.ndarray
    F: np.ndarray
    neumann: np.ndarray
    g: list
    h_value: list
    h_potential: list
    f: list
    n_samples: int
    walks: int
    offset_l: float
    eps: float
    eval_pts: np.ndarray
    src_grid: tuple = (0, 0)
    exact: list | None = None
    seed: int = 0
    meta: dict = field(default_factory=dict)


def star_mixed(n_samples: int = 65536, walks: int = 64, grid: int = 1024, n_seg: int = 20000,
               src_grid=(256, 256), seed: int = 0, n_bumps: int = 8, sigma: float = 0.05) -> MixedWorkload:
    """A Neumann-dominated 2D mixed problem on the 20k-segment star of
    ``star_poisson``: elements whose midpoint angle t has sin(7 t) < 0.5
    (the valleys and flanks, about 2/3 of the boundary, with reflex vertices)
    are Neumann, the lobe tips Dirichlet.  Manufactured solution
    u* = x^2 - y^2 + 8 Gaussian bumps (sigma 0.05, amplitudes U[-10,10]):
    g = u*, h = n . grad u*, f = Laplacian(u*).  65536 samples x 64 walks,
    256^2 source candidates, the 1024^2 grid clipped to the domain;
    eps = 1e-3 x bbox diagonal, l = 5 eps."""
    base = star_poisson(n_samples=n_samples, walks=walks, grid=grid, n_seg=n_seg, src_grid=src_grid, seed=seed,
                        manufactured=True, n_bumps=n_bumps, sigma=sigma)
    mid = element_midpoints(base.V, base.F)
    th = np.arctan2(mid[:, 1], mid[:, 0])
    neu = (np.sin(7.0 * th) < 0.5).astype(np.uint8)
    return MixedWorkload("star_mixed_20kseg", 2, base.V, base.F, neu, base.g, [], base.g, base.f, n_samples, walks,
                         base.offset_l, base.eps, base.eval_pts, src_grid=base.src_grid, exact=base.exact,
                         seed=seed, meta=dict(base.meta))


def box_mixed_3d(cells_per_unit: int = 4, n_samples: int = 4096, walks: int = 64, seed: int = 0) -> MixedWorkload:
    """Unit cube, Dirichlet on the faces x = 0 and x = 1, Neumann on the
    other four; harmonic u* = x^2 - y^2 + 0.5 x z: g = u*, h = n . grad u*."""
    V, F = box_surface((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), cells_per_unit)
    mid = element_midpoints(V, F)
    neu = ((mid[:, 0] > 1e-6) & (mid[:, 0] < 1.0 - 1e-6)).astype(np.uint8)
    u = [(POLY, poly3d_coeffs({(2, 0, 0): 1.0, (0, 2, 0): -1.0, (1, 0, 1): 0.5}))]
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.1, 0.9, (512, 3)).astype(np.float32)
    eps = 1e-3 * bbox_diagonal(V)
    return MixedWorkload("box_mixed_3d", 3, V, F, neu, u, [], u, [], n_samples, walks, 5 * eps, eps, pts, exact=u,
                         seed=seed)


def tunnel_mixed_3d(n_samples: int = 65536, walks: int = 32, n_points: int = 200000, n_box: int = 8,
                    subdiv: int = 5, seed: int = 0) -> MixedWorkload:
    """A 3D mixed channel problem (a wind-tunnel-like setting): the box [-2,2] x [-1,1]^2 with an ellipsoidal obstacle
    (semi-axes 0.5, 0.35, 0.35 at the origin, icosphere subdivision 5: 20,480
    triangles, wound inward); Dirichlet on the inlet and outlet faces x = -2,
    2, Neumann on the four walls and the obstacle.  Manufactured harmonic
    u* = x + 0.3 x y + 0.2 (y^2 - z^2): g = u*, h = n . grad u*.  65,536
    samples x 32 walks; 200,000 uniform points in the domain at least 0.02
    from the boundary.  eps = 1e-3 x bbox diagonal, l = 5 eps.  Walks use a
    silhouette gap of 1/8 (star radii within 7/8 of the exact ones): from a
    point in the channel the obstacle's whole contour is nearly equidistant,
    so the exact closest-silhouette search visits all of it."""
    lo, hi = (-2.0, -1.0, -1.0), (2.0, 1.0, 1.0)
    ax = (0.5, 0.35, 0.35)
    V, F = box_with_obstacles(lo, hi, n_box=n_box, ellipsoids=[((0.0, 0.0, 0.0), ax)], subdiv=subdiv)
    mid = element_midpoints(V, F)
    neu = ~((np.abs(mid[:, 0] - lo[0]) < 1e-6) | (np.abs(mid[:, 0] - hi[0]) < 1e-6))
    u = [(POLY, poly3d_coeffs({(1, 0, 0): 1.0, (1, 1, 0): 0.3, (0, 2, 0): 0.2, (0, 0, 2): -0.2}))]
    rng = np.random.default_rng(seed)
    pts = []
    while sum(len(q) for q in pts) < n_points:
        q = rng.uniform(lo, hi, (2 * n_points, 3))
        pts.append(q[in_domain_box_obstacles(q, lo, hi, [((0.0, 0.0, 0.0), ax)], 0.02)])
    pts = np.concatenate(pts)[:n_points].astype(np.float32)
    eps = 1e-3 * bbox_diagonal(V)
    return MixedWorkload("tunnel_mixed_3d", 3, V, F, neu.astype(np.uint8), u, [], u, [], n_samples, walks, 5 * eps,
                         eps, pts, exact=u, seed=seed, meta={"silhouette_gap": 0.125})
