"""FP64 CPU oracle for Boundary Value Caching (Miller et al., SIGGRAPH 2023).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
product (``paper_2302_11825_gb300``) never imports, loads or calls it, and it
imports nothing from the product: the two sides meet only through the seeded
input generators in ``paper_2302_11825_gb300.workloads``.

The arithmetic lives in ``bvc_oracle.c`` (plain C, double precision); this
module compiles it with gcc on first use and wraps it with ctypes.  Each
function cites the passage of the paper it follows.

Parity status: every function here is pinned by tests in ``tests/`` against
closed forms, a deterministic Green's-identity quadrature, brute force, the
mean-value property or published known answers, except as noted:
  (none: ``sample_source2d`` is pinned by the exact polygon area and the
  closed-form Newtonian potential of a disk, see tests/test_oracle_sampling.py;
  the offset boundary of Sec. 3.2 (``offset_disp``, ``offset_vertices``, the
  samplers) by Green's representation formula over the moved mesh, crossing
  signs of rays, distances to the elements' lines and the offset region's
  area, see tests/test_oracle_offset.py; the screened source weights of a
  walk step (``screened_step_weights``, reading of Eq. 1 with sigma > 0) by
  their sigma -> 0 limit, two closed-form integrals over the ball and walk
  means against a closed-form solution, see tests/test_oracle_screened.py;
  the screened walk on stars (``ball_green_sigma``, ``star_kernel_sigma``,
  ``Wost.walks(sigma=...)``) by the radial equation and boundary value of
  the ball's Green's function, its unit flux at the centre, Green's
  identity on a sphere inside the ball for e^(a.x), the sigma -> 0 limits
  and walk means against closed-form solutions with Neumann data, see
  tests/test_oracle_wost_screened.py)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bvc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TAG_WALK = 0
TAG_BOUNDARY = 1
TAG_SOURCE = 2
TAG_POINTWISE = 3


def build(force: bool = False) -> str:
    """Compile ``bvc_oracle.c`` into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i64, i32, u64, u32, f64 = C.c_int64, C.c_int32, C.c_uint64, C.c_uint32, C.c_double
            sig = {
                "orc_philox4x32_10": (None, [P, P, P]),
                "orc_u01": (f64, [u32]),
                "orc_fn_eval": (f64, [P, C.c_int, P]),
                "orc_green": (None, [C.c_int, P, P, P, P]),
                "orc_closest_brute64": (None, [C.c_int, P, i64, P, i64, P, i64, P, P, P]),
                "orc_closest_brute32": (None, [C.c_int, P, i64, P, i64, P, i64, P, P]),
                "orc_inside2d_f32": (None, [P, P, i64, P, i64, P]),
                "orc_bvh_create": (P, [C.c_int, P, i64, P, i64]),
                "orc_bvh_free": (None, [P]),
                "orc_bvh_closest": (None, [P, P, i64, P, P, P]),
                "orc_boundary_measure": (f64, [C.c_int, P, P, i64]),
                "orc_sample_boundary": (None, [C.c_int, P, i64, P, i64, i64, f64, u64, P, P, P, P]),
                "orc_offset_disp": (f64, [C.c_int, P, i64, P, i64, P, P]),
                "orc_offset_vertices": (None, [C.c_int, P, i64, P, f64, P]),
                "orc_walks": (None, [P, P, P, P, i64, i32, f64, i32, u64, u64, u32, P, P, P, P, P, P]),
                "orc_walks_vg": (None, [P, P, P, P, P, i64, i32, f64, i32, u64, u64, u32, P, P, P, P, P, P]),
                "orc_vertex_interp": (f64, [P, P, i64, P]),
                "orc_winding3d": (f64, [P, P, i64, P]),
                "orc_bessel_i": (f64, [C.c_int, f64]),
                "orc_ray_hits": (C.c_int, [C.c_int, P, P, i64, f64, P, P, P, f64, P, P, P]),
                "orc_clamp_correction": (i64, [P, P, P, f64, P, P, i64, f64, P, i64, f64, i32, i32, f64, i32, u64, P]),
                "orc_bessel_k": (f64, [C.c_int, f64]),
                "orc_green_sigma": (None, [C.c_int, f64, P, P, P, P]),
                "orc_screened_factors": (None, [C.c_int, f64, P, P]),
                "orc_screened_step_weights": (None, [C.c_int, f64, f64, f64, P, P]),
                "orc_walks_sigma": (None, [P, P, P, P, f64, P, i64, i32, f64, i32, u64, u64, u32, P, P, P, P, P, P]),
                "orc_gather_sigma": (None, [C.c_int, f64, i64, P, P, P, P, f64, i64, P, P, i64, P, P, P, P, P, P]),
                "orc_gather_full": (None, [C.c_int, f64, f64, i64, P, P, P, P, f64, P, i64, P, P, i64, P, P, P, P,
                                           P, P]),
                "orc_sample_source3d": (i64, [P, i64, P, i64, i32, i32, i32, u64, P, P, P, P, P]),
                "orc_reduce_walks": (None, [C.c_int, i64, i32, P, P, P, P, P]),
                "orc_sample_source2d": (i64, [P, i64, P, i64, i32, i32, u64, P, P, P, P]),
                "orc_gather": (None, [C.c_int, i64, P, P, P, P, f64, i64, P, P, i64, P, P, P, P, P, P]),
                "orc_sphere_step": (None, [C.c_int, f64, f64, f64, f64, P, P, P, P]),
                "orc_num_threads": (C.c_int, []),
                "orc_set_num_threads": (None, [C.c_int]),
                "orc_sample_boundary_mixed": (None, [C.c_int, P, i64, P, i64, i64, f64, u64, P, P, P, P, P]),
                "orc_fn_grad": (None, [P, C.c_int, P, P]),
                "orc_neumann_eval": (f64, [P, P, C.c_int, P, P]),
                "orc_wost_create": (P, [C.c_int, P, i64, P, i64, P]),
                "orc_wost_free": (None, [P]),
                "orc_wost_counts": (i64, [P, P]),
                "orc_wost_walks": (None, [P, P, P, P, P, P, P, i64, i32, f64, i32, u64, u64, u32, P, P, P, P]),
                "orc_wost_walks_sigma": (None, [P, P, P, P, P, f64, P, P, i64, i32, f64, i32, u64, u64, u32, P, P,
                                                P, P]),
                "orc_ball_green_sigma": (f64, [C.c_int, f64, f64, f64]),
                "orc_star_kernel_sigma": (f64, [C.c_int, f64, f64, f64]),
                "orc_wost_query": (None, [P, P, i64, P, P]),
                "orc_wost_rays": (None, [P, P, P, P, i64, f64, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later parallel loops."""
    _load().orc_set_num_threads(int(n))


# ---------------------------------------------------------------- Philox
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox-4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(r: int) -> float:
    """Uniform in (0,1) from one 32-bit word: (2*(r>>9)+1) * 2^-24."""
    return float(_load().orc_u01(int(r) & 0xFFFFFFFF))


# ---------------------------------------------------------------- functions
def encode_function(terms) -> np.ndarray:
    """[(kind, coeffs), ...] -> flat array [n_terms, kind, n, coeffs..., ...]."""
    out = [float(len(terms))]
    for kind, coeffs in terms:
        coeffs = [float(c) for c in np.asarray(coeffs, dtype=np.float64).ravel()]
        out += [float(kind), float(len(coeffs))] + coeffs
    return np.asarray(out, dtype=np.float64)


def fn_eval(terms, dim: int, x) -> np.ndarray:
    """Evaluate a problem function (g or f of Eq. 1) at points x[n, dim]."""
    lib = _load()
    spec = encode_function(terms)
    x = _f64(np.atleast_2d(x))
    return np.array([lib.orc_fn_eval(_p(spec), dim, _p(x[i])) for i in range(x.shape[0])])


# ---------------------------------------------------------------- Green's functions
def green(dim: int, x, y, ny) -> np.ndarray:
    """App. A: [G, dG/dx (dim), dG/dn_y, d2G/dx dn_y (dim)] for one pair."""
    lib = _load()
    out = np.zeros(2 + 2 * dim)
    lib.orc_green(dim, _p(_f64(x)), _p(_f64(y)), _p(_f64(ny)), _p(out))
    return out


def green_sigma(dim: int, sigma: float, x, y, ny) -> np.ndarray:
    """Screened App. A Green's function and derivatives (layout as green)."""
    lib = _load()
    out = np.zeros(2 + 2 * dim)
    lib.orc_green_sigma(dim, float(np.sqrt(sigma)), _p(_f64(x)), _p(_f64(y)), _p(_f64(ny)), _p(out))
    return out


def bessel_i(n: int, t: float) -> float:
    return _load().orc_bessel_i(int(n), float(t))


def bessel_k(n: int, t: float) -> float:
    return _load().orc_bessel_k(int(n), float(t))


def screened_factors(dim: int, t: float):
    """(C, Qg) of a ball with t = R sqrt(sigma)."""
    C_, Q_ = C.c_double(), C.c_double()
    _load().orc_screened_factors(int(dim), float(t), C.byref(C_), C.byref(Q_))
    return C_.value, Q_.value


def screened_step_weights(dim: int, sigma: float, R: float, rho: float):
    """(w_u, w_g) of a screened step's source sample at radius rho in the ball
    of radius R: minus |S| R rho^(d-1) times the ball's Green's function of
    (sigma - Delta) and of its centre gradient's radial mode."""
    wu, wg = C.c_double(), C.c_double()
    _load().orc_screened_step_weights(int(dim), float(np.sqrt(sigma)), float(R), float(rho), C.byref(wu),
                                      C.byref(wg))
    return wu.value, wg.value


def ball_green_sigma(dim: int, sigma: float, R: float, rho: float) -> float:
    """The Green's function of (sigma - Delta) on the ball of radius R that
    vanishes on its sphere, seen from the centre at distance rho (sigma = 0:
    the Laplace ball's)."""
    return _load().orc_ball_green_sigma(int(dim), float(np.sqrt(sigma)), float(R), float(rho))


def star_kernel_sigma(dim: int, sigma: float, R: float, r: float) -> float:
    """Throughput factor W(r) = -|S| r^(d-1) G'(r) of a screened walk-on-stars
    step whose direction first meets the boundary at distance r (1 for
    sigma = 0)."""
    return _load().orc_star_kernel_sigma(int(dim), float(np.sqrt(sigma)), float(R), float(r))


# ---------------------------------------------------------------- geometry
def closest_brute64(V, F, pts):
    lib = _load()
    V, F, pts = _f32(V), _i32(F), _f64(pts)
    dim = V.shape[1]
    n = pts.shape[0]
    dist, prim, cp = np.zeros(n), np.zeros(n, np.int32), np.zeros((n, dim))
    lib.orc_closest_brute64(dim, _p(V), V.shape[0], _p(F), F.shape[0], _p(pts), n, _p(dist), _p(prim), _p(cp))
    return dist, prim, cp


def closest_brute32(V, F, pts):
    """Canonical FP32 brute force: (squared distance, primitive index)."""
    lib = _load()
    V, F, pts = _f32(V), _i32(F), _f32(pts)
    dim = V.shape[1]
    n = pts.shape[0]
    d2, prim = np.zeros(n, np.float32), np.zeros(n, np.int32)
    lib.orc_closest_brute32(dim, _p(V), V.shape[0], _p(F), F.shape[0], _p(pts), n, _p(d2), _p(prim))
    return d2, prim


def inside2d_f32(V, F, pts) -> np.ndarray:
    lib = _load()
    V, F, pts = _f32(V), _i32(F), _f32(pts)
    out = np.zeros(pts.shape[0], np.int32)
    lib.orc_inside2d_f32(_p(V), _p(F), F.shape[0], _p(pts), pts.shape[0], _p(out))
    return out


class BVH:
    """The oracle's own FP64 median-split BVH over a polygon/triangle mesh."""

    def __init__(self, V, F):
        self._lib = _load()
        self.V, self.F = _f32(V), _i32(F)
        self.dim = self.V.shape[1]
        self.h = self._lib.orc_bvh_create(self.dim, _p(self.V), self.V.shape[0], _p(self.F), self.F.shape[0])

    def closest(self, pts):
        pts = _f64(pts)
        n = pts.shape[0]
        dist, prim, cp = np.zeros(n), np.zeros(n, np.int32), np.zeros((n, self.dim))
        self._lib.orc_bvh_closest(self.h, _p(pts), n, _p(dist), _p(prim), _p(cp))
        return dist, prim, cp

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.orc_bvh_free(self.h)
            self.h = None


def boundary_measure(V, F) -> float:
    V, F = _f32(V), _i32(F)
    return float(_load().orc_boundary_measure(V.shape[1], _p(V), _p(F), F.shape[0]))


def offset_disp(V, F, fixed=None):
    """Sec. 3.2: per-vertex inward displacement directions m_v of the offset
    boundary (the closed surface of the mesh with vertex v moved to
    v - l m_v) and their largest length (the reach).  fixed: optional per-
    element flags of elements that are not moved."""
    lib = _load()
    V, F = _f32(V), _i32(F)
    dim = V.shape[1]
    m = np.zeros((V.shape[0], dim))
    fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
    reach = lib.orc_offset_disp(dim, _p(V), V.shape[0], _p(F), F.shape[0], _p(fx), _p(m))
    return m, float(reach)


def offset_vertices(V, F, l: float, fixed=None) -> np.ndarray:
    """The offset boundary's vertices, fl32(V - l m) (Sec. 3.2)."""
    lib = _load()
    V = _f32(V)
    m, _ = offset_disp(V, F, fixed)
    out = np.zeros_like(V)
    lib.orc_offset_vertices(V.shape[1], _p(V), V.shape[0], _p(m), float(l), _p(out))
    return out


def sample_boundary(V, F, N: int, l: float, seed: int):
    """Sec. 4 Sampling + Sec. 3.2 offset boundary: (z[N,dim], n[N,dim],
    element[N], jac[N]) in FP64; 1/p of sample i is |dOmega| jac[i]."""
    lib = _load()
    V, F = _f32(V), _i32(F)
    dim = V.shape[1]
    z, n, e, j = np.zeros((N, dim)), np.zeros((N, dim)), np.zeros(N, np.int32), np.zeros(N)
    lib.orc_sample_boundary(dim, _p(V), V.shape[0], _p(F), F.shape[0], N, float(l), int(seed), _p(z), _p(n), _p(j),
                            _p(e))
    return z, n, e, j


def sphere_step(dim: int, R: float, u0: float, u1: float, u2: float):
    """Sec. 3.1 step: (direction w, source radius rho, w_u, w_g) for ball radius R."""
    lib = _load()
    om = np.zeros(3)
    rho, wu, wg = C.c_double(), C.c_double(), C.c_double()
    lib.orc_sphere_step(dim, float(R), float(u0), float(u1), float(u2), _p(om), C.byref(rho), C.byref(wu),
                        C.byref(wg))
    return om[:dim].copy(), rho.value, wu.value, wg.value


def walks(bvh: BVH, g_terms, f_terms, starts, W: int, eps: float, max_steps: int, seed: int,
          id_base: int = 0, tag: int = TAG_WALK, want_pend: bool = False, g_vertex=None, sigma: float = 0.0):
    """Sec. 3.1 / Eq. 7: W walks from each FP32 start point.

    g_vertex: optional per-vertex values of g (then g_terms is ignored): g at
    a boundary point is interpolated linearly on the closest element.
    sigma > 0: the screened equation (Delta - sigma) u = f, each step's
    source term weighted by the ball's screened Green's function and by the
    throughput of the balls before it.
    Returns dict with per-walk U, grad[.., dim], steps, prim, scale[.., 2]
    (magnitudes of the terms forming U and the gradient, for error scaling)
    and, if asked, pend (final closest point)."""
    lib = _load()
    starts = _f32(starts)
    n, dim = starts.shape
    T = n * W
    U, grad = np.zeros(T), np.zeros((T, dim))
    steps, prim = np.zeros(T, np.int32), np.zeros(T, np.int32)
    pend = np.zeros((T, dim)) if want_pend else None
    scale = np.zeros((T, 2))
    g = encode_function(g_terms if g_vertex is None else [])
    f = encode_function(f_terms)
    gv = None if g_vertex is None else _f64(g_vertex)
    lib.orc_walks_sigma(bvh.h, _p(g), _p(gv), _p(f), float(np.sqrt(sigma)), _p(starts), n, int(W), float(eps),
                        int(max_steps), int(seed), int(id_base), int(tag), _p(U), _p(grad), _p(steps), _p(prim),
                        _p(pend), _p(scale))
    out = {"U": U, "grad": grad, "steps": steps, "prim": prim, "scale": scale}
    if want_pend:
        out["pend"] = pend
    return out


def vertex_interp(bvh: BVH, gv, elem, pts):
    """g from vertex values at points lying on the given elements."""
    lib = _load()
    gv = _f64(gv)
    pts = _f64(pts)
    return np.array([lib.orc_vertex_interp(bvh.h, _p(gv), int(e), _p(np.ascontiguousarray(p)))
                     for e, p in zip(elem, pts)])


MAX_HITS = 8


def ray_hits(V, F, l: float, x, om, rmax: float):
    """Crossings of the ray x + t om (0 < t <= rmax) with the offset
    boundary at l (the mesh with its vertices moved by -l m_v, Sec. 3.2):
    (t, element, n.om), nearest first."""
    lib = _load()
    V, F = _f32(V), _i32(F)
    m = offset_disp(V, F)[0] if l != 0.0 else None
    t, nw = np.zeros(MAX_HITS), np.zeros(MAX_HITS)
    e = np.zeros(MAX_HITS, np.int64)
    k = lib.orc_ray_hits(V.shape[1], _p(V), _p(F), F.shape[0], float(l), _p(m), _p(_f64(x)), _p(_f64(om)),
                         float(rmax), _p(t), _p(e), _p(nw))
    return t[:k], e[:k], nw[:k]


def clamp_correction(bvh: BVH, g_terms, Vs, Fs, l: float, pts, c: float, n_dirs: int, W: int, eps: float,
                     seed: int, max_steps: int = 1 << 14, g_vertex=None, sigma: float = 0.0):
    """Sec. 3.3: the estimate of int [dG/dn - clamp_c(dG/dn)] u dz per point
    (rays against the sample surface Vs, Fs moved by -l n_e; walks on bvh).
    Returns (u_corr, number of contributing hits)."""
    lib = _load()
    pts = _f64(pts)
    Vs, Fs = _f32(Vs), _i32(Fs)
    out = np.zeros(pts.shape[0])
    g = encode_function(g_terms if g_vertex is None else [])
    gv = None if g_vertex is None else _f64(g_vertex)
    n = lib.orc_clamp_correction(bvh.h, _p(g), _p(gv), float(np.sqrt(sigma)), _p(Vs), _p(Fs), Fs.shape[0], float(l),
                                 _p(pts), pts.shape[0], float(c), int(n_dirs), int(W), float(eps), int(max_steps),
                                 int(seed), _p(out))
    return out, int(n)


def reduce_walks(U, grad, nrm, W: int):
    """Alg. 1: u^ and du/dn^ per sample as means over its W walks."""
    lib = _load()
    U, grad = _f64(U), _f64(grad)
    dim = grad.shape[1]
    n = U.shape[0] // W
    nrm_a = None if nrm is None else _f32(nrm)
    u_hat = np.zeros(n)
    q_hat = np.zeros(n) if nrm is not None else None
    lib.orc_reduce_walks(dim, n, int(W), _p(U), _p(grad), _p(nrm_a), _p(u_hat), _p(q_hat))
    return u_hat, q_hat


def winding3d(V, F, pts):
    """Generalized winding number of a triangle mesh at each point."""
    lib = _load()
    V, F = _f32(V), np.ascontiguousarray(F, dtype=np.int32)
    return np.array([lib.orc_winding3d(_p(V), _p(F), F.shape[0], _p(np.ascontiguousarray(p, dtype=np.float64)))
                     for p in np.atleast_2d(pts)])


def sample_source3d(V, F, grid, seed: int, f_terms, want_winding=False, l: float = 0.0):
    """Sec. 4 Sampling in 3D: jittered grid over the bounding box, kept where
    the winding number of the offset boundary at l (Sec. 3.2; l = 0: the
    mesh) exceeds 1/2.  Returns (y [kept][3], c [kept], ncand) and, if
    asked, every candidate's winding number."""
    lib = _load()
    V, F = _f32(V), np.ascontiguousarray(F, dtype=np.int32)
    Vin = offset_vertices(V, F, l) if l != 0.0 else None
    ncand = int(grid[0]) * int(grid[1]) * int(grid[2])
    y = np.zeros((ncand, 3), np.float32)
    c = np.zeros(ncand)
    wn = np.zeros(ncand) if want_winding else None
    f = encode_function(f_terms)
    k = lib.orc_sample_source3d(_p(V), V.shape[0], _p(F), F.shape[0], int(grid[0]), int(grid[1]), int(grid[2]),
                                int(seed), _p(f), _p(Vin), _p(y), _p(c), _p(wn))
    out = (y[:k], c[:k], ncand)
    return out + (wn,) if want_winding else out


def sample_source2d(V, F, grid, seed: int, f_terms, l: float = 0.0):
    """Sec. 4 Sampling: jittered grid over the bounding box, kept if inside
    the offset boundary at l (Sec. 3.2; l = 0: the polygon itself).

    Returns (y[kept,2] FP32, c[kept] = f(y)|box| FP64, n_candidates)."""
    lib = _load()
    V, F = _f32(V), _i32(F)
    Vin = offset_vertices(V, F, l) if l != 0.0 else None
    G0, G1 = int(grid[0]), int(grid[1])
    y = np.zeros((G0 * G1, 2), np.float32)
    c = np.zeros(G0 * G1)
    f = encode_function(f_terms)
    kept = lib.orc_sample_source2d(_p(V), V.shape[0], _p(F), F.shape[0], G0, G1, int(seed), _p(f), _p(Vin), _p(y),
                                   _p(c))
    return y[:kept].copy(), c[:kept].copy(), G0 * G1


def gather(z, nz, u_hat, q_hat, bnd_measure: float, x, y=None, c=None, want_abs: bool = False, sigma: float = 0.0,
           clamp_c: float = 0.0, jac=None):
    """Eq. 3-6 / Alg. 1 splat: FP64 running sums (u_bnd, u_src, g_bnd, g_src).
    jac: per-sample measure ratios of the offset boundary (1/p = bnd_measure
    jac[i]); None = 1.
    sigma > 0: with the screened Green's functions of App. A.
    clamp_c > 0: dG/dn of the u term clamped to [-c, c] (Sec. 3.3).

    With want_abs, also the per-point sums of |term| (for error scaling):
    array [M, 2 + 2 dim] = [u_bnd, g_bnd(dim), u_src, g_src(dim)]."""
    lib = _load()
    z, nz, x = _f64(z), _f64(nz), _f64(x)
    dim = x.shape[1]
    N, M = z.shape[0], x.shape[0]
    u_hat, q_hat = _f64(u_hat), _f64(q_hat)
    if y is None:
        y = np.zeros((0, dim))
        c = np.zeros(0)
    y, c = _f64(y), _f64(c)
    ub, us = np.zeros(M), np.zeros(M)
    gb, gs = np.zeros((M, dim)), np.zeros((M, dim))
    ab = np.zeros((M, 2 + 2 * dim)) if want_abs else None
    jac = None if jac is None else _f64(jac)
    lib.orc_gather_full(dim, float(np.sqrt(sigma)), float(clamp_c), N, _p(z), _p(nz), _p(u_hat), _p(q_hat),
                        float(bnd_measure), _p(jac), y.shape[0], _p(y), _p(c), M, _p(x), _p(ub), _p(us), _p(gb), _p(gs),
                        _p(ab))
    if want_abs:
        return ub, us, gb, gs, ab
    return ub, us, gb, gs


# ---------------------------------------------------------------- mixed boundaries
def sample_boundary_mixed(V, F, N: int, l: float, seed: int, neumann):
    """Sec. 3.2 for a mixed boundary: samples on the Dirichlet elements of
    the offset boundary built from the Dirichlet elements alone, samples on
    Neumann elements left on the boundary (jac 1).  Returns (z, n, e, jac)."""
    lib = _load()
    V, F = _f32(V), _i32(F)
    dim = V.shape[1]
    nf = np.ascontiguousarray(neumann, dtype=np.uint8)
    z, n, e, j = np.zeros((N, dim)), np.zeros((N, dim)), np.zeros(N, np.int32), np.zeros(N)
    lib.orc_sample_boundary_mixed(dim, _p(V), V.shape[0], _p(F), F.shape[0], N, float(l), int(seed), _p(nf), _p(z),
                                  _p(n), _p(j), _p(e))
    return z, n, e, j


def fn_grad(terms, dim: int, x) -> np.ndarray:
    """Gradient of a problem function at points x[n, dim]."""
    lib = _load()
    spec = encode_function(terms)
    x = _f64(np.atleast_2d(x))
    out = np.zeros((x.shape[0], dim))
    for i in range(x.shape[0]):
        lib.orc_fn_grad(_p(spec), dim, _p(x[i]), _p(out[i]))
    return out


def neumann_eval(h_value, h_potential, dim: int, z, n) -> np.ndarray:
    """Neumann data h(z) = h_value(z) + n . grad h_potential(z)."""
    lib = _load()
    hv, hp = encode_function(h_value), encode_function(h_potential)
    z, n = _f64(np.atleast_2d(z)), _f64(np.atleast_2d(n))
    return np.array([lib.orc_neumann_eval(_p(hv), _p(hp), dim, _p(z[i]), _p(n[i])) for i in range(z.shape[0])])


class Wost:
    """Walk on stars (Sec. 3.1) on a boundary whose elements are flagged
    Neumann (1) or Dirichlet (0): the oracle's brute-force silhouette and ray
    queries and its walks."""

    def __init__(self, V, F, neumann):
        self._lib = _load()
        self.V, self.F = _f32(V), _i32(F)
        self.dim = self.V.shape[1]
        self.neumann = np.ascontiguousarray(neumann, dtype=np.uint8)
        self.h = self._lib.orc_wost_create(self.dim, _p(self.V), self.V.shape[0], _p(self.F), self.F.shape[0],
                                           _p(self.neumann))

    def counts(self):
        """(Dirichlet elements, Neumann elements, silhouette candidates)."""
        out = np.zeros(3, np.int64)
        self._lib.orc_wost_counts(self.h, _p(out))
        return tuple(int(v) for v in out)

    def query(self, pts):
        """Distances to the Dirichlet part and to the closest silhouette."""
        pts = _f64(pts)
        n = pts.shape[0]
        dd, ds = np.zeros(n), np.zeros(n)
        self._lib.orc_wost_query(self.h, _p(pts), n, _p(dd), _p(ds))
        return dd, ds

    def rays(self, org, dirs, tmax: float, skip=None):
        """First crossing (t, element) of each ray with the Neumann part."""
        org, dirs = _f64(org), _f64(dirs)
        n = org.shape[0]
        sk = None if skip is None else _i32(skip)
        t, e = np.zeros(n), np.zeros(n, np.int32)
        self._lib.orc_wost_rays(self.h, _p(org), _p(dirs), _p(sk), n, float(tmax), _p(t), _p(e))
        return t, e

    def walks(self, g_terms, h_value, h_potential, f_terms, starts, start_elem, W: int, eps: float,
              max_steps: int, seed: int, id_base: int = 0, tag: int = TAG_WALK, sigma: float = 0.0):
        """W walks from each FP32 start; start_elem[i] >= 0 puts start i on
        that Neumann element.  Returns per-walk U, grad[.., dim], steps and
        the Dirichlet element of the end.  sigma > 0: the screened equation
        (Delta - sigma) u = f (each step's throughput factor W(r), the ball's
        screened Green's function in the Neumann and source terms)."""
        starts = _f32(starts)
        n, dim = starts.shape
        T = n * W
        U, grad = np.zeros(T), np.zeros((T, dim))
        steps, prim = np.zeros(T, np.int32), np.zeros(T, np.int32)
        se = None if start_elem is None else _i32(start_elem)
        g, hv, hp, f = (encode_function(t) for t in (g_terms, h_value, h_potential, f_terms))
        self._lib.orc_wost_walks_sigma(self.h, _p(g), _p(hv), _p(hp), _p(f), float(np.sqrt(sigma)), _p(starts),
                                       _p(se), n, int(W), float(eps), int(max_steps), int(seed), int(id_base),
                                       int(tag), _p(U), _p(grad), _p(steps), _p(prim))
        return {"U": U, "grad": grad, "steps": steps, "prim": prim}

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.orc_wost_free(self.h)
            self.h = None
