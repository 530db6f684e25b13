"""Thin ctypes binding of ``libbvc.so`` (C ABI in ``include/bvc.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory (tensors) and streams.  The
library is loaded from ``paper_2302_11825_gb300/_build/libbvc.so``; if it is
missing it is built with nvcc, and if that is impossible the first call
raises -- there is no CPU fallback.

Point arrays are structure-of-arrays tensors of shape ``(dim, count)``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_DEGENERATE_MESH, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_WORKSPACE, \
    WARN_WALK_CAP, ERR_BOUNDS = range(10)
FN_POLY, FN_GAUSS, FN_GAUSS_LAPLACIAN, FN_EXP_TRIG = 1, 2, 3, 4
MAX_TERMS = 4
TAG_WALK, TAG_BOUNDARY, TAG_SOURCE, TAG_POINTWISE = 0, 1, 2, 3


class BvcError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class Term(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_coeffs", C.c_int32), ("coeffs", C.POINTER(C.c_double))]


class Function(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("terms", Term * MAX_TERMS)]


class GeometryInfo(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_verts", C.c_int64), ("n_prims", C.c_int64), ("n_nodes", C.c_int64),
                ("boundary_measure", C.c_double), ("bbox_lo", C.c_float * 3), ("bbox_hi", C.c_float * 3),
                ("device_bytes", C.c_size_t), ("offset_reach", C.c_double)]


class CacheStruct(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int64), ("z", C.c_void_p), ("nrm", C.c_void_p), ("jac", C.c_void_p),
                ("u_hat", C.c_void_p), ("dudn_hat", C.c_void_p), ("packed", C.c_void_p),
                ("bnd_measure", C.c_double), ("n_src_cand", C.c_int64), ("src_y", C.c_void_p),
                ("src_c", C.c_void_p), ("src_packed", C.c_void_p), ("n_src_dev", C.c_void_p),
                ("sigma", C.c_double), ("clamp_c", C.c_double)]


class CacheOpts(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("walks_per_sample", C.c_int32), ("max_steps", C.c_int32),
                ("offset_l", C.c_double), ("eps", C.c_double), ("seed", C.c_uint64),
                ("walk_id_base", C.c_uint64), ("src_grid", C.c_int32 * 3), ("sigma", C.c_double),
                ("clamp_c", C.c_double), ("reuse_sources", C.c_int32)]


class MultiCacheStruct(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int64), ("k", C.c_int32), ("z", C.c_void_p), ("nrm", C.c_void_p),
                ("jac", C.c_void_p), ("mom_u", C.c_void_p), ("mom_q", C.c_void_p), ("u_hat", C.c_void_p), ("dudn_hat", C.c_void_p),
                ("packed", C.c_void_p), ("bnd_measure", C.c_double), ("n_bumps", C.c_int32), ("mom_su", C.c_void_p),
                ("mom_sq", C.c_void_p), ("n_src_cand", C.c_int64), ("src_y", C.c_void_p), ("src_psi", C.c_void_p),
                ("n_src_dev", C.c_void_p)]


class BatchMeshStruct(C.Structure):
    _fields_ = [("geom", C.c_void_p), ("n_samples", C.c_int64), ("offset_l", C.c_double), ("eps", C.c_float),
                ("n_points", C.c_int64)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


class EvalStateStruct(C.Structure):
    _fields_ = [("dim", C.c_int32), ("m", C.c_int64), ("x", C.c_void_p), ("u_bnd", C.c_void_p),
                ("u_src", C.c_void_p), ("grad_bnd", C.c_void_p), ("grad_src", C.c_void_p),
                ("counts", C.c_void_p)]


class NeumannStruct(C.Structure):
    _fields_ = [("value", Function), ("potential", Function)]


class MixedInfo(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_dirichlet", C.c_int64), ("n_neumann", C.c_int64),
                ("n_silhouette", C.c_int64), ("n_silhouette_tree", C.c_int64),
                ("dirichlet_measure", C.c_double), ("neumann_measure", C.c_double),
                ("device_bytes", C.c_size_t)]


def _declare(lib):
    P, i32, i64, u32, u64, f32, f64, sz = (C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float,
                                          C.c_double, C.c_size_t)
    S = C.c_int
    sig = {
        "bvc_geometry_create": (S, [i32, P, i64, P, i64, P, C.POINTER(C.c_void_p)]),
        "bvc_geometry_destroy": (S, [P]),
        "bvc_geometry_get_info": (S, [P, C.POINTER(GeometryInfo)]),
        "bvc_geometry_stats": (S, [P, C.POINTER(C.c_uint64), i32, P]),
        "bvc_query_closest": (S, [P, P, i64, P, P, P, P]),
        "bvc_classify_near": (S, [P, P, i64, f32, P, P]),
        "bvc_sample_boundary": (S, [P, i64, f64, u64, P, P, P, P, P]),
        "bvc_walk": (S, [P, C.POINTER(Function), C.POINTER(Function), P, P, i64, i32, f32, i32, u64, u64, u32, P, P,
                         P, P]),
        "bvc_reduce_walks": (S, [P, i64, i32, i32, i32, P, P]),
        "bvc_sample_source_workspace_size": (S, [i64, C.POINTER(sz)]),
        "bvc_sample_source": (S, [P, C.POINTER(Function), C.POINTER(C.c_int32), u64, f64, C.POINTER(CacheStruct), P,
                                  sz, P]),
        "bvc_cache_pack": (S, [C.POINTER(CacheStruct), P]),
        "bvc_cache_build_workspace_size": (S, [P, C.POINTER(CacheOpts), C.POINTER(sz), C.POINTER(sz)]),
        "bvc_cache_build": (S, [P, C.POINTER(Function), C.POINTER(Function), C.POINTER(CacheOpts),
                                C.POINTER(CacheStruct), P, sz, P]),
        "bvc_cache_build_vg": (S, [P, P, C.POINTER(Function), C.POINTER(CacheOpts), C.POINTER(CacheStruct), P, sz,
                                   P]),
        "bvc_evaluate_adjoint_workspace_size": (S, [i64, C.POINTER(sz)]),
        "bvc_evaluate_adjoint": (S, [C.POINTER(CacheStruct), P, i64, P, P, P, P, P, sz, P]),
        "bvc_cache_adjoint_workspace_size": (S, [P, C.POINTER(CacheOpts), C.POINTER(sz), C.POINTER(sz)]),
        "bvc_cache_adjoint": (S, [P, C.POINTER(Function), C.POINTER(CacheOpts), C.POINTER(CacheStruct), P, P, P, P,
                                  P, P, sz, P]),
        "bvc_evaluate_workspace_size": (S, [C.POINTER(CacheStruct), C.POINTER(EvalStateStruct), C.POINTER(sz)]),
        "bvc_evaluate": (S, [C.POINTER(CacheStruct), C.POINTER(EvalStateStruct), P, sz, P]),
        "bvc_get_solution": (S, [C.POINTER(EvalStateStruct), P, P, P]),
        "wos_estimate_workspace_size": (S, [i32, i64, i32, C.POINTER(sz), C.POINTER(sz)]),
        "wos_estimate": (S, [P, C.POINTER(Function), C.POINTER(Function), C.POINTER(EvalStateStruct), i32, f32, i32,
                             u64, u64, P, sz, P]),
        "bvc_eval_state_reset": (S, [C.POINTER(EvalStateStruct), P]),
        "bvc_tune_gather": (S, [C.POINTER(CacheStruct), C.POINTER(EvalStateStruct), P, sz, P,
                                C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
        "bvc_set_gather_shape": (S, [i32, i32, i32]),
        "bvc_last_error": (S, []),
        "wos_estimate_sigma": (S, [P, C.POINTER(Function), C.POINTER(Function), f64, C.POINTER(EvalStateStruct), i32,
                                   f32, i32, u64, u64, P, sz, P]),
        "wos_estimate_static_scratch": (S, [P, C.POINTER(Function), C.POINTER(Function), C.POINTER(EvalStateStruct),
                                            i32, f32, i32, u64, u64, P]),
        "bvc_geometry_set_counting": (S, [P, i32]),
        "bvc_poly_terms": (i32, [i32]),
        "bvc_multi_cache_build_workspace_size": (S, [P, i64, i32, C.POINTER(sz), C.POINTER(sz)]),
        "bvc_multi_cache_build": (S, [P, P, C.POINTER(CacheOpts), C.POINTER(MultiCacheStruct), P, sz, P]),
        "bvc_multi_cache_project": (S, [P, C.POINTER(MultiCacheStruct), P]),
        "bvc_multi_cache_build_source_workspace_size": (S, [P, C.POINTER(CacheOpts), C.POINTER(sz), C.POINTER(sz)]),
        "bvc_multi_cache_build_source": (S, [P, C.POINTER(Function), P, C.POINTER(CacheOpts),
                                             C.POINTER(MultiCacheStruct), P, sz, P]),
        "bvc_evaluate_multi": (S, [C.POINTER(MultiCacheStruct), P, i64, P, P]),
        "bvc_batch_create": (S, [P, i32, i32, i32, i32, P, C.POINTER(C.c_void_p)]),
        "bvc_batch_destroy": (S, [P]),
        "bvc_batch_get_info": (S, [P, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "bvc_batch_build_workspace_size": (S, [P, C.POINTER(sz), C.POINTER(sz)]),
        "bvc_batch_build": (S, [P, P, P, C.POINTER(MultiCacheStruct), P, sz, P]),
        "bvc_batch_set_counting": (S, [P, i32]),
        "bvc_batch_stats": (S, [P, C.POINTER(C.c_uint64), i32, P]),
        "bvc_batch_project": (S, [P, P, C.POINTER(MultiCacheStruct), P]),
        "bvc_batch_evaluate": (S, [P, C.POINTER(MultiCacheStruct), P, P, P]),
        "bvc_cache_build_region": (S, [P, P, C.POINTER(Function), C.POINTER(Function), C.POINTER(CacheOpts),
                                       C.POINTER(CacheStruct), P, sz, P]),
        "bvc_clamp_correction_workspace_size": (S, [i32, i64, i32, i32, C.POINTER(sz)]),
        "bvc_clamp_correction": (S, [P, P, f64, C.POINTER(Function), C.POINTER(Function), f64, f64, P, i64, i32, i32,
                                     f32, i32, u64, P, C.POINTER(C.c_int64), P, sz, P]),
        "bvc_tune_walks_workspace_size": (S, [P, C.POINTER(CacheOpts), C.POINTER(sz)]),
        "bvc_tune_walks": (S, [P, C.POINTER(Function), C.POINTER(Function), C.POINTER(CacheOpts), P, sz, P,
                               C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
        "bvc_geometry_set_walk_shape": (S, [P, i32, i32]),
        "bvc_mixed_create": (S, [i32, P, i64, P, i64, P, P, C.POINTER(C.c_void_p)]),
        "bvc_mixed_destroy": (S, [P]),
        "bvc_mixed_get_info": (S, [P, C.POINTER(MixedInfo)]),
        "bvc_mixed_geometries": (S, [P, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
        "bvc_mixed_set_silhouette_gap": (S, [P, f64]),
        "bvc_mixed_query": (S, [P, P, i64, P, P, P]),
        "bvc_mixed_rays": (S, [P, P, P, P, i64, f32, P, P, P]),
        "bvc_mixed_walk": (S, [P, C.POINTER(Function), C.POINTER(NeumannStruct), C.POINTER(Function), P, P, P, i64,
                               i32, f32, i32, u64, u64, u32, P, P, P, P, P]),
        "bvc_mixed_walk_sigma": (S, [P, C.POINTER(Function), C.POINTER(NeumannStruct), C.POINTER(Function), f64, P,
                                     P, P, i64, i32, f32, i32, u64, u64, u32, P, P, P, P, P]),
        "bvc_mixed_cache_build_workspace_size": (S, [P, C.POINTER(CacheOpts), C.POINTER(sz), C.POINTER(sz)]),
        "bvc_mixed_cache_build": (S, [P, C.POINTER(Function), C.POINTER(NeumannStruct), C.POINTER(Function),
                                      C.POINTER(CacheOpts), C.POINTER(CacheStruct), P, sz, P]),
        "wost_estimate": (S, [P, C.POINTER(Function), C.POINTER(NeumannStruct), C.POINTER(Function),
                              C.POINTER(EvalStateStruct), i32, f32, i32, u64, u64, P, sz, P]),
        "wost_estimate_sigma": (S, [P, C.POINTER(Function), C.POINTER(NeumannStruct), C.POINTER(Function), f64,
                                    C.POINTER(EvalStateStruct), i32, f32, i32, u64, u64, P, sz, P]),
        "bvc_profile_begin": (S, []),
        "bvc_profile_end": (S, [C.POINTER(KernelTime), i32, C.POINTER(C.c_int32)]),
        "bvc_gather_status": (S, [C.POINTER(C.c_uint64), i32]),
        "bvc_wait_selftest": (S, [i64, P]),
        "bvc_status_string": (C.c_char_p, [S]),
        "bvc_version": (i32, []),
        "bvc_debug_build": (i32, []),
        "bvc_debug_set_link": (S, [P, i64, i32, i32, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def lib():
    """The loaded CUDA library (built in-tree on first use).  With the
    environment variable BVC_DEBUG=1 at first use, the debug build
    (libbvc_debug.so: device bounds checks in every BVH traversal)."""
    global _lib
    with _lock:
        if _lib is None:
            debug = os.environ.get("BVC_DEBUG", "0") == "1"
            path = _build.LIB_DEBUG if debug else _build.LIB
            if not os.path.exists(path) or _build._stale(path):
                path = _build.build(debug=debug)
            handle = C.CDLL(path)
            _declare(handle)
            _lib = handle
    return _lib


def library_path() -> str:
    return _build.LIB


def status_string(s: int) -> str:
    return lib().bvc_status_string(int(s)).decode()


def _check(status: int, what: str, allow=(OK,)):
    if status not in allow:
        raise BvcError(status, what)
    return status


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
    return t


def make_function(terms) -> Function:
    """[(kind, coeffs), ...] -> bvc_function (the coefficient arrays are kept
    alive on the returned structure)."""
    f = Function()
    terms = list(terms or [])
    if len(terms) > MAX_TERMS:
        raise ValueError("too many terms")
    f.n_terms = len(terms)
    keep = []
    for i, (kind, coeffs) in enumerate(terms):
        arr = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64).ravel())
        keep.append(arr)
        f.terms[i].kind = int(kind)
        f.terms[i].n_coeffs = int(arr.size)
        f.terms[i].coeffs = arr.ctypes.data_as(C.POINTER(C.c_double))
    f._keep = keep
    return f


def soa(points, device="cuda") -> torch.Tensor:
    """(count, dim) array -> contiguous (dim, count) float32 CUDA tensor."""
    a = np.ascontiguousarray(np.asarray(points, dtype=np.float32).T)
    return torch.from_numpy(a).to(device)


# ---------------------------------------------------------------- geometry
class Geometry:
    """bvc_geometry_create / bvc_geometry_destroy (library-owned BVH)."""

    def __init__(self, V, F, stream=None):
        V = np.ascontiguousarray(V, dtype=np.float32)
        F = np.ascontiguousarray(F, dtype=np.int32)
        self.dim = int(V.shape[1])
        h = C.c_void_p()
        _check(lib().bvc_geometry_create(self.dim, V.ctypes.data_as(C.c_void_p), V.shape[0],
                                         F.ctypes.data_as(C.c_void_p), F.shape[0], _stream(stream), C.byref(h)),
               "bvc_geometry_create")
        self.h = h

    def info(self) -> GeometryInfo:
        inf = GeometryInfo()
        _check(lib().bvc_geometry_get_info(self.h, C.byref(inf)), "bvc_geometry_get_info")
        return inf

    @property
    def boundary_measure(self) -> float:
        return float(self.info().boundary_measure)

    def stats(self, reset=False, stream=None):
        out = (C.c_uint64 * 8)()
        st = lib().bvc_geometry_stats(self.h, out, int(bool(reset)), _stream(stream))
        _check(st, "bvc_geometry_stats", allow=(OK, WARN_WALK_CAP, ERR_BOUNDS))
        return {"steps": int(out[0]), "capped": int(out[1]), "flags": int(out[2]), "nodes": int(out[4]),
                "prims": int(out[5]), "status": st}

    def set_counting(self, on: bool):
        _check(lib().bvc_geometry_set_counting(self.h, int(bool(on))), "bvc_geometry_set_counting")

    def debug_set_link(self, node: int, side: int, link: int, stream=None):
        """bvc_debug_set_link (debug builds only): overwrite one child link of
        the device BVH, to check that the traversal's bounds checks catch it."""
        _check(lib().bvc_debug_set_link(self.h, int(node), int(side), int(link), _stream(stream)),
               "bvc_debug_set_link")

    def close(self):
        if getattr(self, "h", None):
            lib().bvc_geometry_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def query_closest(geom: Geometry, pts: torch.Tensor, want_cp=False, stream=None):
    _dev(pts, torch.float32)
    m = pts.shape[1]
    d2 = torch.empty(m, dtype=torch.float32, device=pts.device)
    prim = torch.empty(m, dtype=torch.int32, device=pts.device)
    cp = torch.empty_like(pts) if want_cp else None
    _check(lib().bvc_query_closest(geom.h, _ptr(pts), m, _ptr(d2), _ptr(prim), _ptr(cp), _stream(stream)),
           "bvc_query_closest")
    return d2, prim, cp


def classify_near(geom: Geometry, pts: torch.Tensor, l: float, stream=None) -> torch.Tensor:
    _dev(pts, torch.float32)
    near = torch.empty(pts.shape[1], dtype=torch.uint8, device=pts.device)
    _check(lib().bvc_classify_near(geom.h, _ptr(pts), pts.shape[1], float(l), _ptr(near), _stream(stream)),
           "bvc_classify_near")
    return near


def sample_boundary(geom: Geometry, n: int, l: float, seed: int, want_elem=True, stream=None):
    """K1: (z, nrm, elem, jac) on the offset boundary at l (1/p = |dOmega| jac)."""
    z = torch.empty((geom.dim, n), dtype=torch.float32, device="cuda")
    nrm = torch.empty_like(z)
    jac = torch.empty(n, dtype=torch.float32, device="cuda")
    elem = torch.empty(n, dtype=torch.int32, device="cuda") if want_elem else None
    _check(lib().bvc_sample_boundary(geom.h, n, float(l), int(seed), _ptr(z), _ptr(nrm), _ptr(jac), _ptr(elem),
                                     _stream(stream)), "bvc_sample_boundary")
    return z, nrm, elem, jac


def walk(geom: Geometry, g_terms, f_terms, starts, nrm, walks: int, eps: float, max_steps: int, seed: int,
         id_base: int = 0, tag: int = TAG_WALK, debug=False, stream=None):
    """bvc_walk: per-walk records (U, and n.grad or grad) as a (planes, n*walks) tensor."""
    _dev(starts, torch.float32)
    n = starts.shape[1]
    planes = 1 if nrm is not None else geom.dim
    rec = torch.empty((1 + planes, n * walks), dtype=torch.float32, device="cuda")
    steps = torch.empty(n * walks, dtype=torch.int32, device="cuda") if debug else None
    prim = torch.empty(n * walks, dtype=torch.int32, device="cuda") if debug else None
    g, f = make_function(g_terms), make_function(f_terms)
    _check(lib().bvc_walk(geom.h, C.byref(g), C.byref(f), _ptr(starts), _ptr(nrm), n, int(walks), float(eps),
                          int(max_steps), int(seed), int(id_base), int(tag), _ptr(rec), _ptr(steps), _ptr(prim),
                          _stream(stream)), "bvc_walk")
    return rec, steps, prim


def reduce_walks(rec: torch.Tensor, n: int, walks: int, mode: int = 0, out=None, stream=None):
    _dev(rec, torch.float32)
    planes = rec.shape[0] - 1
    if rec.dim() != 2 or rec.shape[1] != n * walks:
        raise ValueError(f"records of shape {tuple(rec.shape)} do not hold {n} x {walks} walks")
    if out is None:
        out = torch.zeros((1 + planes, n), dtype=torch.float64, device="cuda")
    _check(lib().bvc_reduce_walks(_ptr(rec), n, int(walks), planes, int(mode), _ptr(out), _stream(stream)),
           "bvc_reduce_walks")
    return out


# ---------------------------------------------------------------- caches
class Cache:
    """Caller-owned device buffers of a bvc_cache (Alg. 1 boundarySamples /
    sourceSamples) as torch tensors."""

    def __init__(self, dim: int, n: int, n_src_cand: int = 0, device="cuda"):
        self.dim, self.n, self.n_src_cand = dim, n, n_src_cand
        self.z = torch.zeros((dim, n), dtype=torch.float32, device=device)
        self.nrm = torch.zeros((dim, n), dtype=torch.float32, device=device)
        self.jac = torch.ones(n, dtype=torch.float32, device=device)
        self.u_hat = torch.zeros(n, dtype=torch.float64, device=device)
        self.dudn_hat = torch.zeros(n, dtype=torch.float64, device=device)
        self.packed = torch.zeros((n, 20), dtype=torch.float32, device=device)
        ms = max(n_src_cand, 1)
        self.src_y = torch.zeros((dim, ms), dtype=torch.float32, device=device)
        self.src_c = torch.zeros(ms, dtype=torch.float64, device=device)
        self.src_packed = torch.zeros((ms, 8), dtype=torch.float32, device=device)
        self.n_src_dev = torch.zeros(1, dtype=torch.int64, device=device)
        self.bnd_measure = 0.0
        self.struct = self._make_struct()

    def _make_struct(self):
        s = CacheStruct()
        s.dim, s.n = self.dim, self.n
        s.z, s.nrm, s.u_hat, s.dudn_hat, s.packed = (_ptr(self.z), _ptr(self.nrm), _ptr(self.u_hat),
                                                     _ptr(self.dudn_hat), _ptr(self.packed))
        s.jac = _ptr(self.jac)
        s.bnd_measure = float(self.bnd_measure)
        s.n_src_cand = self.n_src_cand
        s.src_y, s.src_c, s.src_packed, s.n_src_dev = (_ptr(self.src_y), _ptr(self.src_c), _ptr(self.src_packed),
                                                       _ptr(self.n_src_dev))
        return s

    def set_measure(self, m: float):
        self.bnd_measure = float(m)
        self.struct.bnd_measure = float(m)

    def sync_from_struct(self):
        self.bnd_measure = float(self.struct.bnd_measure)


def n_candidates(dim: int, src_grid) -> int:
    """Source candidates of a grid: G0 x G1 (2D) or G0 x G1 x G2 (3D)."""
    g = list(src_grid) + [0] * (3 - len(src_grid))
    return int(g[0]) * int(g[1]) * (int(g[2]) if dim == 3 else 1)


def cache_opts(n_samples, walks, offset_l, eps, seed, max_steps=1 << 14, walk_id_base=0, src_grid=(0, 0),
               sigma: float = 0.0, clamp_c: float = 0.0):
    o = CacheOpts()
    o.n_samples, o.walks_per_sample, o.max_steps = int(n_samples), int(walks), int(max_steps)
    o.offset_l, o.eps, o.seed, o.walk_id_base = float(offset_l), float(eps), int(seed), int(walk_id_base)
    o.src_grid[0], o.src_grid[1] = int(src_grid[0]), int(src_grid[1])
    o.src_grid[2] = int(src_grid[2]) if len(src_grid) > 2 else 0
    o.sigma = float(sigma)
    o.clamp_c = float(clamp_c)
    return o


def cache_build_workspace_size(geom: Geometry, opts: CacheOpts):
    mn, full = C.c_size_t(), C.c_size_t()
    _check(lib().bvc_cache_build_workspace_size(geom.h, C.byref(opts), C.byref(mn), C.byref(full)),
           "bvc_cache_build_workspace_size")
    return int(mn.value), int(full.value)


def workspace(nbytes: int) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


def cache_build(geom: Geometry, g_terms, f_terms, opts: CacheOpts, cache: Cache, ws: torch.Tensor = None,
                stream=None):
    if ws is None:
        ws = workspace(cache_build_workspace_size(geom, opts)[1])
    g, f = make_function(g_terms), make_function(f_terms)
    _check(lib().bvc_cache_build(geom.h, C.byref(g), C.byref(f), C.byref(opts), C.byref(cache.struct), _ptr(ws),
                                 ws.numel(), _stream(stream)), "bvc_cache_build")
    cache.sync_from_struct()
    return cache


def sample_source(geom: Geometry, f_terms, grid, seed: int, cache: Cache, ws: torch.Tensor = None, stream=None,
                  l: float = 0.0):
    """K4: source candidates kept inside the offset boundary at l (0: the mesh)."""
    need = C.c_size_t()
    _check(lib().bvc_sample_source_workspace_size(cache.n_src_cand, C.byref(need)), "workspace size")
    if ws is None:
        ws = workspace(need.value)
    f = make_function(f_terms)
    gr = (C.c_int32 * 3)(int(grid[0]), int(grid[1]), int(grid[2]) if len(grid) > 2 else 0)
    _check(lib().bvc_sample_source(geom.h, C.byref(f), gr, int(seed), float(l), C.byref(cache.struct), _ptr(ws),
                                   ws.numel(), _stream(stream)), "bvc_sample_source")


def cache_pack(cache: Cache, stream=None):
    _check(lib().bvc_cache_pack(C.byref(cache.struct), _stream(stream)), "bvc_cache_pack")


# ---------------------------------------------------------------- evaluation
class EvalState:
    """Alg. 1 EvaluationPoint running sums for a set of points (dim, m)."""

    def __init__(self, pts: torch.Tensor, grad=True):
        _dev(pts, torch.float32)
        self.x = pts
        self.dim, self.m = pts.shape
        dev = pts.device
        self.u_bnd = torch.zeros(self.m, dtype=torch.float64, device=dev)
        self.u_src = torch.zeros(self.m, dtype=torch.float64, device=dev)
        self.grad_bnd = torch.zeros((self.dim, self.m), dtype=torch.float64, device=dev) if grad else None
        self.grad_src = torch.zeros((self.dim, self.m), dtype=torch.float64, device=dev) if grad else None
        self.counts = torch.zeros(2, dtype=torch.int64, device=dev)
        s = EvalStateStruct()
        s.dim, s.m, s.x = self.dim, self.m, _ptr(pts)
        s.u_bnd, s.u_src = _ptr(self.u_bnd), _ptr(self.u_src)
        s.grad_bnd, s.grad_src = _ptr(self.grad_bnd), _ptr(self.grad_src)
        s.counts = _ptr(self.counts)
        self.struct = s

    def reset(self):
        for t in (self.u_bnd, self.u_src, self.grad_bnd, self.grad_src, self.counts):
            if t is not None:
                t.zero_()


def evaluate_workspace_size(cache: Cache, state: EvalState) -> int:
    b = C.c_size_t()
    _check(lib().bvc_evaluate_workspace_size(C.byref(cache.struct), C.byref(state.struct), C.byref(b)),
           "bvc_evaluate_workspace_size")
    return int(b.value)


def evaluate(cache: Cache, state: EvalState, ws: torch.Tensor = None, stream=None):
    if ws is None:
        ws = workspace(evaluate_workspace_size(cache, state))
    _check(lib().bvc_evaluate(C.byref(cache.struct), C.byref(state.struct), _ptr(ws), ws.numel(), _stream(stream)),
           "bvc_evaluate")


# ---------------------------------------------------------------- regions, clamping
def cache_build_region(domain: Geometry, region: Geometry, g_terms, f_terms, opts: CacheOpts, cache: Cache,
                       ws: torch.Tensor = None, stream=None):
    """Sec. 3.2: samples on the region's boundary, walks in the domain."""
    if ws is None:
        ws = workspace(cache_build_workspace_size(domain, opts)[1])
    g, f = make_function(g_terms), make_function(f_terms)
    _check(lib().bvc_cache_build_region(domain.h, region.h, C.byref(g), C.byref(f), C.byref(opts),
                                        C.byref(cache.struct), _ptr(ws), ws.numel(), _stream(stream)),
           "bvc_cache_build_region")
    return cache


def clamp_correction(domain: Geometry, surface: Geometry, offset_l: float, g_terms, f_terms, clamp_c: float,
                     pts: torch.Tensor, n_dirs: int, walks: int, eps: float, seed: int, max_steps: int = 1 << 14,
                     sigma: float = 0.0, stream=None):
    """Sec. 3.3: the remainder of the clamped double-layer term per point;
    returns (u_corr float64 [m], number of crossings)."""
    _dev(pts, torch.float32)
    m = pts.shape[1]
    b = C.c_size_t()
    _check(lib().bvc_clamp_correction_workspace_size(domain.dim, m, int(n_dirs), int(walks), C.byref(b)),
           "bvc_clamp_correction_workspace_size")
    per = wos_workspace_size(domain.dim, 1, walks)[0]
    ws = workspace(b.value + 4096 * per)
    out = torch.empty(m, dtype=torch.float64, device=pts.device)
    g, f = make_function(g_terms), make_function(f_terms)
    nh = C.c_int64()
    _check(lib().bvc_clamp_correction(domain.h, surface.h, float(offset_l), C.byref(g), C.byref(f), float(sigma),
                                      float(clamp_c), _ptr(pts), m, int(n_dirs), int(walks), float(eps),
                                      int(max_steps), int(seed), _ptr(out), C.byref(nh), _ptr(ws), ws.numel(),
                                      _stream(stream)), "bvc_clamp_correction")
    return out, int(nh.value)


# ---------------------------------------------------------------- walk autotuner
def tune_walks(geom: Geometry, g_terms, f_terms, opts: CacheOpts, stream=None):
    """bvc_tune_walks: returns (blocks per SM, chunk, best ms) and keeps the
    shape in the geometry."""
    b = C.c_size_t()
    _check(lib().bvc_tune_walks_workspace_size(geom.h, C.byref(opts), C.byref(b)), "bvc_tune_walks_workspace_size")
    ws = workspace(b.value)
    g, f = make_function(g_terms), make_function(f_terms)
    shape = (C.c_int32 * 2)()
    ms = C.c_float()
    _check(lib().bvc_tune_walks(geom.h, C.byref(g), C.byref(f), C.byref(opts), _ptr(ws), ws.numel(),
                                _stream(stream), shape, C.byref(ms)), "bvc_tune_walks")
    return int(shape[0]), int(shape[1]), float(ms.value)


def set_walk_shape(geom: Geometry, blocks_per_sm: int, chunk: int):
    _check(lib().bvc_geometry_set_walk_shape(geom.h, int(blocks_per_sm), int(chunk)), "bvc_geometry_set_walk_shape")


# ---------------------------------------------------------------- differentiation
def cache_build_vg(geom: Geometry, g_vertex: torch.Tensor, f_terms, opts: CacheOpts, cache: Cache,
                   ws: torch.Tensor = None, stream=None):
    """bvc_cache_build_vg: g from vertex values (CUDA float32 [n_verts])."""
    _dev(g_vertex, torch.float32)
    if ws is None:
        ws = workspace(cache_build_workspace_size(geom, opts)[1])
    f = make_function(f_terms)
    _check(lib().bvc_cache_build_vg(geom.h, _ptr(g_vertex), C.byref(f), C.byref(opts), C.byref(cache.struct),
                                    _ptr(ws), ws.numel(), _stream(stream)), "bvc_cache_build_vg")
    return cache


def evaluate_adjoint(cache: Cache, pts: torch.Tensor, lam: torch.Tensor, stream=None):
    """dL/du^, dL/d(du/dn^) per boundary sample and dL/dc per source
    candidate from lam = dL/du at the points (CUDA float64 [m])."""
    _dev(pts, torch.float32)
    _dev(lam, torch.float64)
    m = pts.shape[1]
    nb = C.c_size_t()
    _check(lib().bvc_evaluate_adjoint_workspace_size(m, C.byref(nb)), "bvc_evaluate_adjoint_workspace_size")
    ws = workspace(nb.value)
    dev = pts.device
    adj_u = torch.empty(cache.n, dtype=torch.float64, device=dev)
    adj_q = torch.empty(cache.n, dtype=torch.float64, device=dev)
    adj_s = torch.zeros(max(cache.n_src_cand, 1), dtype=torch.float64, device=dev) if cache.n_src_cand else None
    _check(lib().bvc_evaluate_adjoint(C.byref(cache.struct), _ptr(pts), m, _ptr(lam), _ptr(adj_u), _ptr(adj_q),
                                      _ptr(adj_s), _ptr(ws), ws.numel(), _stream(stream)), "bvc_evaluate_adjoint")
    return adj_u, adj_q, adj_s


def cache_adjoint(geom: Geometry, f_terms, opts: CacheOpts, cache: Cache, adj_u, adj_q, adj_s, grad_gv: torch.Tensor,
                  grad_amp: torch.Tensor, ws: torch.Tensor = None, stream=None):
    """Adds dL/dg_vertex and dL/dA (FP64) by replaying the cache walks."""
    _dev(grad_gv, torch.float64)
    _dev(grad_amp, torch.float64)
    if grad_amp.numel() < 8:
        raise ValueError("grad_amp must hold 8 entries")
    if ws is None:
        mn, full = C.c_size_t(), C.c_size_t()
        _check(lib().bvc_cache_adjoint_workspace_size(geom.h, C.byref(opts), C.byref(mn), C.byref(full)),
               "bvc_cache_adjoint_workspace_size")
        ws = workspace(full.value)
    f = make_function(f_terms)
    _check(lib().bvc_cache_adjoint(geom.h, C.byref(f), C.byref(opts), C.byref(cache.struct), _ptr(adj_u),
                                   _ptr(adj_q), _ptr(adj_s), _ptr(grad_gv), _ptr(grad_amp), _ptr(ws), ws.numel(),
                                   _stream(stream)), "bvc_cache_adjoint")


def bump_terms(kind: int, sigma: float, centres, amps) -> list:
    """One GAUSS / GAUSS_LAPLACIAN term [s, A_1, c_1, A_2, c_2, ...]."""
    co = [float(sigma)]
    for a, c in zip(amps, centres):
        co.append(float(a))
        co.extend(float(v) for v in c)
    return [(kind, co)]


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g_vertex, amps, solver):
        cache = solver._forward(g_vertex, amps)
        ctx.solver, ctx.cache = solver, cache
        ctx.amps = amps.detach().cpu().numpy()
        return solver._u

    @staticmethod
    def backward(ctx, lam):
        s = ctx.solver
        gg, ga = s._backward(ctx.cache, ctx.amps, lam.contiguous().double())
        return gg, ga[:len(ctx.amps)], None


class DiffSolver:
    """u at fixed interior points as a differentiable function of the vertex
    values of g and the bump amplitudes of f, with fixed seeds (BVC forward:
    bvc_cache_build_vg + bvc_evaluate; backward: bvc_evaluate_adjoint +
    bvc_cache_adjoint).  bumps: (kind, sigma, centres [nb][dim]) or None."""

    def __init__(self, geom: Geometry, pts: torch.Tensor, n_samples: int, walks: int, offset_l: float, eps: float,
                 seed: int, bumps=None, src_grid=(0, 0), max_steps: int = 1 << 14):
        self.geom, self.pts = geom, pts
        self.dim = geom.dim
        self.bumps = bumps
        self.opts = cache_opts(n_samples, walks, offset_l, eps, seed, max_steps=max_steps,
                               src_grid=src_grid if bumps else (0, 0))
        self.n_src = n_candidates(self.dim, self.opts.src_grid)
        self.ws = workspace(cache_build_workspace_size(geom, self.opts)[1])
        self.n_verts = geom.info().n_verts

    def _f_terms(self, amps):
        if not self.bumps:
            return []
        kind, sigma, centres = self.bumps
        return bump_terms(kind, sigma, centres, amps)

    def _forward(self, g_vertex, amps):
        cache = Cache(self.dim, self.opts.n_samples, n_src_cand=self.n_src)
        f = self._f_terms(amps.detach().cpu().numpy() if amps is not None else [])
        # the kept source candidates depend on the geometry, grid and seed
        # only: classify them once and re-weight them on later solves
        if self.n_src and getattr(self, "_src", None) is not None:
            cache.src_y.copy_(self._src[0])
            cache.n_src_dev.copy_(self._src[1])
            self.opts.reuse_sources = 1
        cache_build_vg(self.geom, g_vertex.detach().float().contiguous(), f, self.opts, cache, self.ws)
        self.opts.reuse_sources = 0
        if self.n_src and getattr(self, "_src", None) is None:
            self._src = (cache.src_y.clone(), cache.n_src_dev.clone())
        st = EvalState(self.pts, grad=False)
        evaluate(cache, st)
        self._u, _ = get_solution(st)
        return cache

    def _backward(self, cache, amps, lam):
        adj_u, adj_q, adj_s = evaluate_adjoint(cache, self.pts, lam)
        gg = torch.zeros(self.n_verts, dtype=torch.float64, device=lam.device)
        ga = torch.zeros(8, dtype=torch.float64, device=lam.device)
        cache_adjoint(self.geom, self._f_terms(amps), self.opts, cache, adj_u, adj_q, adj_s, gg, ga)
        return gg, ga

    def __call__(self, g_vertex: torch.Tensor, amps: torch.Tensor = None):
        if amps is None:
            amps = torch.zeros(0, dtype=torch.float64, device=g_vertex.device)
        return _Solve.apply(g_vertex, amps, self)


def get_solution(state: EvalState, u=None, grad=None, stream=None):
    if u is None:
        u = torch.empty(state.m, dtype=torch.float64, device=state.x.device)
    if grad is None and state.grad_bnd is not None:
        grad = torch.empty((state.dim, state.m), dtype=torch.float64, device=state.x.device)
    _check(lib().bvc_get_solution(C.byref(state.struct), _ptr(u), _ptr(grad), _stream(stream)), "bvc_get_solution")
    return u, grad


def wos_workspace_size(dim: int, m: int, walks: int):
    mn, full = C.c_size_t(), C.c_size_t()
    _check(lib().wos_estimate_workspace_size(dim, m, walks, C.byref(mn), C.byref(full)), "wos workspace size")
    return int(mn.value), int(full.value)


def tune_gather(cache: Cache, state: EvalState, ws: torch.Tensor = None, stream=None):
    """bvc_tune_gather: returns ((boundary, source) points per thread, ms);
    the state's sums are cleared."""
    if ws is None:
        ws = workspace(evaluate_workspace_size(cache, state))
    pts = (C.c_int32 * 2)()
    ms = C.c_float()
    _check(lib().bvc_tune_gather(C.byref(cache.struct), C.byref(state.struct), _ptr(ws), ws.numel(),
                                 _stream(stream), pts, C.byref(ms)), "bvc_tune_gather")
    return (int(pts[0]), int(pts[1])), float(ms.value)


def set_gather_shape(dim: int, kind: int, pts: int):
    _check(lib().bvc_set_gather_shape(int(dim), int(kind), int(pts)), "bvc_set_gather_shape")


def last_error() -> int:
    """bvc_last_error: the calling thread's last status other than OK (cleared)."""
    return int(lib().bvc_last_error())


def debug_build() -> bool:
    """True when the loaded library is the debug build (BVC_DEBUG=1)."""
    return bool(lib().bvc_debug_build())


def eval_state_reset(state: EvalState, stream=None):
    _check(lib().bvc_eval_state_reset(C.byref(state.struct), _stream(stream)), "bvc_eval_state_reset")


def wos_estimate(geom: Geometry, g_terms, f_terms, state: EvalState, walks: int, eps: float, max_steps: int,
                 seed: int, id_base: int = 0, ws: torch.Tensor = None, stream=None, sigma: float = 0.0):
    """Pointwise walk on spheres: adds `walks` walks per point of `state` to
    its running sums (finalise with get_solution).  sigma > 0: the screened
    equation (Delta - sigma) u = 0 (wos_estimate_sigma)."""
    if ws is None:
        ws = workspace(wos_workspace_size(state.dim, state.m, walks)[1])
    g, f = make_function(g_terms), make_function(f_terms)
    if sigma:
        _check(lib().wos_estimate_sigma(geom.h, C.byref(g), C.byref(f), float(sigma), C.byref(state.struct),
                                        int(walks), float(eps), int(max_steps), int(seed), int(id_base), _ptr(ws),
                                        ws.numel(), _stream(stream)), "wos_estimate_sigma")
        return state
    _check(lib().wos_estimate(geom.h, C.byref(g), C.byref(f), C.byref(state.struct), int(walks), float(eps),
                              int(max_steps), int(seed), int(id_base), _ptr(ws), ws.numel(), _stream(stream)),
           "wos_estimate")
    return state


def wos_estimate_static_scratch(geom: Geometry, g_terms, f_terms, state: EvalState, walks: int, eps: float,
                                max_steps: int, seed: int, id_base: int = 0, stream=None):
    """wos_estimate for callers that cannot allocate: the library's own static
    16 MiB device scratch replaces the workspace (see include/bvc.h)."""
    g, f = make_function(g_terms), make_function(f_terms)
    _check(lib().wos_estimate_static_scratch(geom.h, C.byref(g), C.byref(f), C.byref(state.struct), int(walks),
                                             float(eps), int(max_steps), int(seed), int(id_base), _stream(stream)),
           "wos_estimate_static_scratch")
    return state


# ---------------------------------------------------------------- many right-hand sides
MULTI_GROUP = 32


def poly_terms(dim: int) -> int:
    return int(lib().bvc_poly_terms(dim))


MAX_BUMPS = 8


class MultiCache:
    """Caller-owned device buffers of a bvc_multi_cache (k right-hand sides);
    n_src_cand > 0 adds the source part (bvc_multi_cache_build_source)."""

    def __init__(self, dim: int, n: int, k: int, n_src_cand: int = 0, device="cuda"):
        self.dim, self.n, self.k, self.n_src_cand = dim, n, k, n_src_cand
        t = poly_terms(dim)
        groups = (k + MULTI_GROUP - 1) // MULTI_GROUP
        self.z = torch.zeros((dim, n), dtype=torch.float32, device=device)
        self.nrm = torch.zeros((dim, n), dtype=torch.float32, device=device)
        self.jac = torch.ones(n, dtype=torch.float32, device=device)
        self.mom_u = torch.zeros((n, t), dtype=torch.float64, device=device)
        self.mom_q = torch.zeros((n, t), dtype=torch.float64, device=device)
        self.u_hat = torch.zeros((k, n), dtype=torch.float64, device=device)
        self.dudn_hat = torch.zeros((k, n), dtype=torch.float64, device=device)
        self.packed = torch.zeros((groups, n + n_src_cand, 8 + 2 * MULTI_GROUP), dtype=torch.float32, device=device)
        st = MultiCacheStruct()
        st.dim, st.n, st.k = dim, n, k
        st.z, st.nrm, st.mom_u, st.mom_q = _ptr(self.z), _ptr(self.nrm), _ptr(self.mom_u), _ptr(self.mom_q)
        st.jac = _ptr(self.jac)
        st.u_hat, st.dudn_hat, st.packed = _ptr(self.u_hat), _ptr(self.dudn_hat), _ptr(self.packed)
        st.bnd_measure = 0.0
        if n_src_cand > 0:
            self.mom_su = torch.zeros((n, MAX_BUMPS), dtype=torch.float64, device=device)
            self.mom_sq = torch.zeros((n, MAX_BUMPS), dtype=torch.float64, device=device)
            self.src_y = torch.zeros((dim, n_src_cand), dtype=torch.float32, device=device)
            self.src_psi = torch.zeros((n_src_cand, MAX_BUMPS), dtype=torch.float32, device=device)
            self.n_src_dev = torch.zeros(1, dtype=torch.int64, device=device)
            st.mom_su, st.mom_sq = _ptr(self.mom_su), _ptr(self.mom_sq)
            st.n_src_cand = n_src_cand
            st.src_y, st.src_psi, st.n_src_dev = _ptr(self.src_y), _ptr(self.src_psi), _ptr(self.n_src_dev)
        self.struct = st

    @property
    def n_bumps(self) -> int:
        return int(self.struct.n_bumps)


def multi_cache_build_workspace_size(geom: Geometry, n: int, walks: int):
    mn, full = C.c_size_t(), C.c_size_t()
    _check(lib().bvc_multi_cache_build_workspace_size(geom.h, n, walks, C.byref(mn), C.byref(full)),
           "bvc_multi_cache_build_workspace_size")
    return int(mn.value), int(full.value)


def multi_cache_build(geom: Geometry, coeffs: torch.Tensor, opts: CacheOpts, cache: MultiCache,
                      ws: torch.Tensor = None, stream=None):
    """coeffs: CUDA float64 [k][poly_terms(dim)] monomial coefficients of each g_k."""
    _dev(coeffs, torch.float64)
    if tuple(coeffs.shape) != (cache.k, poly_terms(cache.dim)):
        raise ValueError("coefficients must be [k][poly_terms(dim)]")
    if ws is None:
        ws = workspace(multi_cache_build_workspace_size(geom, cache.n, opts.walks_per_sample)[1])
    _check(lib().bvc_multi_cache_build(geom.h, _ptr(coeffs), C.byref(opts), C.byref(cache.struct), _ptr(ws),
                                       ws.numel(), _stream(stream)), "bvc_multi_cache_build")
    return cache


def multi_cache_build_source(geom: Geometry, shape_terms, coeffs: torch.Tensor, opts: CacheOpts, cache: MultiCache,
                             ws: torch.Tensor = None, stream=None):
    """bvc_multi_cache_build_source.  shape_terms: one (GAUSS | GAUSS_LAPLACIAN,
    coeffs) term whose B bumps are the source basis; coeffs: CUDA float64
    [k][poly_terms(dim) + B] (g_k's monomial coefficients, then f_k's bump
    amplitudes)."""
    _dev(coeffs, torch.float64)
    if len(shape_terms) != 1:
        raise ValueError("the source shape is one GAUSS or GAUSS_LAPLACIAN term")
    kind, cs = shape_terms[0]
    head = 3 if kind == FN_GAUSS_LAPLACIAN else 1
    nb = (len(cs) - head) // (1 + cache.dim)
    if tuple(coeffs.shape) != (cache.k, poly_terms(cache.dim) + nb):
        raise ValueError("coefficients must be [k][poly_terms(dim) + bumps]")
    if ws is None:
        mn, full = C.c_size_t(), C.c_size_t()
        _check(lib().bvc_multi_cache_build_source_workspace_size(geom.h, C.byref(opts), C.byref(mn), C.byref(full)),
               "bvc_multi_cache_build_source_workspace_size")
        ws = workspace(int(full.value))
    f = make_function(shape_terms)
    _check(lib().bvc_multi_cache_build_source(geom.h, C.byref(f), _ptr(coeffs), C.byref(opts), C.byref(cache.struct),
                                              _ptr(ws), ws.numel(), _stream(stream)), "bvc_multi_cache_build_source")
    return cache


def multi_cache_project(coeffs: torch.Tensor, cache: MultiCache, stream=None):
    _dev(coeffs, torch.float64)
    if tuple(coeffs.shape) != (cache.k, poly_terms(cache.dim) + cache.n_bumps):
        raise ValueError("coefficients must be [k][poly_terms(dim) + bumps]")
    _check(lib().bvc_multi_cache_project(_ptr(coeffs), C.byref(cache.struct), _stream(stream)),
           "bvc_multi_cache_project")


def evaluate_multi(cache: MultiCache, pts: torch.Tensor, u: torch.Tensor = None, stream=None):
    """u[k][x] for every right-hand side (Eq. 3, plus Eq. 4's source term
    when the cache has one)."""
    _dev(pts, torch.float32)
    m = pts.shape[1]
    if u is None:
        u = torch.empty((cache.k, m), dtype=torch.float64, device=pts.device)
    _check(lib().bvc_evaluate_multi(C.byref(cache.struct), _ptr(pts), m, _ptr(u), _stream(stream)),
           "bvc_evaluate_multi")
    return u


class Batch:
    """bvc_batch_create / bvc_batch_destroy: independent problems on several
    meshes of one dimension, walked and gathered in one launch each.
    meshes: list of (Geometry, n_samples, offset_l, eps, n_points)."""

    def __init__(self, meshes, walks: int, max_steps: int, k: int, stream=None):
        self.geoms = [m[0] for m in meshes]  # keep the borrowed geometries alive
        arr = (BatchMeshStruct * len(meshes))()
        for j, (g, n, l, eps, m) in enumerate(meshes):
            arr[j].geom, arr[j].n_samples, arr[j].offset_l = g.h.value, int(n), float(l)
            arr[j].eps, arr[j].n_points = float(eps), int(m)
        h = C.c_void_p()
        _check(lib().bvc_batch_create(C.cast(arr, C.c_void_p), len(meshes), int(walks), int(max_steps), int(k),
                                      _stream(stream), C.byref(h)), "bvc_batch_create")
        self.h = h
        dim, n, m = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().bvc_batch_get_info(h, C.byref(dim), C.byref(n), C.byref(m)), "bvc_batch_get_info")
        self.dim, self.n_total, self.m_total, self.k = dim.value, n.value, m.value, int(k)
        self.sample_offsets = np.concatenate([[0], np.cumsum([int(x[1]) for x in meshes])])
        self.point_offsets = np.concatenate([[0], np.cumsum([int(x[4]) for x in meshes])])

    def workspace_size(self):
        mn, full = C.c_size_t(), C.c_size_t()
        _check(lib().bvc_batch_build_workspace_size(self.h, C.byref(mn), C.byref(full)),
               "bvc_batch_build_workspace_size")
        return int(mn.value), int(full.value)

    def cache(self, device="cuda") -> MultiCache:
        return MultiCache(self.dim, self.n_total, self.k, device=device)

    def build(self, coeffs: torch.Tensor, seed, cache: MultiCache, ws: torch.Tensor = None, stream=None):
        """coeffs: CUDA float64 [meshes][k][poly_terms(dim)].  seed: an int,
        or a CUDA int64 tensor of one element read when the kernels run (a
        captured graph then replays with the value it holds)."""
        _dev(coeffs, torch.float64)
        if tuple(coeffs.shape) != (len(self.geoms), self.k, poly_terms(self.dim)):
            raise ValueError("coefficients must be [meshes][k][poly_terms(dim)]")
        if isinstance(seed, torch.Tensor):
            _dev(seed, torch.int64)
            if seed.numel() != 1:
                raise ValueError("seed tensor must hold one element")
            seed_t = seed
        else:
            if not hasattr(self, "_seed"):
                self._seed = torch.zeros(1, dtype=torch.int64, device=coeffs.device)
            self._seed.fill_(int(seed))
            seed_t = self._seed
        if ws is None:
            ws = workspace(self.workspace_size()[1])
        _check(lib().bvc_batch_build(self.h, _ptr(coeffs), _ptr(seed_t), C.byref(cache.struct), _ptr(ws),
                                     ws.numel(), _stream(stream)), "bvc_batch_build")
        return cache

    def set_counting(self, on: bool):
        _check(lib().bvc_batch_set_counting(self.h, 1 if on else 0), "bvc_batch_set_counting")

    def stats(self, reset=False, stream=None):
        out = (C.c_uint64 * 8)()
        st = lib().bvc_batch_stats(self.h, out, 1 if reset else 0, _stream(stream))
        _check(st, "bvc_batch_stats", allow=(OK, WARN_WALK_CAP, ERR_BOUNDS))
        return {"steps": out[0], "capped": out[1], "flags": out[2], "nodes": out[4], "prims": out[5]}

    def project(self, coeffs: torch.Tensor, cache: MultiCache, stream=None):
        _dev(coeffs, torch.float64)
        if tuple(coeffs.shape) != (len(self.geoms), self.k, poly_terms(self.dim)):
            raise ValueError("coefficients must be [meshes][k][poly_terms(dim)]")
        _check(lib().bvc_batch_project(self.h, _ptr(coeffs), C.byref(cache.struct), _stream(stream)),
               "bvc_batch_project")

    def evaluate(self, cache: MultiCache, pts: torch.Tensor, u: torch.Tensor = None, stream=None):
        """pts: CUDA float32 [dim][m_total]; returns u [k][m_total] (float64)."""
        _dev(pts, torch.float32)
        if tuple(pts.shape) != (self.dim, self.m_total):
            raise ValueError("points must be [dim][m_total]")
        if u is None:
            u = torch.empty((self.k, self.m_total), dtype=torch.float64, device=pts.device)
        _check(lib().bvc_batch_evaluate(self.h, C.byref(cache.struct), _ptr(pts), _ptr(u), _stream(stream)),
               "bvc_batch_evaluate")
        return u

    def close(self):
        if getattr(self, "h", None):
            lib().bvc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def profile_begin():
    _check(lib().bvc_profile_begin(), "bvc_profile_begin")


def profile_end():
    """Per-kernel {name: (launches, total_ms)} since profile_begin (synchronises)."""
    out = (KernelTime * 64)()
    n = C.c_int32()
    _check(lib().bvc_profile_end(out, 64, C.byref(n)), "bvc_profile_end")
    return {out[i].name.decode(): (int(out[i].launches), float(out[i].total_ms)) for i in range(n.value)}


def gather_status(reset=False):
    f = C.c_uint64()
    st = lib().bvc_gather_status(C.byref(f), int(bool(reset)))
    return int(f.value), st


# ---------------------------------------------------------------- mixed boundaries (WoSt)
def make_neumann(h) -> NeumannStruct:
    """h = (value_terms, potential_terms): Neumann data value(z) + n . grad potential(z)."""
    hv, hp = (h or ([], []))
    out = NeumannStruct()
    fv, fp = make_function(hv), make_function(hp)
    out.value, out.potential = fv, fp
    out._keep = (fv, fp)
    return out


class _BorrowedGeometry(Geometry):
    """A geometry handle owned by another object (not destroyed here)."""

    def __init__(self, h, dim):
        self.h = h
        self.dim = dim

    def close(self):
        self.h = None


class Mixed:
    """bvc_mixed_create / bvc_mixed_destroy: a boundary whose elements are
    Dirichlet (neumann[e] == 0) or Neumann, with its walk-on-stars trees."""

    def __init__(self, V, F, neumann, stream=None):
        V = np.ascontiguousarray(V, dtype=np.float32)
        F = np.ascontiguousarray(F, dtype=np.int32)
        fl = np.ascontiguousarray(np.asarray(neumann) != 0, dtype=np.uint8)
        if fl.shape[0] != F.shape[0]:
            raise ValueError("one Neumann flag per element")
        self.dim = int(V.shape[1])
        h = C.c_void_p()
        _check(lib().bvc_mixed_create(self.dim, V.ctypes.data_as(C.c_void_p), V.shape[0],
                                      F.ctypes.data_as(C.c_void_p), F.shape[0], fl.ctypes.data_as(C.c_void_p),
                                      _stream(stream), C.byref(h)), "bvc_mixed_create")
        self.h = h
        w, d, n = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(lib().bvc_mixed_geometries(self.h, C.byref(w), C.byref(d), C.byref(n)), "bvc_mixed_geometries")
        self.whole = _BorrowedGeometry(w, self.dim)
        self.dirichlet = _BorrowedGeometry(d, self.dim)
        self.neumann = _BorrowedGeometry(n, self.dim) if n.value else None

    def info(self) -> MixedInfo:
        inf = MixedInfo()
        _check(lib().bvc_mixed_get_info(self.h, C.byref(inf)), "bvc_mixed_get_info")
        return inf

    def set_silhouette_gap(self, gap: float):
        """bvc_mixed_set_silhouette_gap: 0 = exact silhouette distances; in
        (0, 1) a certified lower bound within the factor 1 - gap."""
        _check(lib().bvc_mixed_set_silhouette_gap(self.h, float(gap)), "bvc_mixed_set_silhouette_gap")

    def close(self):
        if getattr(self, "h", None):
            for g in (self.whole, self.dirichlet, self.neumann):
                if g is not None:
                    g.close()
            lib().bvc_mixed_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mixed_query(m: Mixed, pts: torch.Tensor, stream=None):
    """Distances to the Dirichlet part and to the closest silhouette."""
    _dev(pts, torch.float32)
    n = pts.shape[1]
    dd = torch.empty(n, dtype=torch.float32, device=pts.device)
    ds = torch.empty(n, dtype=torch.float32, device=pts.device)
    _check(lib().bvc_mixed_query(m.h, _ptr(pts), n, _ptr(dd), _ptr(ds), _stream(stream)), "bvc_mixed_query")
    return dd, ds


def mixed_rays(m: Mixed, org: torch.Tensor, dirs: torch.Tensor, tmax: float, skip: torch.Tensor = None,
               stream=None):
    """First crossing (t, Neumann element) of each ray with the Neumann part."""
    _dev(org, torch.float32)
    _dev(dirs, torch.float32)
    n = org.shape[1]
    t = torch.empty(n, dtype=torch.float32, device=org.device)
    e = torch.empty(n, dtype=torch.int32, device=org.device)
    _check(lib().bvc_mixed_rays(m.h, _ptr(org), _ptr(dirs), _ptr(skip), n, float(tmax), _ptr(t), _ptr(e),
                                _stream(stream)), "bvc_mixed_rays")
    return t, e


def mixed_walk(m: Mixed, g_terms, h, f_terms, starts, start_elem, nrm, walks: int, eps: float, max_steps: int,
               seed: int, id_base: int = 0, tag: int = TAG_WALK, debug=False, stream=None, sigma: float = 0.0):
    """bvc_mixed_walk: per-walk records (U, and n.grad / h or grad).
    sigma > 0: the screened equation (bvc_mixed_walk_sigma)."""
    _dev(starts, torch.float32)
    n = starts.shape[1]
    planes = 1 if nrm is not None else m.dim
    rec = torch.empty((1 + planes, n * walks), dtype=torch.float32, device="cuda")
    steps = torch.empty(n * walks, dtype=torch.int32, device="cuda") if debug else None
    prim = torch.empty(n * walks, dtype=torch.int32, device="cuda") if debug else None
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    g, f, hn = make_function(g_terms), make_function(f_terms), make_neumann(h)
    if sigma:
        _check(lib().bvc_mixed_walk_sigma(m.h, C.byref(g), C.byref(hn), C.byref(f), float(sigma), _ptr(starts),
                                          _ptr(start_elem), _ptr(nrm), n, int(walks), float(eps), int(max_steps),
                                          int(seed), int(id_base), int(tag), _ptr(rec), _ptr(steps), _ptr(prim),
                                          _ptr(counter), _stream(stream)), "bvc_mixed_walk_sigma")
        return rec, steps, prim
    _check(lib().bvc_mixed_walk(m.h, C.byref(g), C.byref(hn), C.byref(f), _ptr(starts), _ptr(start_elem), _ptr(nrm),
                                n, int(walks), float(eps), int(max_steps), int(seed), int(id_base), int(tag),
                                _ptr(rec), _ptr(steps), _ptr(prim), _ptr(counter), _stream(stream)),
           "bvc_mixed_walk")
    return rec, steps, prim


def mixed_cache_build_workspace_size(m: Mixed, opts: CacheOpts):
    mn, full = C.c_size_t(), C.c_size_t()
    _check(lib().bvc_mixed_cache_build_workspace_size(m.h, C.byref(opts), C.byref(mn), C.byref(full)),
           "bvc_mixed_cache_build_workspace_size")
    return int(mn.value), int(full.value)


def mixed_cache_build(m: Mixed, g_terms, h, f_terms, opts: CacheOpts, cache: Cache, ws: torch.Tensor = None,
                      stream=None):
    """The mixed cache (Sec. 3.2): Neumann samples on the boundary with
    du/dn = h, Dirichlet samples at offset l, u by walks on stars."""
    if ws is None:
        ws = workspace(mixed_cache_build_workspace_size(m, opts)[1])
    g, f, hn = make_function(g_terms), make_function(f_terms), make_neumann(h)
    _check(lib().bvc_mixed_cache_build(m.h, C.byref(g), C.byref(hn), C.byref(f), C.byref(opts),
                                       C.byref(cache.struct), _ptr(ws), ws.numel(), _stream(stream)),
           "bvc_mixed_cache_build")
    cache.sync_from_struct()
    return cache


def wost_estimate(m: Mixed, g_terms, h, f_terms, state: EvalState, walks: int, eps: float, max_steps: int,
                  seed: int, id_base: int = 0, ws: torch.Tensor = None, stream=None, sigma: float = 0.0):
    """Pointwise walk on stars: adds `walks` walks per point to the state's
    running sums (finalise with get_solution).  sigma > 0: the screened
    equation (wost_estimate_sigma)."""
    if ws is None:
        ws = workspace(wos_workspace_size(state.dim, state.m, walks)[1])
    g, f, hn = make_function(g_terms), make_function(f_terms), make_neumann(h)
    if sigma:
        _check(lib().wost_estimate_sigma(m.h, C.byref(g), C.byref(hn), C.byref(f), float(sigma),
                                         C.byref(state.struct), int(walks), float(eps), int(max_steps), int(seed),
                                         int(id_base), _ptr(ws), ws.numel(), _stream(stream)), "wost_estimate_sigma")
        return state
    _check(lib().wost_estimate(m.h, C.byref(g), C.byref(hn), C.byref(f), C.byref(state.struct), int(walks),
                               float(eps), int(max_steps), int(seed), int(id_base), _ptr(ws), ws.numel(),
                               _stream(stream)), "wost_estimate")
    return state


def wait_selftest(limit_ns: int = 1_000_000, stream=None):
    """Runs the bounded-wait self-test (a wait that nothing completes)."""
    _check(lib().bvc_wait_selftest(int(limit_ns), _stream(stream)), "bvc_wait_selftest")
